"""The work partitioning (pg_set_tuning, the autotuner's tables) changes how
the valuation is computed, never what: under every candidate value of every
parameter the solves equal the CPU oracle's bit for bit. A table loaded from
a file applies its entries by game size, and malformed tables are refused."""
import numpy as np
import pytest

from paper_1705_02313_gb300 import gen, tune

from test_gpu_deep import climbing_game
from test_gpu_parity import assert_same, oracle_solution

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    from paper_1705_02313_gb300 import build, pg as _pg
    build.build()
    return _pg


@pytest.fixture(scope="module")
def ctx(pg):
    c = pg.pg_ctx_create(0, tuning=False)
    yield c
    pg.pg_ctx_destroy(c)


def settings():
    """The defaults, every candidate of each parameter alone, and a few mixes."""
    out = [dict(tune.DEFAULTS)]
    for name, values in tune.CANDIDATES.items():
        for v in values:
            if v != tune.DEFAULTS[name]:
                out.append(dict(tune.DEFAULTS, **{name: v}))
    out.append(dict(walk_cap=16, switch_block=512, loop_ranks=1, deep_cut=8, ruler_bits=3))
    out.append(dict(walk_cap=128, switch_block=128, loop_ranks=0, deep_cut=256, ruler_bits=7))
    return out


def test_every_setting_gives_the_oracles_results(pg, ctx):
    games = [gen.random_game(20000, 2, 5, 3), gen.ladder_game(5000, 6), climbing_game(3000, 2, 0.05),
             gen.random_game(1000, 1, 4, 8)]
    wants = [oracle_solution(g)[2] for g in games]
    try:
        for st in settings():
            pg.pg_set_tuning_table(ctx, [(2**62, st)])
            for g, want in zip(games, wants):
                got = pg.solve_arrays(ctx, g.n, *g.arrays())
                assert_same(got, want, "%s n=%d" % (st, g.n))
    finally:
        pg.pg_set_tuning_table(ctx, [])


def loop_kernels(pg, ctx, g):
    """Kernel classes that ran during a timed (host-loop) solve of g."""
    pg.pg_set_timing(ctx, True)
    game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
    try:
        pg.pg_solve(ctx, game, win=np.empty(g.n, np.uint8))
        return {k for k, v in pg.pg_kernel_stats(game).items() if v[2] > 0}
    finally:
        pg.pg_game_free(game)
        pg.pg_set_timing(ctx, False)


def test_a_table_file_applies_by_size(pg, ctx, tmp_path):
    path = tmp_path / "table.txt"
    path.write_text(tune.table_text([(5000, dict(tune.DEFAULTS, loop_ranks=1, walk_cap=16)),
                                     (2**62, dict(tune.DEFAULTS, switch_block=512))], "test"))
    pg.pg_load_tuning(ctx, str(path))
    try:
        small, large = gen.random_game(1000, 1, 4, 1), gen.random_game(30000, 2, 5, 2)
        assert "classify" not in loop_kernels(pg, ctx, small)  # ranks every iteration: no comparison passes
        assert "classify" in loop_kernels(pg, ctx, large)
        for g in (small, large):
            assert_same(pg.solve_arrays(ctx, g.n, *g.arrays()), oracle_solution(g)[2], "n=%d" % g.n)
    finally:
        pg.pg_set_tuning_table(ctx, [])


@pytest.mark.parametrize("text", ["1000 64 5 64 256\n",                       # a field missing
                                  "1000 64 5 63 256 0\n",                     # walk cap not a candidate
                                  "1000 64 5 64 256 0\n900 64 5 64 256 0\n",  # max_ids not increasing
                                  "1000 64 17 64 256 0\n"])                   # ruler bits out of range
def test_malformed_tables_are_refused(pg, ctx, tmp_path, text):
    path = tmp_path / "bad.txt"
    path.write_text("# a comment\n" + text)
    with pytest.raises(pg.PgError) as e:
        pg.pg_load_tuning(ctx, str(path))
    assert e.value.code == pg.PG_EINVAL
    with pytest.raises(pg.PgError):
        pg.pg_load_tuning(ctx, str(tmp_path / "missing.txt"))
