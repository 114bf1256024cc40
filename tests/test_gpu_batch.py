"""GPU parity of pg_solve_batch: every game of a batch must get exactly the
result (strategies, winners, valuations, per-game iteration counts) that the
oracle computes for it alone, and the same as pg_solve gives for it alone."""
import numpy as np
import pytest

from oracle import o2
from paper_1705_02313_gb300 import gen

pytestmark = pytest.mark.gpu

KEYS = ["win", "sigma", "tau", "val_class", "val_depth", "val_rank"]


@pytest.fixture(scope="module")
def pg():
    from paper_1705_02313_gb300 import build, pg as _pg
    build.build()
    return _pg


@pytest.fixture(scope="module")
def ctx(pg):
    c = pg.pg_ctx_create(0)
    yield c
    pg.pg_ctx_destroy(c)


def mixed_games(count, seed):
    rng = np.random.default_rng(seed)
    games = []
    for i in range(count):
        kind = i % 4
        n = int(np.exp(rng.uniform(np.log(2), np.log(20000))))
        if kind == 3 and n >= 2:
            games.append(gen.ladder_game(n, seed=1000 + i))
        else:
            dmin, dmax = [(1, 4), (2, 6), (2, 8)][kind]
            games.append(gen.random_game(n, dmin, dmax, seed=gen.batch_seed(i)))
    return games


def run_batch(pg, ctx, games, device=False):
    packed = pg.pack_games(games)
    vb, eb = packed[0], packed[1]
    arrays = list(packed[2:])
    n0 = int(vb[-1])
    if device:
        import torch
        arrays = [torch.from_numpy(a).cuda() for a in arrays]
        out = dict(win=torch.empty(n0, dtype=torch.uint8, device="cuda"),
                   sigma=torch.empty(n0, dtype=torch.int32, device="cuda"),
                   tau=torch.empty(n0, dtype=torch.int32, device="cuda"),
                   val_class=torch.empty(n0, dtype=torch.int8, device="cuda"),
                   val_depth=torch.empty(n0, dtype=torch.int32, device="cuda"),
                   val_rank=torch.empty(n0, dtype=torch.int32, device="cuda"),
                   dummy_sigma=torch.empty(n0 * 2 + 1, dtype=torch.int8, device="cuda"))
    else:
        out = dict(win=np.empty(n0, np.uint8), sigma=np.empty(n0, np.int32), tau=np.empty(n0, np.int32),
                   val_class=np.empty(n0, np.int8), val_depth=np.empty(n0, np.int32),
                   val_rank=np.empty(n0, np.int32), dummy_sigma=np.empty(n0 * 2 + 1, np.int8))
    res = pg.pg_solve_batch(ctx, len(games), vb, eb, *arrays, **out)
    if device:
        out = {k: v.cpu().numpy() for k, v in out.items()}
    return vb, res, out


def test_batch_matches_oracle_per_game(pg, ctx):
    games = mixed_games(24, 5)
    vb, res, out = run_batch(pg, ctx, games)
    assert res["rc"] == pg.PG_OK and (res["status"] == 0).all()
    db = res["dummy_base"]
    for i, g in enumerate(games):
        gp, r, want = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
        sl = slice(int(vb[i]), int(vb[i + 1]))
        for k in KEYS:
            assert np.array_equal(out[k][sl], np.asarray(want[k])), (i, g.n, k)
        assert (res["major"][i], res["inner"][i]) == (want["major"], want["inner"]), i
        dsig = (r["strat"][gp["n_orig"]:] != gp["n"]).astype(np.int8)
        assert np.array_equal(out["dummy_sigma"][int(db[i]):int(db[i + 1])], dsig), i
    assert res["iterations"] == res["inner"].max()


@pytest.mark.parametrize("loop_ranks", [0, 1])
def test_batch_with_wide_offsets_matches_oracle_per_game(pg, ctx, loop_ranks):
    """The layout of batches of 2^31 or more edges (64-bit edge offsets: the
    packing, the initial profile and both switching kernels on int64 offsets),
    forced on a small batch with a few larger games, in both loop modes."""
    games = mixed_games(16, 23) + [gen.random_game(150_000, 2, 6, gen.batch_seed(9001)),
                                   gen.ladder_game(60_000, seed=9002)]
    pg.pg_set_wide_offsets(ctx, 1)
    pg.pg_set_loop_ranks(ctx, loop_ranks)
    try:
        vb, res, out = run_batch(pg, ctx, games, device=True)
    finally:
        pg.pg_set_wide_offsets(ctx, 0)
        pg.pg_set_loop_ranks(ctx, 0)
    assert res["rc"] == pg.PG_OK and (res["status"] == 0).all()
    db = res["dummy_base"]
    for i, g in enumerate(games):
        gp, r, want = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
        sl = slice(int(vb[i]), int(vb[i + 1]))
        for k in KEYS:
            assert np.array_equal(out[k][sl], np.asarray(want[k])), (i, g.n, k)
        assert (res["major"][i], res["inner"][i]) == (want["major"], want["inner"]), i
        dsig = (r["strat"][gp["n_orig"]:] != gp["n"]).astype(np.int8)
        assert np.array_equal(out["dummy_sigma"][int(db[i]):int(db[i + 1])], dsig), i


def test_batch_equals_single_solves_device_inputs(pg, ctx):
    games = mixed_games(9, 11)
    vb, res, out = run_batch(pg, ctx, games, device=True)
    for i, g in enumerate(games):
        single = pg.solve_arrays(ctx, g.n, *g.arrays())
        sl = slice(int(vb[i]), int(vb[i + 1]))
        for k in KEYS:
            assert np.array_equal(out[k][sl], single[k]), (i, k)
        assert (res["major"][i], res["inner"][i]) == (single["major"], single["inner"])


def test_batch_of_one_and_tiny_games(pg, ctx):
    for games in [[gen.random_game(1, 1, 1, 0)], [gen.random_game(1, 1, 1, s) for s in range(5)],
                  [gen.random_game(3000, 2, 5, 7)]]:
        vb, res, out = run_batch(pg, ctx, games)
        for i, g in enumerate(games):
            _, _, want = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
            sl = slice(int(vb[i]), int(vb[i + 1]))
            for k in KEYS:
                assert np.array_equal(out[k][sl], np.asarray(want[k])), (i, k)


def test_batch_errors(pg, ctx):
    games = mixed_games(3, 2)
    vb, eb, off, tgt, own, pri = pg.pack_games(games)
    bad = vb.copy()
    bad[1] = bad[0]
    with pytest.raises(pg.PgError) as e:
        pg.pg_solve_batch(ctx, 3, bad, eb, off, tgt, own, pri)
    assert e.value.code == pg.PG_EINVAL
    tgt2 = tgt.copy()
    tgt2[int(eb[1])] = 10**6
    with pytest.raises(pg.PgError) as e:
        pg.pg_solve_batch(ctx, 3, vb, eb, off, tgt2, own, pri)
    assert e.value.code == pg.PG_EINVAL
