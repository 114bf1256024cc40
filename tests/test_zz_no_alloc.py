"""pg_valuate_static against pg_valuate.

pg_valuate_static is for callers that cannot allocate device memory (for
example code running while a CUDA graph is captured, or a framework that owns
every allocation): it works in a fixed array compiled into the library. This
test checks, through the C ABI, that two calls in a row (different profiles,
so the second call starts from the first call's leftovers) give exactly the
class, depth and rank that pg_valuate gives for the same profiles. It lives in
its own file, collected last, and passes alone or after the other tests.
"""
import numpy as np
import pytest

from paper_1705_02313_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    from paper_1705_02313_gb300 import build, pg as _pg
    build.build()
    return _pg


def all_even_game(n, seed):
    """A game whose vertices all belong to Even: the preprocessing adds no
    dummy, so a profile is just sigma and the library's internal ids are the
    priority ranks."""
    g = gen.random_game(n, 1, 4, seed)
    g.owner[:] = 0
    return g


def random_sigma(g, rng):
    sigma = np.empty(g.n, np.int32)
    for v in range(g.n):
        row = list(g.targets[g.offsets[v]:g.offsets[v + 1]]) + [-1]
        sigma[v] = row[rng.integers(0, len(row))]
    return sigma


def test_static_matches_pg_valuate_on_two_calls(pg):
    import torch
    rng = np.random.default_rng(11)
    ctx = pg.pg_ctx_create(0)
    try:
        for call, (n, seed) in enumerate([(50_000, 3), (20_011, 4)]):
            g = all_even_game(n, seed)
            sigma = random_sigma(g, rng)
            game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
            try:
                assert pg.pg_game_info(game)[2] == 0
                want = dict(val_class=np.empty(n, np.int8), val_depth=np.empty(n, np.int32),
                            val_rank=np.empty(n, np.int32))
                rc_want = pg.pg_valuate(ctx, game, sigma, None, None, **want)
            finally:
                pg.pg_game_free(game)
            # the same profile in priority-rank ids
            rank_of = np.empty(n, np.int64)
            rank_of[np.argsort(g.pri, kind="stable")] = np.arange(n)
            succ = np.empty(n, np.int32)
            succ[rank_of] = np.where(sigma < 0, n, rank_of[np.maximum(sigma, 0)])
            odd = np.empty(n, np.uint8)
            odd[rank_of] = (g.pri & 1).astype(np.uint8)
            d = torch.device("cuda")
            out = dict(val_class=torch.full((n,), 7, dtype=torch.int8, device=d),
                       val_depth=torch.full((n,), -7, dtype=torch.int32, device=d),
                       val_rank=torch.full((n,), -7, dtype=torch.int32, device=d))
            rc = pg.pg_valuate_static(n, torch.from_numpy(succ).to(d), torch.from_numpy(odd).to(d), **out)
            torch.cuda.synchronize()
            assert rc == rc_want, call
            for k in ["val_class", "val_depth", "val_rank"]:
                got = out[k].cpu().numpy()[rank_of]
                assert np.array_equal(got, want[k]), (call, k)
    finally:
        pg.pg_ctx_destroy(ctx)


def test_static_rejects_oversize_without_device_work(pg):
    import torch
    d = torch.device("cuda")
    succ = torch.zeros(1, dtype=torch.int32, device=d)
    odd = torch.zeros(1, dtype=torch.uint8, device=d)
    with pytest.raises(pg.PgError) as e:
        pg.pg_valuate_static((1 << 18) + 1, succ, odd)
    assert e.value.code == pg.PG_EUNSUPPORTED
