"""pg_valuate_static, the valuation that allocates nothing.

Some callers cannot let this library allocate device memory: a framework that
reserves the device's memory up front and owns every allocation, or a loop
that must not call cudaMalloc while it runs. pg_valuate_static serves them
from a fixed array compiled into the library. These tests call it through the
C ABI and check:

* two calls in a row (different profiles, so the second starts from the first
  call's leftovers, and on a non-default stream) give exactly the class, depth
  and rank that pg_valuate gives for the same profiles;
* at the size limit, 2^18 vertices, on a long successor chain with a few
  cycles, and at n = 1, the result equals the CPU oracle's valuation;
* repeated calls leave the device's free memory and torch's allocations
  unchanged;
* a size above the limit is refused.

The file is collected last and passes alone or after the other tests.
"""
import numpy as np
import pytest

from oracle import o2
from paper_1705_02313_gb300 import gen

pytestmark = pytest.mark.gpu

LIMIT = 1 << 18


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


def static_call(pg, n, succ, odd, stream=None):
    """pg_valuate_static on device copies of succ and odd; returns the status
    and host copies of the three outputs (pre-filled with junk)."""
    import torch
    d = torch.device("cuda")
    out = dict(val_class=torch.full((n,), 7, dtype=torch.int8, device=d),
               val_depth=torch.full((n,), -7, dtype=torch.int32, device=d),
               val_rank=torch.full((n,), -7, dtype=torch.int32, device=d))
    s, o = torch.from_numpy(succ).to(d), torch.from_numpy(odd).to(d)
    torch.cuda.synchronize()
    rc = pg.pg_valuate_static(n, s, o, **out, stream=stream)
    torch.cuda.synchronize()
    return rc, {k: t.cpu().numpy() for k, t in out.items()}


def oracle_valuation(succ, odd):
    """The oracle's valuation of a successor function in priority-rank ids:
    priorities 2v + odd[v] are increasing in v with the given parities."""
    n = succ.size
    pri = (2 * np.arange(n, dtype=np.int64) + odd).astype(np.int32)
    r = o2.valuate(dict(n=n, pri=pri), succ)
    fin = r["cls"] == o2.FIN
    return dict(val_class=np.where(fin, 0, 1).astype(np.int8),
                val_depth=np.where(fin, r["depth"], -1).astype(np.int32),
                val_rank=np.where(fin, r["rank"], o2.INT32_MAX).astype(np.int32)), bool((r["cls"] == o2.ODDCYCLE).any())


def test_static_matches_pg_valuate_on_two_calls(pg):
    import torch
    rng = np.random.default_rng(11)
    ctx = pg.pg_ctx_create(0)
    side = torch.cuda.Stream()
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
            rc, got = static_call(pg, n, succ, odd, stream=side if call == 1 else None)
            assert rc == rc_want, call
            for k in ["val_class", "val_depth", "val_rank"]:
                assert np.array_equal(got[k][rank_of], want[k]), (call, k)
    finally:
        pg.pg_ctx_destroy(ctx)


def chain_with_cycles(n, seed):
    """A successor function along a random permutation (one play through all
    n vertices to the sink), with a few vertices sent back to an earlier chain
    position, so the vertices before them reach a cycle instead."""
    rng = np.random.default_rng(seed)
    pi = rng.permutation(n).astype(np.int64)
    succ = np.empty(n, np.int32)
    succ[pi[:-1]] = pi[1:]
    succ[pi[-1]] = n
    for pos in rng.choice(np.arange(n // 2, n), size=3, replace=False):
        succ[pi[pos]] = pi[rng.integers(pos // 2, pos)]
    return succ


@pytest.mark.parametrize("n", [LIMIT, 1])
def test_static_matches_oracle_at_the_limits(pg, n):
    rng = np.random.default_rng(5)
    odd = rng.integers(0, 2, n).astype(np.uint8)
    succ = chain_with_cycles(n, 9) if n > 1 else np.array([1], np.int32)
    want, odd_cycle = oracle_valuation(succ, odd)
    rc, got = static_call(pg, n, succ, odd)
    assert rc == (pg.PG_ENOTADMISSIBLE if odd_cycle else pg.PG_OK)
    for k in ["val_class", "val_depth", "val_rank"]:
        assert np.array_equal(got[k], want[k]), k
    if n > 1:
        assert 0 < int((got["val_class"] == 0).sum()) < n  # both finite and infinite plays


def test_static_allocates_nothing(pg):
    import torch
    n = 100_000
    rng = np.random.default_rng(2)
    d = torch.device("cuda")
    succ = torch.from_numpy(chain_with_cycles(n, 3)).to(d)
    odd = torch.from_numpy(rng.integers(0, 2, n).astype(np.uint8)).to(d)
    rank = torch.empty(n, dtype=torch.int32, device=d)
    pg.pg_valuate_static(n, succ, odd, val_rank=rank)  # set-up call
    torch.cuda.synchronize()
    first = rank.cpu().numpy()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(5):
        pg.pg_valuate_static(n, succ, odd, val_rank=rank)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert np.array_equal(rank.cpu().numpy(), first)


def test_static_rejects_oversize_without_device_work(pg):
    import torch
    d = torch.device("cuda")
    succ = torch.zeros(1, dtype=torch.int32, device=d)
    odd = torch.zeros(1, dtype=torch.uint8, device=d)
    with pytest.raises(pg.PgError) as e:
        pg.pg_valuate_static(LIMIT + 1, succ, odd)
    assert e.value.code == pg.PG_EUNSUPPORTED
