"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer results must be bit-exact: winners, both strategies, the valuation
class, depth and rank of every vertex, the dummies' strategies and the
iteration counts (Algorithm 1 with the tie-breaks of the C ABI is
deterministic). Inputs are seeded synthetic games from the generators; the
expected values come only from oracle/.
"""
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


def oracle_solution(g):
    gp, res, out = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
    out["dummy_sigma"] = (res["strat"][gp["n_orig"]:] != gp["n"]).astype(np.int8)
    return gp, res, out


def assert_same(got, want, label=""):
    for k in KEYS + ["dummy_sigma"]:
        a, b = np.asarray(got[k]), np.asarray(want[k])
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0]
            raise AssertionError("%s %s differs at %d positions, first %s: got %s want %s" %
                                 (label, k, bad.size, bad[:5], a[bad[:5]], b[bad[:5]]))
    assert (got["major"], got["inner"]) == (want["major"], want["inner"]), label


def test_c1_random_1k_seeds(pg, ctx):
    # the 1,000-vertex random workload, seeds 0..99
    for seed in range(100):
        g = gen.random_game(1000, 1, 4, seed)
        got = pg.solve_arrays(ctx, g.n, *g.arrays())
        _, _, want = oracle_solution(g)
        assert_same(got, want, "seed %d" % seed)


@pytest.mark.parametrize("n,dmin,dmax,seed", [
    (1, 1, 1, 0), (2, 1, 2, 1), (3, 1, 3, 2), (7, 1, 4, 3), (64, 1, 4, 4), (2047, 2, 5, 5), (2049, 2, 8, 6),
    (4097, 1, 4, 7), (20000, 2, 5, 8), (60000, 2, 8, 9), (100003, 2, 6, 10),
])
def test_random_sizes_and_ragged_tails(pg, ctx, n, dmin, dmax, seed):
    g = gen.random_game(n, dmin, dmax, seed)
    got = pg.solve_arrays(ctx, g.n, *g.arrays())
    _, _, want = oracle_solution(g)
    assert_same(got, want, "n=%d" % n)


@pytest.mark.parametrize("n,seed", [(2, 0), (10, 1), (1000, 2), (30011, 3)])
def test_ladder(pg, ctx, n, seed):
    g = gen.ladder_game(n, seed)
    got = pg.solve_arrays(ctx, g.n, *g.arrays())
    _, _, want = oracle_solution(g)
    assert_same(got, want, "ladder n=%d" % n)


def test_all_even_and_all_odd(pg, ctx):
    for p_odd in [0.0, 1.0, 0.9, 0.1]:
        g = gen.random_game(3000, 1, 3, seed=5, p_odd=p_odd)
        got = pg.solve_arrays(ctx, g.n, *g.arrays())
        _, _, want = oracle_solution(g)
        assert_same(got, want, "p_odd=%s" % p_odd)


def test_device_outputs_match_host_outputs(pg, ctx):
    import torch
    g = gen.random_game(5000, 2, 5, 12)
    host = pg.solve_arrays(ctx, g.n, *g.arrays())
    dev_in = [torch.from_numpy(a).cuda() for a in g.arrays()]
    dev = pg.solve_arrays(ctx, g.n, *dev_in, device_outputs=True)
    for k in KEYS + ["dummy_sigma"]:
        assert np.array_equal(host[k], dev[k].cpu().numpy()), k


def random_profile(gp, rng):
    n = gp["n"]
    strat = np.empty(n, np.int32)
    for v in range(n):
        row = gp["tgt"][gp["off"][v]:gp["off"][v + 1]]
        choices = list(row) + ([n] if gp["own"][v] == 0 else [])
        strat[v] = choices[rng.integers(0, len(choices))]
    return strat


def profile_to_original(gp, strat):
    """(sigma, tau, dummy_sigma) in original ids for a G' profile."""
    n0, n = gp["n_orig"], gp["n"]
    own = gp["own"][:n0]
    s = strat[:n0].astype(np.int64)
    sigma = np.where(own == 0, np.where(s == n, -1, s), -1).astype(np.int32)
    tr = np.where(s >= n0, gp["dummy_of"][np.clip(s - n0, 0, max(gp["k"] - 1, 0))] if gp["k"] else s, s)
    tau = np.where(own == 1, tr, -1).astype(np.int32)
    dsig = (strat[n0:] != n).astype(np.int8)
    return sigma, tau, dsig


def test_valuate_random_profiles(pg, ctx):
    rng = np.random.default_rng(0)
    for trial, (n, d) in enumerate([(50, (1, 4)), (3000, (1, 4)), (20000, (2, 5)), (70000, (2, 8))]):
        g = gen.random_game(n, d[0], d[1], 40 + trial)
        gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        strat = random_profile(gp, rng)
        want = o2.valuate(gp, strat)
        sigma, tau, dsig = profile_to_original(gp, strat)
        game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
        try:
            out = dict(val_class=np.empty(n, np.int8), val_depth=np.empty(n, np.int32),
                       val_rank=np.empty(n, np.int32), dom=np.empty(n, np.int32))
            rc = pg.pg_valuate(ctx, game, sigma, tau, dsig, **out)
        finally:
            pg.pg_game_free(game)
        n0 = gp["n_orig"]
        odd = want["cls"][:n0] == o2.ODDCYCLE
        assert rc == (pg.PG_ENOTADMISSIBLE if (want["cls"] == o2.ODDCYCLE).any() else pg.PG_OK)
        assert np.array_equal(out["val_class"], (want["cls"][:n0] != 0).astype(np.int8))
        assert np.array_equal(out["val_depth"], want["depth"][:n0])
        assert np.array_equal(out["val_rank"], want["rank"][:n0])
        assert np.array_equal(out["dom"], want["dom"][:n0])
        assert np.array_equal(odd, (out["dom"] >= 0) & (out["dom"] % 2 == 1))  # odd dominant priority iff odd cycle


@pytest.mark.parametrize("n", [5000, 300001])
def test_valuate_long_chain(pg, ctx, n):
    # one n-long successor chain: walks run out of steps and pointer jumping finishes
    g, sigma = gen.chain_profile(n, seed=7)
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    strat = np.where(sigma < 0, gp["n"], sigma).astype(np.int32)
    want = o2.valuate(gp, strat)
    game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
    try:
        out = dict(val_class=np.empty(n, np.int8), val_depth=np.empty(n, np.int32), val_rank=np.empty(n, np.int32))
        rc = pg.pg_valuate(ctx, game, sigma, None, None, **out)
    finally:
        pg.pg_game_free(game)
    assert rc == pg.PG_OK
    assert np.array_equal(out["val_depth"], want["depth"][:n])
    assert np.array_equal(out["val_rank"], want["rank"][:n])
    assert out["val_depth"].max() == n


def test_valuate_cycles_and_tails(pg, ctx):
    # profiles with long cycles and long tails into them (TOP vertices)
    n = 40000
    g, sigma = gen.chain_profile(n, seed=9)
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    rng = np.random.default_rng(3)
    # close the chain into a cycle at a random point: the last vertex goes back
    last = int(np.nonzero(sigma < 0)[0][0])
    row = g.targets[g.offsets[last]:g.offsets[last + 1]]
    sig = sigma.copy()
    sig[last] = row[0]
    strat = np.where(sig < 0, gp["n"], sig).astype(np.int32)
    want = o2.valuate(gp, strat)
    game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
    try:
        out = dict(val_class=np.empty(n, np.int8), val_depth=np.empty(n, np.int32), val_rank=np.empty(n, np.int32),
                   dom=np.empty(n, np.int32))
        rc = pg.pg_valuate(ctx, game, sig, None, None, **out)
    finally:
        pg.pg_game_free(game)
    assert np.array_equal(out["val_class"], (want["cls"][:n] != 0).astype(np.int8))
    assert np.array_equal(out["dom"], want["dom"][:n])
    assert np.array_equal(out["val_rank"], want["rank"][:n])
    assert rc == (pg.PG_ENOTADMISSIBLE if (want["cls"] == o2.ODDCYCLE).any() else pg.PG_OK)
    del rng


def test_best_response(pg, ctx):
    for seed, n in [(0, 1000), (1, 20000)]:
        g = gen.random_game(n, 2, 6, 60 + seed)
        gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        full = o2.run(gp)
        for strat0 in [o2.initial_profile(gp), full["strat"]]:
            want = o2.run(gp, strat=strat0, mode="best_response")
            sigma, tau0, dsig = profile_to_original(gp, strat0)
            wsig, wtau, _ = profile_to_original(gp, want["strat"])
            game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
            try:
                tau = tau0.copy()
                vr = np.empty(n, np.int32)
                iters = pg.pg_best_response(ctx, game, sigma, tau, dsig, val_rank=vr)
            finally:
                pg.pg_game_free(game)
            assert iters == want["inner"]
            assert np.array_equal(tau, wtau)
            assert np.array_equal(vr, want["rank"][:n])


def test_warm_start_from_solution(pg, ctx):
    g = gen.random_game(20000, 2, 5, 77)
    first = pg.solve_arrays(ctx, g.n, *g.arrays())
    game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
    try:
        out = dict(win=np.empty(g.n, np.uint8), sigma=np.empty(g.n, np.int32), tau=np.empty(g.n, np.int32))
        major, inner = pg.pg_solve(ctx, game, sigma_init=first["sigma"], tau_init=first["tau"],
                                   dummy_sigma_init=first["dummy_sigma"].copy(), **out)
    finally:
        pg.pg_game_free(game)
    assert major == 0 and inner == 1
    for k in ["win", "sigma", "tau"]:
        assert np.array_equal(out[k], first[k])


def test_c2_random_1m_full_parity(pg, ctx):
    # the 1,000,000-vertex workload (out-degree U[2,8]) end to end
    g = gen.random_game(1_000_000, 2, 8, 0)
    got = pg.solve_arrays(ctx, g.n, *g.arrays())
    _, _, want = oracle_solution(g)
    assert_same(got, want, "random-1m")


def test_errors(pg, ctx):
    ok = gen.random_game(10, 1, 3, 1)
    # a vertex without edges
    off = ok.offsets.copy()
    off[3] = off[2]
    with pytest.raises(pg.PgError) as e:
        pg.pg_load_csr(ctx, ok.n, ok.m, off, ok.targets, ok.owner, ok.pri)
    assert e.value.code == pg.PG_EINVAL
    tgt = ok.targets.copy()
    tgt[0] = ok.n
    with pytest.raises(pg.PgError) as e:
        pg.pg_load_csr(ctx, ok.n, ok.m, ok.offsets, tgt, ok.owner, ok.pri)
    assert e.value.code == pg.PG_EINVAL
    own = ok.owner.copy()
    own[0] = 2
    with pytest.raises(pg.PgError) as e:
        pg.pg_load_csr(ctx, ok.n, ok.m, ok.offsets, ok.targets, own, ok.pri)
    assert e.value.code == pg.PG_EINVAL
    pri = ok.pri.copy()
    pri[0] = -1
    with pytest.raises(pg.PgError) as e:
        pg.pg_load_csr(ctx, ok.n, ok.m, ok.offsets, ok.targets, ok.owner, pri)
    assert e.value.code == pg.PG_EINVAL
    # repeated priorities: count-vector mode, at most 5 distinct priorities after preprocessing
    pri = ok.pri % 7
    with pytest.raises(pg.PgError) as e:
        pg.pg_load_csr(ctx, ok.n, ok.m, ok.offsets, ok.targets, ok.owner, pri)
    assert e.value.code == pg.PG_EUNSUPPORTED
    # a strategy that is not an edge
    game = pg.pg_load_csr(ctx, ok.n, ok.m, *ok.arrays())
    try:
        sigma = np.full(ok.n, -1, np.int32)
        v = int(np.nonzero(ok.owner == 0)[0][0])
        row = set(ok.targets[ok.offsets[v]:ok.offsets[v + 1]].tolist())
        sigma[v] = [x for x in range(ok.n) if x not in row][0]
        with pytest.raises(pg.PgError) as e:
            pg.pg_solve(ctx, game, win=np.empty(ok.n, np.uint8), sigma_init=sigma)
        assert e.value.code == pg.PG_EINVAL
    finally:
        pg.pg_game_free(game)
    # an Even self-loop of odd priority chosen by sigma: not admissible
    n = 2
    off = np.array([0, 1, 2], np.int32)
    tgt = np.array([0, 0], np.int32)
    own = np.array([0, 1], np.uint8)
    pri = np.array([1, 2], np.int32)
    game = pg.pg_load_csr(ctx, n, 2, off, tgt, own, pri)
    try:
        sigma = np.array([0, -1], np.int32)
        rc = pg.pg_valuate(ctx, game, sigma, None, None, dom=np.empty(n, np.int32))
        assert rc == pg.PG_ENOTADMISSIBLE
        with pytest.raises(pg.PgError) as e:
            pg.pg_best_response(ctx, game, sigma)
        assert e.value.code == pg.PG_ENOTADMISSIBLE
    finally:
        pg.pg_game_free(game)


def test_memory_pool_reuse_and_release(pg, ctx):
    # freed game memory stays cached in the pool and is reused by the next
    # load; releasing it hands it back to the device; results do not change
    import torch
    g = gen.random_game(200_000, 2, 5, 3)
    first = pg.solve_arrays(ctx, g.n, *g.arrays())
    for _ in range(2):
        again = pg.solve_arrays(ctx, g.n, *g.arrays())
        for k in KEYS:
            assert np.array_equal(first[k], again[k]), k
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    pg.pg_release_cached_memory(0)
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after - free_before >= 16 << 20  # at least the game's own arrays were cached
    again = pg.solve_arrays(ctx, g.n, *g.arrays())
    for k in KEYS:
        assert np.array_equal(first[k], again[k]), k
    with pytest.raises(pg.PgError):
        pg.pg_release_cached_memory(-1)


def test_memory_release_keeps_live_games(pg, ctx):
    # releasing the cache while a game is loaded leaves that game intact
    a = gen.random_game(50_000, 2, 5, 4)
    b = gen.random_game(120_000, 2, 5, 5)
    want = pg.solve_arrays(ctx, a.n, *a.arrays())
    live = pg.pg_load_csr(ctx, a.n, a.m, *a.arrays())
    try:
        pg.solve_arrays(ctx, b.n, *b.arrays())  # loads, solves and frees another game
        pg.pg_release_cached_memory(0)
        win = np.empty(a.n, np.uint8)
        sigma = np.empty(a.n, np.int32)
        major, inner = pg.pg_solve(ctx, live, win=win, sigma=sigma)
    finally:
        pg.pg_game_free(live)
    assert np.array_equal(win, want["win"]) and np.array_equal(sigma, want["sigma"])
    assert (major, inner) == (want["major"], want["inner"])
