"""GPU parity of the count-vector mode (games whose priorities repeat)
against the count-vector oracle O-3: strategies, winners, classes, depths,
count vectors (Section 3, L(p)), dominant priorities and iteration counts,
bit for bit."""
import numpy as np
import pytest

from oracle import o2, o3
from paper_1705_02313_gb300 import gen

pytestmark = pytest.mark.gpu

KEYS = ["win", "sigma", "tau", "val_class", "val_depth", "val_counts"]


@pytest.fixture(scope="module")
def pg():
    from paper_1705_02313_gb300 import build, pg as _pg
    build.build()
    return _pg


@pytest.fixture()
def ctx(pg):
    c = pg.pg_ctx_create(0)
    yield c
    pg.pg_ctx_destroy(c)


def solve_cv(pg, ctx, g, **kw):
    game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
    try:
        _, _, k = pg.pg_game_info(game)
        lev = pg.pg_game_levels(game)
        d = lev.size
        out = dict(win=np.empty(g.n, np.uint8), sigma=np.empty(g.n, np.int32), tau=np.empty(g.n, np.int32),
                   val_class=np.empty(g.n, np.int8), val_depth=np.empty(g.n, np.int32),
                   val_rank=np.empty(g.n, np.int32), val_counts=np.empty(g.n * max(d, 1), np.int32),
                   dummy_sigma=np.empty(max(k, 1), np.int8))
        major, inner = pg.pg_solve(ctx, game, **out, **kw)
    finally:
        pg.pg_game_free(game)
    out["val_counts"] = out["val_counts"][: g.n * d].reshape(g.n, d)
    out["dummy_sigma"] = out["dummy_sigma"][:k]
    return out, major, inner, lev


def check_solve(pg, ctx, g, reset=False, label=""):
    out, major, inner, lev = solve_cv(pg, ctx, g, reset_tau=reset)
    gp, res, want = o3.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri, reset=reset)
    assert np.array_equal(lev, want["level_pri"]), label
    for key in KEYS:
        assert np.array_equal(out[key], np.asarray(want[key])), (label, key)
    assert (out["val_rank"] == -1).all()
    dsig = (res["strat"][gp["n_orig"]:] != gp["n"]).astype(np.int8)
    assert np.array_equal(out["dummy_sigma"], dsig), label
    assert (major, inner) == (want["major"], want["inner"]), label


@pytest.mark.parametrize("levels", [2, 3, 4])
def test_cv_random_games(pg, ctx, levels):
    for n, seed in [(1, 0), (2, 1), (33, 2), (1000, 3), (4095, 4), (4097, 5), (30000, 6)]:
        g = gen.random_game(n, 1, 5, seed=100 * levels + seed, levels=levels)
        if np.unique(g.pri).size == n:  # tiny games may draw distinct priorities
            continue
        check_solve(pg, ctx, g, label="levels %d n %d" % (levels, n))


def test_cv_ladders_and_owner_mixes(pg, ctx):
    for n, seed, lv in [(500, 1, 2), (5000, 2, 3), (20000, 3, 4)]:
        g = gen.ladder_game(n, seed)
        g.pri[:] = g.pri % lv
        check_solve(pg, ctx, g, label="ladder %d" % n)
    for p_odd in (0.0, 0.2, 0.8, 1.0):
        g = gen.random_game(3000, 2, 6, seed=77, p_odd=p_odd, levels=3)
        check_solve(pg, ctx, g, label="p_odd %s" % p_odd)


def test_cv_si_reset_and_graph_loop(pg, ctx):
    g = gen.random_game(8000, 2, 5, seed=5, levels=4)
    check_solve(pg, ctx, g, reset=True, label="reset")
    pg.pg_set_graphs(ctx, False)
    check_solve(pg, ctx, g, label="host loop")
    pg.pg_set_graphs(ctx, True)


def random_profile(gp, rng):
    n = gp["n"]
    strat = np.empty(n, np.int32)
    for v in range(n):
        row = gp["tgt"][gp["off"][v]:gp["off"][v + 1]]
        choices = list(row) + ([n] if gp["own"][v] == 0 else [])
        strat[v] = choices[rng.integers(0, len(choices))]
    return strat


def original_profile(gp, strat):
    n0, n = gp["n_orig"], gp["n"]
    own = gp["own"][:n0]
    s = strat[:n0].astype(np.int64)
    sigma = np.where(own == 0, np.where(s == n, -1, s), -1).astype(np.int32)
    tr = np.where(s >= n0, gp["dummy_of"][np.clip(s - n0, 0, max(gp["k"] - 1, 0))] if gp["k"] else s, s)
    tau = np.where(own == 1, tr, -1).astype(np.int32)
    dsig = (strat[n0:] != n).astype(np.int8)
    return sigma, tau, dsig


def valuate_cv(pg, ctx, g, sigma, tau, dsig):
    game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
    try:
        d = pg.pg_game_levels(game).size
        out = dict(val_class=np.empty(g.n, np.int8), val_depth=np.empty(g.n, np.int32),
                   dom=np.empty(g.n, np.int32), val_counts=np.empty(g.n * d, np.int32))
        rc = pg.pg_valuate(ctx, game, sigma, tau, dsig, **out)
    finally:
        pg.pg_game_free(game)
    out["val_counts"] = out["val_counts"].reshape(g.n, d)
    return rc, out


def test_cv_valuate_random_profiles(pg, ctx):
    rng = np.random.default_rng(0)
    for trial, (n, levels) in enumerate([(60, 2), (3000, 3), (25000, 4), (25000, 2)]):
        g = gen.random_game(n, 1, 5, seed=40 + trial, levels=levels)
        gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        strat = random_profile(gp, rng)
        want = o3.valuate(gp, strat)
        rc, out = valuate_cv(pg, ctx, g, *original_profile(gp, strat))
        n0 = gp["n_orig"]
        assert rc == (pg.PG_ENOTADMISSIBLE if (want["cls"] == o3.ODDCYCLE).any() else pg.PG_OK)
        assert np.array_equal(out["val_class"], (want["cls"][:n0] != 0).astype(np.int8))
        assert np.array_equal(out["val_depth"], want["depth"][:n0])
        assert np.array_equal(out["val_counts"], want["counts"][:n0])
        assert np.array_equal(out["dom"], want["dom"][:n0])


@pytest.mark.parametrize("n", [5000, 300001])
def test_cv_long_chain(pg, ctx, n):
    # one n-long successor chain: walks run out of steps and pointer jumping
    # carries the count-vector weights
    g, sigma = gen.chain_profile(n, seed=7)
    g.pri[:] = g.pri % 4
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    strat = np.where(sigma < 0, gp["n"], sigma).astype(np.int32)
    want = o3.valuate(gp, strat)
    rc, out = valuate_cv(pg, ctx, g, sigma, None, None)
    assert rc == pg.PG_OK
    assert np.array_equal(out["val_depth"], want["depth"][:n])
    assert np.array_equal(out["val_counts"], want["counts"][:n])
    assert out["val_depth"].max() == n


def test_cv_cycles_and_tails(pg, ctx):
    n = 40000
    g, sigma = gen.chain_profile(n, seed=9)
    g.pri[:] = g.pri % 3
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    last = int(np.nonzero(sigma < 0)[0][0])
    sig = sigma.copy()
    sig[last] = g.targets[g.offsets[last]]
    strat = np.where(sig < 0, gp["n"], sig).astype(np.int32)
    want = o3.valuate(gp, strat)
    rc, out = valuate_cv(pg, ctx, g, sig, None, None)
    assert np.array_equal(out["val_class"], (want["cls"][:n] != 0).astype(np.int8))
    assert np.array_equal(out["dom"], want["dom"][:n])
    assert np.array_equal(out["val_counts"], want["counts"][:n])
    assert rc == (pg.PG_ENOTADMISSIBLE if (want["cls"] == o3.ODDCYCLE).any() else pg.PG_OK)


def test_cv_best_response(pg, ctx):
    g = gen.random_game(20000, 2, 6, seed=61, levels=3)
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    for strat0 in [o2.initial_profile(gp), o3.run(gp)["strat"]]:
        want = o3.run(gp, strat=strat0, mode="best_response")
        sigma, tau0, dsig = original_profile(gp, strat0)
        _, wtau, _ = original_profile(gp, want["strat"])
        game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
        try:
            d = pg.pg_game_levels(game).size
            tau = tau0.copy()
            cnt = np.empty(g.n * d, np.int32)
            iters = pg.pg_best_response(ctx, game, sigma, tau, dsig, val_counts=cnt)
        finally:
            pg.pg_game_free(game)
        assert iters == want["inner"]
        assert np.array_equal(tau, wtau)
        assert np.array_equal(cnt.reshape(g.n, d), want["counts"][: g.n])


def test_cv_one_million(pg, ctx):
    # a Table-1-shaped game: 1M vertices, 4 priorities, out-degree U[2,5]
    g = gen.native_random_game(1_000_000, 2, 5, seed=3, levels=4)
    check_solve(pg, ctx, g, label="1m")


def test_cv_limits(pg, ctx):
    g = gen.random_game(200, 1, 3, seed=1, levels=6)  # 6 priorities (+ the dummies' level)
    with pytest.raises(pg.PgError) as e:
        pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
    assert e.value.code == pg.PG_EUNSUPPORTED
    g = gen.random_game(300, 1, 3, seed=2, levels=5, p_odd=0.0)  # 5 priorities, no dummies: accepted
    game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
    try:
        assert pg.pg_game_levels(game).size == 5 and pg.pg_game_info(game)[2] == 0
    finally:
        pg.pg_game_free(game)
    # the load probes the first 2^16 priorities for repeats; a repeat further on is found when the priorities
    # are ranked, and the load runs again in the count-vector mode (refused here: 70,000 distinct values)
    g = gen.random_game(70_000, 1, 3, seed=4)
    pri = g.pri.copy()
    pri[-1] = pri[-2]
    with pytest.raises(pg.PgError) as e:
        pg.pg_load_csr(ctx, g.n, g.m, g.offsets, g.targets, g.owner, pri)
    assert e.value.code == pg.PG_EUNSUPPORTED
    game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())  # the distinct game itself still loads
    pg.pg_game_free(game)
    # each level's digit is one bit wider than the bit length of the level's size: 5 levels of 2^24 / 5 ids
    # take 5 x 23 bits, within the key's 126
    n = (1 << 24)
    off = np.arange(n + 1, dtype=np.int32)
    tgt = ((np.arange(n, dtype=np.int64) + 1) % n).astype(np.int32)
    game = pg.pg_load_csr(ctx, n, n, off, tgt, np.zeros(n, np.uint8), (np.arange(n) % 5).astype(np.int32))
    try:
        assert pg.pg_game_levels(game).size == 5
    finally:
        pg.pg_game_free(game)


def test_cv_bellman_ford_best_response(pg, ctx):
    # Bellman-Ford (Section 4) and one-player strategy improvement reach the
    # same best-response values (shortest paths to the sink are unique in value)
    for n, levels, seed in [(3000, 3, 1), (30000, 4, 2), (20000, 2, 3)]:
        g = gen.random_game(n, 2, 5, seed=seed, levels=levels)
        gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        for strat0 in [o2.initial_profile(gp), o3.run(gp)["strat"]]:
            want = o3.run(gp, strat=strat0, mode="best_response")
            sigma, tau0, dsig = original_profile(gp, strat0)
            game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
            try:
                d = pg.pg_game_levels(game).size
                out = dict(val_class=np.empty(g.n, np.int8), val_depth=np.empty(g.n, np.int32),
                           val_counts=np.empty(g.n * d, np.int32))
                tau = np.empty(g.n, np.int32)
                rounds = pg.pg_best_response_bf(ctx, game, sigma, tau, dsig, **out)
            finally:
                pg.pg_game_free(game)
            assert 1 <= rounds <= gp["n"] + 8
            assert np.array_equal(out["val_class"], (want["cls"][: g.n] != 0).astype(np.int8))
            assert np.array_equal(out["val_counts"].reshape(g.n, d), want["counts"][: g.n])
            assert np.array_equal(out["val_depth"], want["depth"][: g.n])
    g = gen.random_game(500, 1, 4, 9)  # distinct priorities: not supported
    game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
    try:
        with pytest.raises(pg.PgError) as e:
            pg.pg_best_response_bf(ctx, game, np.full(g.n, -1, np.int32))
        assert e.value.code == pg.PG_EUNSUPPORTED
    finally:
        pg.pg_game_free(game)
