"""The device-side loop (one CUDA graph launch per solve, a conditional WHILE
node around one iteration) against the host-driven loop and the oracle: same
results, same iteration counts, same behaviour at the iteration cap."""
import numpy as np
import pytest

from oracle import o2
from paper_1705_02313_gb300 import gen
from test_gpu_parity import profile_to_original

pytestmark = pytest.mark.gpu

KEYS = ["win", "sigma", "tau", "val_class", "val_depth", "val_rank"]


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


def host_outputs(n, k):
    return dict(win=np.empty(n, np.uint8), sigma=np.empty(n, np.int32), tau=np.empty(n, np.int32),
                val_class=np.empty(n, np.int8), val_depth=np.empty(n, np.int32), val_rank=np.empty(n, np.int32),
                dummy_sigma=np.empty(max(k, 1), np.int8))


def solve(pg, ctx, g, graphs, max_inner=0):
    pg.pg_set_graphs(ctx, graphs)
    game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
    try:
        _, _, k = pg.pg_game_info(game)
        out = host_outputs(g.n, k)
        try:
            major, inner = pg.pg_solve(ctx, game, max_inner=max_inner, **out)
            rc = pg.PG_OK
        except pg.PgError as e:
            rc, major, inner = e.code, None, None
        used, iters = pg.pg_last_loop(game)
    finally:
        pg.pg_game_free(game)
    return rc, major, inner, used, iters, out


GAMES = [("random-1k", lambda: gen.random_game(1000, 1, 4, 0)),
         ("random-20k", lambda: gen.random_game(20000, 2, 6, 3)),
         ("ladder-5000", lambda: gen.ladder_game(5000, 2)),
         ("single-vertex", lambda: gen.random_game(1, 1, 1, 0))]


@pytest.mark.parametrize("name,make", GAMES, ids=[x[0] for x in GAMES])
def test_graph_loop_matches_host_loop_and_oracle(pg, ctx, name, make):
    g = make()
    rc_g, major_g, inner_g, used_g, it_g, out_g = solve(pg, ctx, g, True)
    rc_h, major_h, inner_h, used_h, it_h, out_h = solve(pg, ctx, g, False)
    assert rc_g == rc_h == pg.PG_OK
    assert used_g and not used_h
    assert (major_g, inner_g) == (major_h, inner_h) and it_g == it_h == inner_g
    for k in KEYS + ["dummy_sigma"]:
        assert np.array_equal(out_g[k], out_h[k]), k
    _, _, want = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
    for k in KEYS:
        assert np.array_equal(out_g[k], np.asarray(want[k])), k
    assert (major_g, inner_g) == (want["major"], want["inner"])


def test_graph_loop_iteration_cap(pg, ctx):
    # the cap ends the device-side loop exactly where it ends the host loop
    g = gen.random_game(5000, 2, 5, 9)
    rc_g, _, _, used_g, it_g, out_g = solve(pg, ctx, g, True, max_inner=3)
    rc_h, _, _, used_h, it_h, out_h = solve(pg, ctx, g, False, max_inner=3)
    assert rc_g == rc_h == pg.PG_ETIMEOUT
    assert used_g and it_g == it_h == 3
    for k in KEYS:
        assert np.array_equal(out_g[k], out_h[k]), k


def test_iteration_cap_matches_oracle_at_every_cap(pg, ctx):
    # at every cap, across Odd and Even switching rounds, the returned profile
    # is the oracle's after as many valuations, and the returned valuation is
    # the oracle's valuation of that profile
    g = gen.random_game(4000, 2, 5, 21)
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    total = o2.run(gp)["inner"]
    assert total > 5
    for cap in range(1, total + 1):
        rc, _, _, used, it, out = solve(pg, ctx, g, True, max_inner=cap)
        r = o2.run(gp, max_inner=cap, allow_timeout=True)
        assert rc == r["status"] == (pg.PG_OK if cap == total else pg.PG_ETIMEOUT), cap
        assert used and it == cap
        sigma, tau, dsig = profile_to_original(gp, r["strat"])
        want = o2.map_back(gp, dict(o2.valuate(gp, r["strat"]), strat=r["strat"]))
        want.update(sigma=sigma, tau=tau, dummy_sigma=dsig)
        for k in KEYS + ["dummy_sigma"]:
            assert np.array_equal(out[k][: len(want[k])], np.asarray(want[k])), (cap, k)


def test_graph_reused_across_calls(pg, ctx):
    # a second solve on the same loaded game reuses its graph and agrees
    g = gen.random_game(3000, 2, 6, 4)
    pg.pg_set_graphs(ctx, True)
    game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
    try:
        _, _, k = pg.pg_game_info(game)
        a, b = host_outputs(g.n, k), host_outputs(g.n, k)
        ra = pg.pg_solve(ctx, game, **a)
        rb = pg.pg_solve(ctx, game, **b)
        assert pg.pg_last_loop(game)[0]
    finally:
        pg.pg_game_free(game)
    assert ra == rb
    for key in KEYS:
        assert np.array_equal(a[key], b[key])


def test_graph_best_response_and_batch(pg, ctx):
    g = gen.random_game(8000, 2, 6, 61)
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    strat0 = o2.initial_profile(gp)
    want = o2.run(gp, strat=strat0, mode="best_response")
    sigma0, tau0, dsig0 = profile_to_original(gp, strat0)
    res = {}
    for graphs in (True, False):
        pg.pg_set_graphs(ctx, graphs)
        game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
        try:
            tau = tau0.copy()
            vr = np.empty(g.n, np.int32)
            iters = pg.pg_best_response(ctx, game, sigma0, tau, dsig0, val_rank=vr)
            assert pg.pg_last_loop(game)[0] == graphs
        finally:
            pg.pg_game_free(game)
        res[graphs] = (iters, tau, vr)
    assert res[True][0] == res[False][0] == want["inner"]
    assert np.array_equal(res[True][1], res[False][1]) and np.array_equal(res[True][2], res[False][2])
    assert np.array_equal(res[True][2], want["rank"][:g.n])

    games = [gen.random_game(n, 2, 6, gen.batch_seed(i)) for i, n in enumerate([5, 300, 4000, 20000, 1])]
    vb, eb, off, tgt, own, pri = pg.pack_games(games)
    outs = {}
    for graphs in (True, False):
        pg.pg_set_graphs(ctx, graphs)
        n0 = int(vb[-1])
        o = dict(win=np.empty(n0, np.uint8), sigma=np.empty(n0, np.int32), val_rank=np.empty(n0, np.int32))
        r = pg.pg_solve_batch(ctx, len(games), vb, eb, off, tgt, own, pri, **o)
        outs[graphs] = (r, o)
    (rg, og), (rh, oh) = outs[True], outs[False]
    assert rg["iterations"] == rh["iterations"] == rg["inner"].max()
    assert np.array_equal(rg["inner"], rh["inner"]) and np.array_equal(rg["major"], rh["major"])
    for key in og:
        assert np.array_equal(og[key], oh[key])


@pytest.mark.parametrize("graphs", [True, False])
def test_si_reset_matches_oracle(pg, ctx, graphs):
    # SI-Reset (Section 6): every best response restarts from the first edges
    pg.pg_set_graphs(ctx, graphs)
    for g in [gen.random_game(2000, 1, 5, 31), gen.random_game(15000, 2, 6, 32), gen.ladder_game(3000, 33)]:
        game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
        try:
            _, _, k = pg.pg_game_info(game)
            out = host_outputs(g.n, k)
            major, inner = pg.pg_solve(ctx, game, reset_tau=True, **out)
            assert pg.pg_last_loop(game)[0] == graphs
            plain = host_outputs(g.n, k)
            major0, inner0 = pg.pg_solve(ctx, game, **plain)
        finally:
            pg.pg_game_free(game)
        _, _, want = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri, reset=True)
        for key in KEYS:
            assert np.array_equal(out[key], np.asarray(want[key])), key
        assert (major, inner) == (want["major"], want["inner"])
        assert major == major0 and inner >= inner0
