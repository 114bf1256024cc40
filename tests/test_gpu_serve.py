"""Serving with continuous batching: games submitted while others are being
solved are admitted between rounds, and every game's result is the one it
gets alone (pg_solve, and the oracle on every key, the dummies' choices
included), for small games in waves and for games of 1e5-1e6 vertices in a
layout with 64-bit edge offsets."""
import time

import numpy as np
import pytest

from oracle import o2
from paper_1705_02313_gb300 import gen

pytestmark = pytest.mark.gpu

KEYS = ["win", "sigma", "tau", "val_class", "val_depth", "val_rank", "dummy_sigma"]


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


def stream_games(count, seed):
    rng = np.random.default_rng(seed)
    games = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(20), np.log(30000))))
        if i % 5 == 4:
            games.append(gen.ladder_game(max(n, 2), seed=500 + i))
        else:
            games.append(gen.random_game(n, 2, 6, seed=gen.batch_seed(1000 + i)))
    return games


def drain(pg, sv, want, timeout_s=120):
    got = {}
    t0 = time.time()
    while len(got) < want and time.time() - t0 < timeout_s:
        for r in pg.pg_server_poll(sv, 64, 200):
            got[r["tag"]] = r
    return got


def test_results_alone_and_in_the_mix(pg, ctx):
    games = stream_games(30, 1)
    # a capacity that holds only a few games at once, and short rounds: games are
    # admitted while others are resident, and leave as they finish
    sv = pg.pg_server_create(0, max_vertices=60000, max_edges=400000, max_games=6, round_iters=3)
    try:
        for wave in range(3):
            for i in range(wave * 10, wave * 10 + 10):
                g = games[i]
                pg.pg_server_submit(sv, g.n, g.m, *g.arrays(), tag=1000 + i)
            time.sleep(0.05)
        got = drain(pg, sv, len(games))
        assert len(got) == len(games), pg.pg_server_error(sv)
        stats = pg.pg_server_get_stats(sv)
        results = {t: pg.pg_server_fetch(sv, t, got[t]["n"], got[t]["k"]) for t in got}
    finally:
        pg.pg_server_destroy(sv)
    assert stats["admitted"] == stats["completed"] == len(games)
    assert stats["admitted_while_busy"] > 0 and stats["max_resident"] > 1
    for i, g in enumerate(games):
        r, out = got[1000 + i], results[1000 + i]
        assert r["status"] == pg.PG_OK and r["latency_us"] >= r["queue_us"] >= 0
        alone = pg.solve_arrays(ctx, g.n, *g.arrays())
        for k in KEYS:
            assert np.array_equal(out[k], alone[k]), (i, g.n, k)
        assert (r["major"], r["inner"]) == (alone["major"], alone["inner"])
        want = oracle_result(g)  # and the oracle, every key
        for k in KEYS:
            assert np.array_equal(out[k], np.asarray(want[k])), (i, k)
        assert (r["major"], r["inner"]) == (want["major"], want["inner"]), i


def oracle_result(g):
    """The oracle's solve of g alone, with the dummies' choices (1 = their edge)."""
    gp, r, want = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
    want["dummy_sigma"] = (r["strat"][gp["n_orig"]:gp["n"]] != gp["n"]).astype(np.int8)
    return want


def test_large_games_with_wide_offsets_equal_oracle(pg):
    """Games of 1e5-1e6 vertices (random and ladder) arriving while others are
    resident, in a layout with 64-bit edge offsets (the layout of the largest
    servers), each equal to the oracle's solve of it alone on every key."""
    games = [gen.random_game(120_000, 2, 6, gen.batch_seed(7001)), gen.ladder_game(250_000, seed=7002),
             gen.random_game(700_000, 2, 6, gen.batch_seed(7003)), gen.random_game(300_000, 2, 6, gen.batch_seed(7004)),
             gen.random_game(1_000_000, 2, 6, gen.batch_seed(7005))]
    sv = pg.pg_server_create(0, max_vertices=2_400_000, max_edges=12_000_000, max_games=4, round_iters=2,
                             wide_offsets=True)
    try:
        for i, g in enumerate(games):  # one burst: the server admits what fits, the rest as room frees up
            pg.pg_server_submit(sv, g.n, g.m, *g.arrays(), tag=i)
        got = drain(pg, sv, len(games), timeout_s=300)
        assert len(got) == len(games), pg.pg_server_error(sv)
        stats = pg.pg_server_get_stats(sv)
        results = {t: pg.pg_server_fetch(sv, t, got[t]["n"], got[t]["k"]) for t in got}
    finally:
        pg.pg_server_destroy(sv)
    assert stats["max_resident"] > 1
    for i, g in enumerate(games):
        want = oracle_result(g)
        assert got[i]["status"] == pg.PG_OK
        for k in KEYS:
            assert np.array_equal(results[i][k], np.asarray(want[k])), (i, g.n, k)
        assert (got[i]["major"], got[i]["inner"]) == (want["major"], want["inner"]), i


def test_iteration_cap_and_rejections(pg, ctx):
    sv = pg.pg_server_create(0, max_vertices=16000, max_edges=100000, max_games=4, round_iters=2, max_inner=3)
    try:
        g = gen.random_game(3000, 2, 5, 3)
        pg.pg_server_submit(sv, g.n, g.m, *g.arrays(), tag=1)
        big = gen.random_game(15000, 2, 5, 4)  # more than the capacity after preprocessing
        pg.pg_server_submit(sv, big.n, big.m, *big.arrays(), tag=2)
        bad = gen.random_game(50, 1, 3, 5)
        off = bad.offsets.copy()
        off[3] = off[2]  # a vertex without edges
        pg.pg_server_submit(sv, bad.n, bad.m, off, bad.targets, bad.owner, bad.pri, tag=3)
        with pytest.raises(pg.PgError) as e:
            pg.pg_server_submit(sv, g.n, g.m, *g.arrays(), tag=1)  # tag in use
        assert e.value.code == pg.PG_EINVAL
        got = drain(pg, sv, 3)
        with pytest.raises(pg.PgError):
            pg.pg_server_fetch(sv, 99, 1, 0)
        capped = pg.pg_server_fetch(sv, 1, g.n, got[1]["k"])
    finally:
        pg.pg_server_destroy(sv)
    assert got[1]["status"] == pg.PG_ETIMEOUT and got[1]["inner"] == 3
    assert got[2]["status"] == pg.PG_ENOMEM
    assert got[3]["status"] == pg.PG_EINVAL
    # the capped result is the profile after three iterations, valuated
    game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
    try:
        ref = dict(win=np.empty(g.n, np.uint8), sigma=np.empty(g.n, np.int32), val_rank=np.empty(g.n, np.int32))
        with pytest.raises(pg.PgError):
            pg.pg_solve(ctx, game, max_inner=3, **ref)
    finally:
        pg.pg_game_free(game)
    for k in ref:
        assert np.array_equal(capped[k], ref[k]), k


def test_destroy_with_work_in_flight(pg):
    sv = pg.pg_server_create(0, max_vertices=200000, max_edges=1000000, max_games=8, round_iters=2)
    for i in range(6):
        g = gen.random_game(20000, 2, 6, gen.batch_seed(i))
        pg.pg_server_submit(sv, g.n, g.m, *g.arrays(), tag=i)
    time.sleep(0.02)
    pg.pg_server_destroy(sv)  # returns without waiting for the queue
