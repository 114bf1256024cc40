"""The ruling-set path: valuations ranked through an Euler tour of the
nearest-greater forest and a sparse ruling-set list ranking, taken when a
g-chain is longer than the cutover depth (pg_set_tuning). Every result is
compared bit for bit with the CPU oracle:

* deep forests the default path would walk quadratically: one n-long chain of
  increasing priorities (depth n) and chains of increasing runs, valuated;
* full solves whose plays climb long increasing runs (paths of increasing
  priorities with a few back edges), which switch to the ruling-set path
  mid-solve, in the graph loop and in the host loop;
* the path forced on ordinary inputs (cutover 1): the tree shapes of every
  segment-sorting class, random workloads, ladders and a batch, with several
  ruler strides (one element in 2, 32 and 512 a ruler).
"""
import numpy as np
import pytest

from oracle import o2
from paper_1705_02313_gb300 import gen
from paper_1705_02313_gb300.gen import Game

import test_gpu_tree_shapes as shapes
from test_gpu_parity import assert_same, oracle_solution

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    from paper_1705_02313_gb300 import build, pg as _pg
    build.build()
    return _pg


@pytest.fixture
def ctx(pg):
    c = pg.pg_ctx_create(0, tuning=False)
    yield c
    pg.pg_ctx_destroy(c)


def valuate(pg, ctx, g, sigma):
    """pg_valuate of an all-Even game's profile, with the counters."""
    n = g.n
    game = pg.pg_load_csr(ctx, n, g.m, *g.arrays())
    try:
        out = dict(val_class=np.empty(n, np.int8), val_depth=np.empty(n, np.int32), val_rank=np.empty(n, np.int32),
                   dom=np.empty(n, np.int32))
        rc = pg.pg_valuate(ctx, game, sigma, None, None, **out)
        cnt = pg.pg_game_counters(game)
    finally:
        pg.pg_game_free(game)
    return rc, out, cnt


def oracle_valuation(g, sigma):
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    assert gp["n"] == g.n  # all Even: no dummies
    return o2.valuate(gp, np.where(sigma < 0, gp["n"], sigma).astype(np.int32))


def assert_valuation(rc, out, want, n, pg):
    assert rc == (pg.PG_ENOTADMISSIBLE if (want["cls"] == o2.ODDCYCLE).any() else pg.PG_OK)
    assert np.array_equal(out["val_class"], (want["cls"][:n] != 0).astype(np.int8))
    assert np.array_equal(out["val_depth"], want["depth"][:n])
    assert np.array_equal(out["val_rank"], want["rank"][:n])
    assert np.array_equal(out["dom"], want["dom"][:n])


def climbing_profile(n, run, seed, cycles):
    """An all-Even game with a profile whose plays climb: vertex v's priority
    is 2v + (random parity bit), and sigma sends v to v + 1 (to the sink at
    the end) except that every ``run`` vertices one is sent to the sink, or
    with ``cycles`` also to a random vertex below it (closing a cycle that
    can be longer than the run). Without cycles the g-chains are increasing
    runs of ``run`` vertices (run = n: one chain of depth n). Each vertex also
    has one random edge."""
    rng = np.random.default_rng(seed)
    pri = (2 * np.arange(n) + rng.integers(0, 2, n)).astype(np.int64)
    sigma = np.arange(1, n + 1, dtype=np.int64)
    sigma[-1] = -1
    if run < n:
        cuts = np.arange(run - 1, n - 1, run)
        back = rng.integers(0, 3, cuts.size) if cycles else np.zeros(cuts.size, np.int64)
        sigma[cuts] = np.where(back == 0, -1, rng.integers(0, np.maximum(cuts, 1)))
    rows = []
    for v in range(n):
        e = {int(rng.integers(0, n))}
        if sigma[v] >= 0:
            e.add(int(sigma[v]))
        rows.append(sorted(e))
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    tgt = np.array([x for r in rows for x in r], np.int32)
    perm = rng.permutation(n)  # shuffle vertex ids
    inv = np.empty(n, np.int64)
    inv[perm] = np.arange(n)
    # vertex perm[i] plays the role of i
    rows2 = [None] * n
    for i in range(n):
        rows2[perm[i]] = sorted(int(perm[x]) for x in rows[i])
    off2 = np.zeros(n + 1, np.int64)
    off2[1:] = np.cumsum([len(r) for r in rows2])
    tgt2 = np.array([x for r in rows2 for x in r], np.int32)
    pri2 = np.empty(n, np.int64)
    pri2[perm] = pri
    sigma2 = np.full(n, -1, np.int64)
    sigma2[perm] = np.where(sigma >= 0, perm[np.maximum(sigma, 0)], -1)
    g = Game(n, off2.astype(np.int32), tgt2, np.zeros(n, np.uint8), pri2.astype(np.int32))
    return g, sigma2.astype(np.int32)


@pytest.mark.parametrize("n,run,cycles,deep", [(200_000, 200_000, False, 1), (150_000, 700, True, 1),
                                               (50_000, 200, True, 1), (50_000, 20, False, 0), (3, 3, False, 0),
                                               (1, 1, False, 0)])
def test_deep_chains_take_the_ruling_set_path(pg, ctx, n, run, cycles, deep):
    g, sigma = climbing_profile(n, run, seed=n + run, cycles=cycles)
    rc, out, cnt = valuate(pg, ctx, g, sigma)
    want = oracle_valuation(g, sigma)
    assert_valuation(rc, out, want, n, pg)
    assert cnt["deep"] == deep
    if deep:
        assert cnt["n_rulers"] > 0 and cnt["deep_rounds"] > 0


@pytest.mark.parametrize("ruler_bits", [1, 5, 9])
def test_tree_shapes_forced_through_the_ruling_set(pg, ctx, ruler_bits):
    pg.pg_set_tuning(ctx, deep_cut=1, ruler_bits=ruler_bits)
    t = pg.pg_get_tuning(ctx)
    assert (t["deep_cut"], t["ruler_bits"]) == (1, ruler_bits)
    rng = np.random.default_rng(10 + ruler_bits)
    trees = [
        shapes.build_tree([[40], [1, 3, 20, 33], [0, 2, 9, 50], [0, 1, 4]], rng),   # small, mid segments
        shapes.build_tree([[5000], [0, 0, 1, 2]], rng),                              # one segment beyond 4,096
        shapes.build_tree([[4097], [0, 1]], rng),
        shapes.build_tree([[4096], [0]], rng),
        shapes.build_tree([[1], [1], [1], [1], [1], [9], [1], [32], [0, 1]], rng),
        shapes.build_tree([[16], [17], [0, 1]], rng),                                # at the register-sort limit
    ]
    for cycles in (set(), {0, 2}):
        g, sigma = shapes.profile_game(trees, cycle_roots=cycles, rng=rng)
        rc, out, cnt = valuate(pg, ctx, g, sigma)
        assert cnt["deep"] == 1
        assert_valuation(rc, out, oracle_valuation(g, sigma), g.n, pg)


def climbing_game(n, seed, back):
    """A path i -> i+1 whose priorities increase along it (2i + a random parity
    bit), the last vertex an even-priority Even vertex with a self-loop, and
    with probability ``back`` one more edge from i to a random j < i. Solved
    profiles then have plays that climb long runs (deep g-forests)."""
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        r = {i + 1} if i < n - 1 else {i}
        if 0 < i < n - 1 and rng.random() < back:
            r.add(int(rng.integers(0, i)))
        rows.append(sorted(r))
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    tgt = np.array([x for r in rows for x in r], np.int32)
    own = rng.integers(0, 2, n).astype(np.uint8)
    own[-1] = 0
    pri = 2 * np.arange(n) + rng.integers(0, 2, n)
    pri[-1] = 2 * (n - 1)
    return Game(n, off.astype(np.int32), tgt, own, pri.astype(np.int32))


def solve_with_stats(pg, ctx, g, timing):
    n = g.n
    pg.pg_set_timing(ctx, timing)
    game = pg.pg_load_csr(ctx, g.n, g.m, *g.arrays())
    try:
        _, _, k = pg.pg_game_info(game)
        out = dict(win=np.empty(n, np.uint8), sigma=np.empty(n, np.int32), tau=np.empty(n, np.int32),
                   val_class=np.empty(n, np.int8), val_depth=np.empty(n, np.int32), val_rank=np.empty(n, np.int32),
                   dummy_sigma=np.empty(max(k, 1), np.int8))
        major, inner = pg.pg_solve(ctx, game, **out)
        out["dummy_sigma"] = out["dummy_sigma"][:k]
        stats = pg.pg_kernel_stats(game)
    finally:
        pg.pg_game_free(game)
        pg.pg_set_timing(ctx, False)
    out.update(major=major, inner=inner)
    return out, stats


@pytest.mark.parametrize("n,back,seed", [(3000, 0.0, 1), (5000, 0.05, 3), (4000, 0.1, 5)])
def test_solves_that_turn_deep(pg, ctx, n, back, seed):
    g = climbing_game(n, seed, back)
    _, _, want = oracle_solution(g)
    for timing in (False, True):  # the graph loop, and the host loop with per-kernel timing
        out, stats = solve_with_stats(pg, ctx, g, timing)
        assert_same(out, want, "climbing game n=%d back=%s timing=%s" % (n, back, timing))
        if timing:
            assert stats["ruling_set"][2] > 0  # some valuations took the ruling-set path


@pytest.mark.parametrize("ruler_bits", [1, 5, 9])
def test_solves_forced_through_the_ruling_set(pg, ctx, ruler_bits):
    pg.pg_set_tuning(ctx, deep_cut=1, ruler_bits=ruler_bits)
    games = [gen.random_game(1000, 1, 4, s) for s in range(8)] + \
        [gen.random_game(20000, 2, 5, 9), gen.ladder_game(5000, 4), gen.random_game(3000, 1, 3, 5, p_odd=0.9)]
    for i, g in enumerate(games):
        got = pg.solve_arrays(ctx, g.n, *g.arrays())
        _, _, want = oracle_solution(g)
        assert_same(got, want, "game %d (n=%d)" % (i, g.n))


def test_batch_forced_through_the_ruling_set(pg, ctx):
    from test_gpu_batch import KEYS, mixed_games, run_batch
    pg.pg_set_tuning(ctx, deep_cut=1, ruler_bits=3)
    games = mixed_games(12, 31) + [climbing_game(2000, 7, 0.05)]
    vb, res, out = run_batch(pg, ctx, games)
    assert res["rc"] == pg.PG_OK
    for i, g in enumerate(games):
        _, _, want = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
        sl = slice(int(vb[i]), int(vb[i + 1]))
        for k in KEYS:
            assert np.array_equal(out[k][sl], np.asarray(want[k])), (i, g.n, k)
        assert (res["major"][i], res["inner"][i]) == (want["major"], want["inner"]), i


def test_tuning_arguments(pg, ctx):
    before = pg.pg_get_tuning(ctx)
    assert before == {"deep_cut": 64, "ruler_bits": 5, "walk_cap": 64, "switch_block": 256, "loop_ranks": 0}
    for bad in (dict(deep_cut=-1), dict(ruler_bits=17), dict(ruler_bits=-2), dict(walk_cap=48),
                dict(switch_block=64)):
        with pytest.raises(pg.PgError) as e:
            pg.pg_set_tuning(ctx, **bad)
        assert e.value.code == pg.PG_EINVAL
    pg.pg_set_tuning(ctx)  # zeros keep the values
    assert pg.pg_get_tuning(ctx) == before
