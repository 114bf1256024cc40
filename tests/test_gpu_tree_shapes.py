"""Valuations of profiles whose nearest-greater forests have chosen shapes:
parents with one child, a few children (one thread), up to 32 (one warp),
up to 4,096 (one block, sorted in shared memory) and more (the id-ordered
scan); nested many-children parents; the same shapes below a cycle (TOP
trees). Expected values come from the oracle's valuation."""
import numpy as np
import pytest

from oracle import o2
from paper_1705_02313_gb300.gen import Game

pytestmark = pytest.mark.gpu


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


def build_tree(fanouts, rng):
    """parent[] of a rooted tree given as a list of (depth-first) fan-out
    rules: ``fanouts[d]`` is a list of child counts to draw from at depth d.
    Returns parent (root: -1) in breadth-first order."""
    parent = [-1]
    frontier = [0]
    for choices in fanouts:
        nxt = []
        for v in frontier:
            k = int(rng.choice(choices))
            for _ in range(k):
                parent.append(v)
                nxt.append(len(parent) - 1)
        frontier = nxt
    return np.array(parent, np.int64)


def profile_game(parents_list, cycle_roots, rng):
    """An all-Even game whose profile sends every vertex to its tree parent.
    The root of a tree listed in cycle_roots goes to its first child (which
    goes back to it: a cycle whose largest priority is the root's); other
    roots go to the sink. Priorities decrease along breadth-first order inside
    every tree, so a parent's priority is above its children's. Returns
    (game, sigma) in shuffled vertex ids."""
    sizes = [len(p) for p in parents_list]
    n = int(sum(sizes))
    order_pri = np.empty(n, np.int64)
    succ = np.empty(n, np.int64)
    base = 0
    top = n
    for t, par in enumerate(parents_list):
        k = len(par)
        # breadth-first index i gets priority top - 1 - i
        order_pri[base:base + k] = top - 1 - np.arange(k)
        top -= k
        s = np.where(par >= 0, par + base, -1)
        if t in cycle_roots and k > 1:
            s[0] = base + 1  # root -> its first child, which points back to the root: a cycle
        succ[base:base + k] = s
        base += k
    perm = rng.permutation(n)  # vertex id of breadth-first position i
    sigma = np.full(n, -1, np.int64)
    pri = np.empty(n, np.int64)
    pri[perm] = order_pri
    sigma[perm] = np.where(succ >= 0, perm[np.maximum(succ, 0)], -1)
    # edges: the profile's edge plus one random other vertex
    rows = []
    for v in range(n):
        e = {int(rng.integers(0, n))}
        if sigma[v] >= 0:
            e.add(int(sigma[v]))
        rows.append(sorted(e))
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    tgt = np.array([x for r in rows for x in r], np.int32)
    game = Game(n, off.astype(np.int32), tgt, np.zeros(n, np.uint8), pri.astype(np.int32))
    return game, sigma.astype(np.int32)


def check(pg, ctx, g, sigma):
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    assert gp["n"] == g.n  # no Odd vertices: no dummies
    strat = np.where(sigma < 0, gp["n"], sigma).astype(np.int32)
    want = o2.valuate(gp, strat)
    n = g.n
    game = pg.pg_load_csr(ctx, n, g.m, *g.arrays())
    try:
        out = dict(val_class=np.empty(n, np.int8), val_depth=np.empty(n, np.int32), val_rank=np.empty(n, np.int32),
                   dom=np.empty(n, np.int32))
        rc = pg.pg_valuate(ctx, game, sigma, None, None, **out)
    finally:
        pg.pg_game_free(game)
    assert rc == (pg.PG_ENOTADMISSIBLE if (want["cls"] == o2.ODDCYCLE).any() else pg.PG_OK)
    assert np.array_equal(out["val_class"], (want["cls"][:n] != 0).astype(np.int8))
    assert np.array_equal(out["val_depth"], want["depth"][:n])
    assert np.array_equal(out["val_rank"], want["rank"][:n])
    assert np.array_equal(out["dom"], want["dom"][:n])
    return want


def test_fanout_classes_and_nesting(pg, ctx):
    rng = np.random.default_rng(1)
    trees = [
        build_tree([[40], [1, 3, 20, 33], [0, 2, 9, 50], [0, 1, 4]], rng),       # nested warp/block parents
        build_tree([[5000], [0, 0, 1, 2]], rng),                                  # one huge parent (id scan)
        build_tree([[3], [33, 31], [33, 8, 0], [0, 3]], rng),                     # block below block
        build_tree([[4097], [0, 1]], rng),                                        # just above the smem limit
        build_tree([[4096], [0]], rng),                                           # exactly at the smem limit
        build_tree([[1], [1], [1], [1], [1], [9], [1], [32], [0, 1]], rng),        # thin chain, then fans
    ]
    g, sigma = profile_game(trees, cycle_roots=set(), rng=rng)
    want = check(pg, ctx, g, sigma)
    assert (want["cls"] == 0).all()


def test_fanouts_below_cycles(pg, ctx):
    rng = np.random.default_rng(2)
    trees = [build_tree([[6000], [0, 1]], rng), build_tree([[50], [0, 40]], rng), build_tree([[9], [0, 9]], rng),
             build_tree([[300], [2]], rng)]
    g, sigma = profile_game(trees, cycle_roots={0, 1, 2}, rng=rng)
    want = check(pg, ctx, g, sigma)
    assert (want["cls"] != 0).any() and (want["cls"] == 0).any()


def test_many_random_forests(pg, ctx):
    rng = np.random.default_rng(3)
    for _ in range(4):
        trees = [build_tree([[int(rng.integers(1, 70))], [0, 1, 2, 5, 12, 40], [0, 0, 3, 35]], rng) for _ in range(30)]
        g, sigma = profile_game(trees, cycle_roots={int(x) for x in rng.integers(0, 30, 6)}, rng=rng)
        check(pg, ctx, g, sigma)
