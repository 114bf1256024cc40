"""The seeded generators: determinism, shapes and the structure each workload
promises (permuted priorities, degree ranges, distinct sorted targets)."""
import numpy as np

from paper_1705_02313_gb300 import gen


def check_csr(g, dmin, dmax):
    deg = np.diff(g.offsets)
    assert g.offsets[0] == 0 and (deg >= dmin).all() and (deg <= dmax).all()
    assert g.targets.min() >= 0 and g.targets.max() < g.n
    for v in range(min(g.n, 2000)):
        row = g.targets[g.offsets[v]:g.offsets[v + 1]]
        assert (np.diff(row) > 0).all()


def test_random_game_shape_and_determinism():
    a = gen.random_game(5000, 2, 8, seed=3)
    b = gen.random_game(5000, 2, 8, seed=3)
    c = gen.random_game(5000, 2, 8, seed=4)
    for x, y in zip(a.arrays(), b.arrays()):
        assert np.array_equal(x, y)
    assert not np.array_equal(a.targets, c.targets)
    check_csr(a, 2, 8)
    assert sorted(a.pri.tolist()) == list(range(a.n))
    assert 0.45 < a.owner.mean() < 0.55


def test_splitmix64_published_values():
    # SplitMix64 from state 0: first outputs of the published generator
    z = gen.splitmix64(np.uint64(0))
    assert int(z) == 0xE220A8397B1DCDAF
    z2 = gen.splitmix64(gen.GOLDEN)
    assert int(z2) == 0x6E789E6AA1B965F4


def test_ladder_and_chain():
    g = gen.ladder_game(1000, 1)
    check_csr(g, 1, 2)
    assert g.targets[0] == 1
    for i in range(1, 999):
        row = g.targets[g.offsets[i]:g.offsets[i + 1]]
        assert row[1] == i + 1 and row[0] < i
    game, sigma = gen.chain_profile(1000, 2)
    check_csr(game, 1, 3)
    assert (sigma == -1).sum() == 1
    # sigma follows existing edges and visits every vertex once
    x = int(np.nonzero(np.bincount(sigma[sigma >= 0], minlength=1000) == 0)[0][0])
    seen = 0
    while x != -1:
        seen += 1
        nxt = sigma[x]
        if nxt >= 0:
            assert nxt in game.targets[game.offsets[x]:game.offsets[x + 1]]
        x = nxt
    assert seen == 1000


def test_log_uniform_sizes():
    s = gen.log_uniform_sizes(4096, 1000, 1_000_000)
    assert s.min() >= 1000 and s.max() <= 1_000_000
    assert 100_000 < s.mean() < 200_000


def test_native_generator_matches_numpy():
    # the C generator must produce exactly the numpy generator's games
    for n, dmin, dmax, seed, p in [(1, 1, 1, 0, 0.5), (2, 1, 4, 3, 0.5), (1000, 1, 4, 0, 0.5), (3000, 2, 8, 7, 0.3),
                                   (20000, 2, 6, gen.batch_seed(5), 0.5), (50, 40, 60, 1, 0.9)]:
        a = gen.random_game(n, dmin, dmax, seed, p_odd=p)
        b = gen.native_random_game(n, dmin, dmax, seed, p_odd=p, nthreads=3)
        for x, y in zip(a.arrays(), b.arrays()):
            assert x.dtype == y.dtype and np.array_equal(x, y), (n, seed)


def test_native_batch_matches_packed_numpy_batch():
    from paper_1705_02313_gb300 import pg
    want = pg.pack_games(gen.batch_games(37, 3, 30000, 2, 6))
    got = gen.native_batch(37, 3, 30000, 2, 6, nthreads=4)
    for x, y in zip(want, got):
        assert np.array_equal(x, y)


def test_native_batch_subset_packs_the_same_games():
    # one rank's share of a batch (indices, in any order) holds exactly those games of the whole batch
    vb, eb, off, tgt, own, pri = gen.native_batch(12, 50, 900, 1, 5)
    idx = [9, 2, 11, 0]
    vb2, eb2, off2, tgt2, own2, pri2 = gen.native_batch(12, 50, 900, 1, 5, indices=idx)
    assert int(vb2[-1]) == sum(int(vb[i + 1] - vb[i]) for i in idx)
    for k, i in enumerate(idx):
        a, b, c, d = int(vb[i]), int(vb[i + 1]), int(vb2[k]), int(vb2[k + 1])
        assert np.array_equal(pri[a:b], pri2[c:d]) and np.array_equal(own[a:b], own2[c:d])
        assert np.array_equal(tgt[eb[i]:eb[i + 1]], tgt2[eb2[k]:eb2[k + 1]])
        assert np.array_equal(off[a + i:b + i + 1], off2[c + k:d + k + 1])
