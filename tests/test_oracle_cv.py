"""Pins of the count-vector oracle (O-3) for games whose priorities repeat.

O-3 is checked against things other than itself: the definitional O-1
(count vectors as dicts, literal Maxdiff, Section 3), brute force over
positional strategies and Zielonka's algorithm for the winning regions, the
distinct-priority oracle O-2 (an independent encoding of the same order),
and the literal counts of priorities along each play."""
import numpy as np
import pytest

from oracle import o1, o2, o3, pins
from paper_1705_02313_gb300 import gen

KEYS = ["win", "sigma", "tau", "val_class", "val_depth"]


def level_games(count, nmin, nmax, levels, base_seed):
    rng = np.random.default_rng(base_seed)
    for s in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        if s % 4 == 3 and n >= 2:
            g = gen.ladder_game(n, seed=base_seed + s)
            g.pri[:] = g.pri % levels
        else:
            g = gen.random_game(n, 1, 5, seed=base_seed + s, levels=levels)
        yield s, g


@pytest.mark.parametrize("levels", [2, 3, 4])
def test_o3_equals_o1(levels):
    for s, g in level_games(25, 5, 160, levels, 300 * levels):
        gp1, r1, out1 = o1.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
        gp3, r3, out3 = o3.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
        assert gp1["k"] == gp3["k"] and list(gp1["pri"]) == list(gp3["pri"])
        for k in KEYS:
            assert np.array_equal(np.asarray(out1[k]), np.asarray(out3[k])), (levels, s, k)
        assert (out1["major"], out1["inner"]) == (out3["major"], out3["inner"]), (levels, s)
        assert list(r1["level_pri"]) == list(r3["level_pri"])
        assert np.array_equal(np.asarray(r1["counts"])[: g.n], out3["val_counts"]), (levels, s)


def test_o3_si_reset_equals_o1():
    for s, g in level_games(12, 10, 120, 3, 4400):
        _, r1, out1 = o1.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri, reset=True)
        _, r3, out3 = o3.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri, reset=True)
        for k in KEYS:
            assert np.array_equal(np.asarray(out1[k]), np.asarray(out3[k])), (s, k)
        assert (out1["major"], out1["inner"]) == (out3["major"], out3["inner"])
        _, _, plain = o3.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
        assert plain["major"] == out3["major"] and np.array_equal(plain["win"], out3["win"])


@pytest.mark.parametrize("levels", [2, 3, 4])
def test_o3_winners_brute_force(levels):
    for s, g in level_games(40, 2, 7, levels, 5000 + levels):
        even = set(pins.brute_force_winners(g.n, g.offsets, g.targets, g.owner, g.pri))
        _, _, out = o3.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
        assert list(out["win"]) == [0 if v in even else 1 for v in range(g.n)], (levels, s)


def test_o3_winners_zielonka():
    for n, levels, seed in [(60, 2, 1), (200, 3, 2), (400, 4, 3), (500, 2, 4)]:
        g = gen.random_game(n, 2, 5, seed, levels=levels)
        weven, wodd = pins.zielonka_winners(g.n, g.offsets, g.targets, g.owner, g.pri)
        _, _, out = o3.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
        assert [v for v in range(n) if out["win"][v] == 0] == sorted(weven)
    g = gen.ladder_game(300, 5)
    g.pri[:] = g.pri % 3
    weven, _ = pins.zielonka_winners(g.n, g.offsets, g.targets, g.owner, g.pri)
    _, _, out = o3.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
    assert [v for v in range(g.n) if out["win"][v] == 0] == sorted(weven)


def test_o3_equals_o2_on_distinct_priorities():
    # with distinct priorities the count vectors are sets and O-2 ranks them by
    # an independent construction (Kruskal order): same trajectory
    for s in range(8):
        g = gen.random_game(40 + 30 * s, 1, 5, seed=7000 + s)
        gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        r2 = o2.run(gp)
        r3 = o3.run(gp)
        assert np.array_equal(r2["strat"], r3["strat"]), s
        assert (r2["major"], r2["inner"]) == (r3["major"], r3["inner"])
        assert np.array_equal(r2["cls"], r3["cls"]) and np.array_equal(r2["depth"], r3["depth"])


def test_o3_counts_are_play_counts():
    # the count vector of every finite vertex is the number of occurrences of
    # each priority on its play to the sink, v included (Section 3, L(p))
    g = gen.random_game(3000, 2, 5, 81, levels=4)
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    rng = np.random.default_rng(5)
    for trial in range(3):
        strat = o2.initial_profile(gp) if trial == 0 else o3.run(gp, max_inner=5 * trial, allow_timeout=True)["strat"]
        res = o3.valuate(gp, strat)
        lp = list(res["level_pri"])
        for v in rng.choice(gp["n"], 300, replace=False):
            seen, x, counts = set(), int(v), [0] * len(lp)
            while x != gp["n"] and x not in seen:
                seen.add(x)
                counts[lp.index(int(gp["pri"][x]))] += 1
                x = int(strat[x])
            if x == gp["n"]:
                assert res["cls"][v] == o3.FIN and list(res["counts"][v]) == counts
                assert res["depth"][v] == sum(counts)
            else:
                assert res["cls"][v] != o3.FIN


def test_planted_count_mistakes_are_caught(monkeypatch):
    # plausible mistakes in a count-vector comparison, planted in O-1, are
    # caught by the comparison with O-3 (and the brute-force winners)
    real = o1.compare

    def dropped_lowest(a, b):  # ignores the lowest priority's counts (e.g. the dummies' level)
        (ka, La, da), (kb, Lb, db) = a, b
        if ka == o1.FIN and kb == o1.FIN:
            lo = min(list(La) + list(Lb) + [0])
            La = {p: c for p, c in La.items() if p != lo}
            Lb = {p: c for p, c in Lb.items() if p != lo}
        return real((ka, La, da), (kb, Lb, db))

    def equal_is_smaller(a, b):  # equal count vectors compared as different
        r = real(a, b)
        return -1 if r == 0 and a is not b else r

    for wrong in (dropped_lowest, equal_is_smaller):
        monkeypatch.setattr(o1, "compare", wrong)
        caught = False
        for s, g in level_games(30, 6, 60, 3, 8800):
            _, _, want = o3.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
            try:
                _, _, got = o1.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
            except (o1.NotAdmissible, TimeoutError):
                caught = True
                break
            if not all(np.array_equal(np.asarray(got[k]), np.asarray(want[k])) for k in KEYS) or \
                    (got["major"], got["inner"]) != (want["major"], want["inner"]):
                caught = True
                break
        monkeypatch.setattr(o1, "compare", real)
        assert caught, wrong.__name__
