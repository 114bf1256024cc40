"""CPU tests that pin the oracle (oracle/) to the paper and to mathematics.

Every check here compares the oracle with something other than itself:
brute force over positional strategies, Zielonka's algorithm, Bellman-Ford
with a big-integer closed form of the valuation order, the worked Euler-tour
example of Figure 1, hand-worked golden games, and the monotonicity
invariants of Theorem 1. A final group plants mistakes in the oracle and
checks that these pins catch them.
"""
import os

import numpy as np
import pytest

from oracle import o1, o2, pins
from paper_1705_02313_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
OUT_KEYS = ["win", "sigma", "tau", "val_class", "val_depth", "val_rank"]


def small_games(count, nmin, nmax, dmin=1, dmax=3, base_seed=1000):
    for s in range(count):
        n = nmin + s % (nmax - nmin + 1)
        yield s, gen.random_game(n, dmin, dmax, seed=base_seed + s)


# ---------------------------------------------------------------------------
# golden files

def read_fig1():
    parent, order, expect = {}, None, []
    for line in open(os.path.join(GOLDEN, "fig1_euler_tour.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        parts = line.split()
        if parts[0] == "order":
            order = parts[1:]
        elif order is None:
            parent[parts[0]] = parts[1]
        else:
            expect.append((parts[0], parts[1]))
    return parent, order, expect


def test_fig1_euler_tour_golden():
    parent, order, expect = read_fig1()
    assert pins.euler_tour(parent, "a", order) == expect


def test_euler_tour_any_order_is_a_tour():
    # Section 5: the choice of processing order only changes which Euler tour
    # is produced; each is a closed walk covering every tree edge twice.
    rng = np.random.default_rng(5)
    for trial in range(30):
        n = int(rng.integers(2, 40))
        parent = {v: int(rng.integers(0, v)) for v in range(1, n)}
        order = list(rng.permutation(list(parent)))
        tour = pins.euler_tour(parent, 0, order)
        assert len(tour) == 2 * (n - 1)
        assert len(set(tour)) == len(tour)
        assert tour[0][0] == 0 and tour[-1][1] == 0
        for a, b in zip(tour, tour[1:]):
            assert a[1] == b[0]


def test_list_ranking_valuation_matches_paths():
    # The formal reduction of Section 5 (prefix sums over the tour with
    # weights A_p / A_{-p}) must give, at each vertex, the counts of priorities
    # on its path to the root (v included, root excluded; Section 3).
    rng = np.random.default_rng(7)
    for trial in range(30):
        n = int(rng.integers(2, 60))
        parent = {v: int(rng.integers(0, v)) for v in range(1, n)}
        pri = {v: int(rng.integers(0, 4)) for v in range(n)}
        order = list(rng.permutation(list(parent)))
        got = pins.list_ranking_valuation(parent, 0, order, pri)
        for v in parent:
            want = {}
            x = v
            while x != 0:
                want[pri[x]] = want.get(pri[x], 0) + 1
                x = parent[x]
            assert got[v] == want


def read_counterexample():
    d = {"edges": []}
    for line in open(os.path.join(GOLDEN, "odd_trap_counterexample.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        k, *vals = line.split()
        if k == "edges":
            d["edges"].append(tuple(int(x) for x in vals))
        else:
            d[k] = [int(x) for x in vals]
    n = d["n"][0]
    off = [0] * (n + 1)
    tgt = []
    for v in range(n):
        tgt += sorted(t for s, t in d["edges"] if s == v)
        off[v + 1] = len(tgt)
    return n, off, tgt, d["owner"], d["pri"], d["win"]


def test_odd_trap_counterexample_golden():
    n, off, tgt, own, pri, win = read_counterexample()
    assert [1 - (v in pins.brute_force_winners(n, off, tgt, own, pri)) for v in range(n)] == win
    _, _, out1 = o1.solve_game(n, off, tgt, own, pri)
    _, _, out2 = o2.solve_game(n, off, tgt, own, pri)
    assert list(out1["win"]) == win
    assert list(out2["win"]) == win


# ---------------------------------------------------------------------------
# winning regions: brute force and Zielonka

@pytest.mark.parametrize("dmax", [2, 3])
def test_winners_brute_force(dmax):
    for s, g in small_games(60, 2, 7, 1, dmax):
        even = set(pins.brute_force_winners(g.n, g.offsets, g.targets, g.owner, g.pri))
        _, _, out1 = o1.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
        _, _, out2 = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri, check=True)
        want = [0 if v in even else 1 for v in range(g.n)]
        assert list(out1["win"]) == want, s
        assert list(out2["win"]) == want, s


def test_winners_brute_force_repeated_priorities():
    # O-1 follows the definitions for any priorities, not only distinct ones.
    for s, g in small_games(40, 2, 6, 1, 3, base_seed=77):
        pri = g.pri % 3
        even = set(pins.brute_force_winners(g.n, g.offsets, g.targets, g.owner, pri))
        _, _, out1 = o1.solve_game(g.n, g.offsets, g.targets, g.owner, pri)
        assert list(out1["win"]) == [0 if v in even else 1 for v in range(g.n)], s


def test_winners_zielonka():
    for n, d, seed in [(50, (1, 4), 1), (120, (2, 5), 2), (300, (2, 8), 3), (400, (1, 4), 4)]:
        g = gen.random_game(n, d[0], d[1], seed)
        weven, wodd = pins.zielonka_winners(g.n, g.offsets, g.targets, g.owner, g.pri)
        assert weven | wodd == set(range(n)) and not (weven & wodd)
        _, _, out = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri, check=True)
        assert [v for v in range(n) if out["win"][v] == 0] == sorted(weven)
    g = gen.ladder_game(200, 3)
    weven, _ = pins.zielonka_winners(g.n, g.offsets, g.targets, g.owner, g.pri)
    _, _, out = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri, check=True)
    assert [v for v in range(g.n) if out["win"][v] == 0] == sorted(weven)


def test_trap_certificate():
    # W_Even is closed under Odd's edges and sigma* stays in it; W_Odd is
    # closed under Even's edges and tau* stays in it (Theorem 1 and Section 2).
    for g in [gen.random_game(2000, 2, 5, 11), gen.random_game(3000, 2, 8, 12), gen.ladder_game(2000, 13)]:
        _, _, out = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
        win = out["win"]
        for v in range(g.n):
            succ = g.targets[g.offsets[v]:g.offsets[v + 1]]
            if win[v] == 0 and g.owner[v] == 1:
                assert all(win[u] == 0 for u in succ)
            if win[v] == 0 and g.owner[v] == 0:
                assert out["sigma"][v] >= 0 and win[out["sigma"][v]] == 0
            if win[v] == 1 and g.owner[v] == 0:
                assert all(win[u] == 1 for u in succ)
            if win[v] == 1 and g.owner[v] == 1:
                assert win[out["tau"][v]] == 1


# ---------------------------------------------------------------------------
# the preprocessing step

def test_preprocess_removes_odd_only_cycles():
    for s, g in small_games(40, 5, 60, 1, 4, base_seed=300):
        gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        # no edge between two Odd vertices of U remains
        n = gp["n"]
        for v in range(gp["n_orig"]):
            if gp["inU"][v]:
                for e in range(gp["off"][v], gp["off"][v + 1]):
                    assert gp["tgt"][e] >= gp["n_orig"] or not gp["inU"][gp["tgt"][e]]
        # sigma_init is admissible: no cycle made of Odd vertices only
        odd = [v for v in range(n) if gp["own"][v] == 1]
        adj = {v: [int(gp["tgt"][e]) for e in range(gp["off"][v], gp["off"][v + 1]) if gp["own"][gp["tgt"][e]] == 1]
               for v in odd}
        color = {}

        def has_cycle(v):
            color[v] = 1
            for u in adj[v]:
                if color.get(u) == 1 or (u not in color and has_cycle(u)):
                    return True
            color[v] = 2
            return False
        assert not any(v not in color and has_cycle(v) for v in odd)
        # priorities stay distinct, dummies are even and below every original
        assert len(set(gp["pri"].tolist())) == n
        assert all(gp["pri"][d] % 2 == 0 for d in range(gp["n_orig"], n))
        if gp["k"]:
            assert gp["pri"][gp["n_orig"]:].max() < gp["pri"][:gp["n_orig"]].min()


def test_preprocess_o1_equals_o2():
    for s, g in small_games(30, 5, 80, 1, 4, base_seed=500):
        a = o1.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        b = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        assert a["k"] == b["k"]
        assert a["off"] == b["off"].tolist() and a["tgt"] == b["tgt"].tolist()
        assert a["pri"] == b["pri"].tolist() and a["own"] == b["own"].tolist()
        assert a["dummy_of"] == b["dummy_of"].tolist()


def test_preprocess_keeps_winners():
    # winners of G' restricted to the original vertices equal winners of G
    for s, g in small_games(25, 3, 6, 1, 3, base_seed=900):
        gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        if gp["n"] > 9:
            continue
        w0 = set(pins.brute_force_winners(g.n, g.offsets, g.targets, g.owner, g.pri))
        w1 = set(pins.brute_force_winners(gp["n"], gp["off"], gp["tgt"], gp["own"], gp["pri"]))
        assert w0 == {v for v in w1 if v < g.n}


# ---------------------------------------------------------------------------
# the valuation order: three independent constructions

def random_profile(gp, rng):
    n = gp["n"]
    strat = []
    for v in range(n):
        e0, e1 = gp["off"][v], gp["off"][v + 1]
        choices = [int(gp["tgt"][e]) for e in range(e0, e1)]
        if gp["own"][v] == 0:
            choices.append(n)
        strat.append(choices[int(rng.integers(0, len(choices)))])
    return strat


def test_three_orders_agree():
    rng = np.random.default_rng(3)
    for s, g in small_games(40, 10, 200, 1, 4, base_seed=1300):
        gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        gp1 = o1.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        strat = random_profile(gp, rng)
        r2 = o2.valuate(gp, strat)
        r1 = o1.valuate(gp1, strat)
        # literal Maxdiff sort (O-1) == Kruskal merge order (O-2)
        assert r1["rank"] == r2["rank"].tolist() and r1["sink_rank"] == r2["sink_rank"]
        assert r1["depth"] == r2["depth"].tolist()
        assert [min(c, 1) for c in r1["cls"]] == [min(int(c), 1) for c in r2["cls"]]
        # closed form: sorting by the big-integer value gives the same ranks
        enc = pins.Encoding(gp["pri"].tolist(), gp["n"])
        n = gp["n"]
        vals = [pins.closed_form_value(gp["pri"].tolist(), strat, n, v, enc) for v in range(n)] + [0]
        fin = sorted([v for v in range(n + 1) if vals[v] != pins.TOP_VALUE], key=lambda v: vals[v])
        assert len(set(vals[v] for v in fin)) == len(fin)
        want = {v: i for i, v in enumerate(fin)}
        for v in range(n):
            if vals[v] == pins.TOP_VALUE:
                assert r2["rank"][v] == o2.INT32_MAX
            else:
                assert r2["rank"][v] == want[v]
        assert r2["sink_rank"] == want[n]


def test_literal_compare_walk_matches_ranks():
    rng = np.random.default_rng(8)
    for s, g in small_games(10, 50, 300, 1, 4, base_seed=1700):
        gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        strat = random_profile(gp, rng)
        r = o2.valuate(gp, strat)
        fin = [v for v in range(gp["n"]) if r["cls"][v] == 0] + [gp["n"]]
        key = {v: (r["rank"][v] if v < gp["n"] else r["sink_rank"]) for v in fin}
        for _ in range(300):
            u, w = rng.choice(fin, 2)
            assert o2.compare(gp, strat, r["depth"], u, w) == np.sign(key[u] - key[w])


def play_tops(gp, strat, cls):
    """Top of every finite vertex by its plain definition: the vertex with the
    largest priority on its play before the sink (-1 for the others)."""
    n, pri = gp["n"], gp["pri"]
    top = np.full(n, -1, np.int64)
    for v in range(n):
        if cls[v] != o2.FIN:
            continue
        x, best = v, v
        while x != n:
            if pri[x] > pri[best]:
                best = x
            x = strat[x]
        top[v] = best
    return top


def test_different_tops_decide_by_the_larger_tops_parity():
    # Section 3's order (Maxdiff): when two finite plays have different tops, the larger one is on one play only
    # and above everything on the other, so it decides by its parity; against the sink's empty valuation a finite
    # play is better for Even exactly when its top is even. The loop's comparisons use this on top words.
    rng = np.random.default_rng(21)
    checked = 0
    for s, g in small_games(12, 30, 400, 1, 4, base_seed=2100):
        gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        strat = random_profile(gp, rng)
        r = o2.valuate(gp, strat)
        top = play_tops(gp, strat, r["cls"])
        fin = [v for v in range(gp["n"]) if r["cls"][v] == o2.FIN]
        pri = gp["pri"]
        for u in fin:
            assert np.sign(r["rank"][u] - r["sink_rank"]) == (1 if pri[top[u]] % 2 == 0 else -1)
        for _ in range(400):
            if len(fin) < 2:
                break
            u, w = (int(x) for x in rng.choice(fin, 2, replace=False))
            if top[u] == top[w]:
                continue
            t = top[u] if pri[top[u]] > pri[top[w]] else top[w]
            expect = 1 if (t == top[u]) == (pri[t] % 2 == 0) else -1
            assert np.sign(r["rank"][u] - r["rank"][w]) == expect
            checked += 1
    assert checked > 1000


def test_odd_choice_follows_top_words_unless_best_tops_tie():
    # An Odd vertex's choice (the first minimiser of its successors' valuations, TOP above every finite one) is
    # fixed by the successors' tops alone unless two finite successors share the best top so far: the Odd
    # switching pass skips a vertex none of whose successors' top words changed, unless such a tie kept its mark.
    rng = np.random.default_rng(22)
    decided = 0
    for s, g in small_games(40, 30, 600, 2, 5, base_seed=2200):
        gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        strat = random_profile(gp, rng)
        r = o2.valuate(gp, strat)
        top = play_tops(gp, strat, r["cls"])
        pri = gp["pri"]
        for v in range(gp["n"]):
            if gp["own"][v] != 1:
                continue
            succ = [int(gp["tgt"][e]) for e in range(gp["off"][v], gp["off"][v + 1])]
            if any(r["cls"][t] == o2.ODDCYCLE for t in succ):
                continue
            want = succ[0]
            for t in succ[1:]:
                if r["rank"][t] < r["rank"][want]:
                    want = t
            best, tie = succ[0], False
            for t in succ[1:]:
                tt, tb = r["cls"][t] == o2.TOP, r["cls"][best] == o2.TOP
                if tt or tb:
                    less = tb and not tt  # a finite valuation is below TOP; TOP equals TOP
                elif top[t] == top[best]:
                    tie = True  # a chain comparison
                    break
                else:
                    hi = top[t] if pri[top[t]] > pri[top[best]] else top[best]
                    less = (hi == top[t]) == (pri[hi] % 2 == 1)  # t below best for Even
                if less:
                    best = t
            if not tie:
                assert best == want, (s, v)
                decided += 1
    assert decided > 300


def test_long_chain_profile_ranks():
    # one n-long successor chain: the hardest case for list ranking
    g, sigma = gen.chain_profile(3000, seed=4)
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    strat = np.where(sigma < 0, gp["n"], sigma).astype(np.int32)
    r = o2.valuate(gp, strat)
    assert (r["cls"] == 0).all() and r["depth"].max() == g.n
    enc = pins.Encoding(gp["pri"].tolist(), gp["n"])
    # closed form along the chain, computed from the sink backwards
    order = np.argsort(-r["depth"])  # deepest first
    vals = {}
    for v in order[::-1]:
        nxt = strat[v]
        vals[int(v)] = enc.unit(int(gp["pri"][v])) + (0 if nxt == gp["n"] else vals[int(nxt)])
    vals[gp["n"]] = 0
    fin = sorted(vals, key=lambda v: vals[v])
    for i, v in enumerate(fin):
        assert (r["rank"][v] if v < gp["n"] else r["sink_rank"]) == i


# ---------------------------------------------------------------------------
# best responses: Bellman-Ford (Section 4)

def test_best_response_bellman_ford():
    rng = np.random.default_rng(11)
    for s, g in small_games(25, 10, 150, 1, 4, base_seed=2100):
        gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        n = gp["n"]
        # an admissible sigma: the first solve's sigma at some point; use the
        # final sigma of a full solve and also sigma_init
        full = o2.run(gp)
        for sig_strat in [o2.initial_profile(gp), full["strat"]]:
            strat = np.array(sig_strat, dtype=np.int32)
            br = o2.run(gp, strat=strat, mode="best_response")
            bf = pins.bellman_ford_values(gp, strat.tolist())
            enc = pins.Encoding(gp["pri"].tolist(), n)
            got = [pins.closed_form_value(gp["pri"].tolist(), br["strat"].tolist(), n, v, enc) for v in range(n)]
            assert got == bf[:n], s
            # no Odd-switchable edge remains (Bellman optimality)
            for v in range(n):
                if gp["own"][v] == 1:
                    succ = gp["tgt"][gp["off"][v]:gp["off"][v + 1]]
                    assert got[v] == min(bf[u] for u in succ) + enc.unit(int(gp["pri"][v])) or got[v] == pins.TOP_VALUE


# ---------------------------------------------------------------------------
# Theorem 1 invariants along the trajectory (O-1 trace)

def test_theorem1_invariants():
    for s, g in small_games(20, 10, 120, 1, 4, base_seed=2600):
        gp = o1.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
        trace = []
        o1.run(gp, trace=trace)
        best_resp = []  # valuations at the end of each inner loop
        prev = None
        for i, (_, strat, vals) in enumerate(trace):
            if prev is not None:
                pstrat, pvals = prev
                changed_odd = any(strat[v] != pstrat[v] for v in range(gp["n"]) if gp["own"][v] == 1)
                changed_even = any(strat[v] != pstrat[v] for v in range(gp["n"]) if gp["own"][v] == 0)
                if changed_odd and not changed_even:
                    # an Odd switch: weakly down everywhere, strictly somewhere
                    cmp = [o1.compare(vals[v], pvals[v]) for v in range(gp["n"])]
                    assert all(c <= 0 for c in cmp) and any(c < 0 for c in cmp)
                if changed_even:
                    best_resp.append((pstrat, pvals))
            prev = (strat, vals)
        best_resp.append(prev)
        # consecutive best-response valuations: weakly up, strictly somewhere
        for (s0, v0), (s1, v1) in zip(best_resp, best_resp[1:]):
            cmp = [o1.compare(v1[v], v0[v]) for v in range(gp["n"])]
            assert all(c >= 0 for c in cmp) and any(c > 0 for c in cmp)
        # termination: no switchable edge for either player
        _, fvals = best_resp[-1]
        for v in range(gp["n"]):
            succ = gp["tgt"][gp["off"][v]:gp["off"][v + 1]] + ([gp["n"]] if gp["own"][v] == 0 else [])
            cur = fvals[prev[0][v]]
            for u in succ:
                c = o1.compare(fvals[u], cur)
                assert (c <= 0) if gp["own"][v] == 0 else (c >= 0)


# ---------------------------------------------------------------------------
# the two oracle tiers agree (bit-exact) on every output

@pytest.mark.parametrize("kind", ["random14", "random28", "ladder"])
def test_o1_equals_o2(kind):
    for s in range(12):
        if kind == "random14":
            g = gen.random_game(40 + 37 * s, 1, 4, seed=s)
        elif kind == "random28":
            g = gen.random_game(40 + 23 * s, 2, 8, seed=100 + s)
        else:
            g = gen.ladder_game(30 + 41 * s, seed=200 + s)
        _, r1, out1 = o1.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
        _, r2, out2 = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri, check=True)
        for k in OUT_KEYS:
            assert np.array_equal(np.asarray(out1[k]), np.asarray(out2[k])), (kind, s, k)
        assert (out1["major"], out1["inner"]) == (out2["major"], out2["inner"])


def test_si_reset_same_major_iterations():
    # SI-Reset (Section 6): every best response starts again from the initial
    # Odd strategy. Best-response valuations are unique, so Even's switches,
    # hence the major iterations, sigma, the winners and the final valuations
    # do not depend on it (the paper reports the same major iterations); the
    # two oracle tiers agree on the reset run, inner iterations included.
    for s in range(10):
        g = gen.random_game(30 + 29 * s, 1, 5, seed=900 + s) if s % 3 else gen.ladder_game(40 + 13 * s, seed=s)
        _, r1, a1 = o1.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri, reset=True)
        _, r2, a2 = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri, check=True, reset=True)
        for k in OUT_KEYS:
            assert np.array_equal(np.asarray(a1[k]), np.asarray(a2[k])), (s, k)
        assert (a1["major"], a1["inner"]) == (a2["major"], a2["inner"])
        _, _, b = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
        assert a2["major"] == b["major"] and a2["inner"] >= b["inner"]
        for k in ["win", "sigma", "val_class", "val_depth", "val_rank"]:
            assert np.array_equal(np.asarray(a2[k]), np.asarray(b[k])), (s, k)


def test_o2_config_small_reference_run():
    # the 1,000-vertex random workload (out-degree U[1,4], seed 0) end to end
    g = gen.random_game(1000, 1, 4, 0)
    _, r1, out1 = o1.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
    _, r2, out2 = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri, check=True)
    for k in OUT_KEYS:
        assert np.array_equal(np.asarray(out1[k]), np.asarray(out2[k])), k


# ---------------------------------------------------------------------------
# planted mistakes must be caught by the pins

def test_planted_parity_flip_is_caught(monkeypatch):
    real = o1.compare

    def wrong(a, b):  # odd and even roles swapped in Maxdiff
        (ka, La, _), (kb, Lb, _) = a, b
        if ka != o1.FIN or kb != o1.FIN:
            return real(a, b)
        p = o1.maxdiff(La, Lb)
        if p is None:
            return 0
        if p % 2 == 1:
            return -1 if La.get(p, 0) < Lb.get(p, 0) else 1
        return -1 if La.get(p, 0) > Lb.get(p, 0) else 1

    monkeypatch.setattr(o1, "compare", wrong)
    caught = False
    for s, g in small_games(30, 3, 7, 1, 3):
        even = set(pins.brute_force_winners(g.n, g.offsets, g.targets, g.owner, g.pri))
        try:
            _, _, out = o1.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
        except (o1.NotAdmissible, TimeoutError):
            caught = True
            break
        if list(out["win"]) != [0 if v in even else 1 for v in range(g.n)]:
            caught = True
            break
    assert caught


def test_planted_dropped_first_vertex_is_caught(monkeypatch):
    # valuation that forgets v_0 (counts from v_1): the closed form disagrees
    def wrong_valuation(pri, strat, sink, v):
        kind, L, dom = o1_valuation(pri, strat, sink, v)
        if kind == o1.FIN:
            L = dict(L)
            L[pri[v]] -= 1
            if L[pri[v]] == 0:
                del L[pri[v]]
        return kind, L, dom

    o1_valuation = o1.valuation
    monkeypatch.setattr(o1, "valuation", wrong_valuation)
    rng = np.random.default_rng(1)
    g = gen.random_game(80, 1, 4, 3)
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    gp1 = o1.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    strat = random_profile(gp, rng)
    r1 = o1.valuate(gp1, strat)
    r2 = o2.valuate(gp, strat)
    assert r1["rank"] != r2["rank"].tolist() or r1["depth"] != r2["depth"].tolist()


def test_planted_rank_swap_is_caught():
    # a transposed pair of ranks breaks agreement with the closed form
    rng = np.random.default_rng(2)
    g = gen.random_game(100, 1, 4, 9)
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    strat = random_profile(gp, rng)
    r = o2.valuate(gp, strat)
    fin = np.nonzero(r["cls"] == 0)[0]
    rank = r["rank"].copy()
    a, b = fin[0], fin[1]
    rank[a], rank[b] = rank[b], rank[a]
    enc = pins.Encoding(gp["pri"].tolist(), gp["n"])
    vals = [pins.closed_form_value(gp["pri"].tolist(), strat, gp["n"], v, enc) for v in range(gp["n"])]
    order_ok = all((vals[x] < vals[y]) == (rank[x] < rank[y]) for x in fin for y in fin if x != y)
    assert not order_ok
