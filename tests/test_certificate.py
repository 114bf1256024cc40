"""The stopping-condition certificate (tests/certificate.py) that the
full-size GPU tests rely on: it accepts the oracle's own solutions and
rejects plausible mistakes planted in them (on the CPU)."""
import numpy as np
import pytest

from oracle import o2
from paper_1705_02313_gb300 import gen

import certificate as cert


def solved(g):
    gp, res, out = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
    out["dummy_sigma"] = (res["strat"][gp["n_orig"]:] != gp["n"]).astype(np.int8)
    return gp, res, out


GAMES = [lambda: gen.random_game(3000, 1, 4, 1), lambda: gen.random_game(40000, 2, 5, 2),
         lambda: gen.ladder_game(5000, 3), lambda: gen.random_game(2000, 1, 3, 4, p_odd=0.9)]


@pytest.mark.parametrize("make", GAMES)
def test_oracle_solutions_are_certified(make):
    g = make()
    gp, res, out = solved(g)
    strat = cert.profile_to_gprime(gp, g.offsets, g.targets, out["sigma"], out["tau"], out["dummy_sigma"])
    assert np.array_equal(strat, res["strat"])  # the mapping back to G' is exact
    cert.certify(gp, g.offsets, g.targets, out)


def test_planted_mistakes_are_rejected():
    g = gen.random_game(20000, 2, 5, 7)
    gp, res, out = solved(g)
    key = cert.switch_keys(gp, o2.valuate(gp, res["strat"]))
    off, tgt = gp["off"], gp["tgt"]
    n0 = gp["n_orig"]
    # an Odd vertex moved to a strictly worse edge than its best one
    odd = [v for v in range(n0) if gp["own"][v] == 1 and off[v + 1] - off[v] >= 2
           and len(set(key[tgt[off[v]:off[v + 1]]])) >= 2]
    v = odd[0]
    worst = tgt[off[v] + int(np.argmax(key[tgt[off[v]:off[v + 1]]]))]
    bad = dict(out, tau=out["tau"].copy())
    bad["tau"][v] = worst if worst < n0 else gp["dummy_of"][worst - n0]
    with pytest.raises(AssertionError):
        cert.certify(gp, g.offsets, g.targets, bad)
    # an Even vertex sent to the sink while one of its edges is strictly better
    even = [v for v in range(n0) if gp["own"][v] == 0 and out["sigma"][v] >= 0
            and key[out["sigma"][v]] > key[gp["n"]]]
    bad = dict(out, sigma=out["sigma"].copy())
    bad["sigma"][even[0]] = -1
    with pytest.raises(AssertionError):
        cert.certify(gp, g.offsets, g.targets, bad)
    # a wrong reported rank, depth, class or winner at one vertex
    for k in ("val_rank", "val_depth", "val_class", "win"):
        bad = dict(out)
        bad[k] = out[k].copy()
        bad[k][123] ^= 1
        with pytest.raises(AssertionError):
            cert.certify(gp, g.offsets, g.targets, bad)


def test_profile_before_the_end_is_rejected():
    # the profile after the first valuations still has switchable vertices
    g = gen.random_game(20000, 2, 5, 8)
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    r = o2.run(gp, max_inner=2, allow_timeout=True)
    val = o2.valuate(gp, r["strat"])
    bad_odd, bad_even = cert.stopping_violations(gp, r["strat"], val)
    assert bad_odd.size + bad_even.size > 0


def test_count_vector_keys_follow_the_order():
    # the dense keys agree with the definitional comparison of O-1 (literal
    # Maxdiff on count vectors) on every pair of a small game's vertices
    from oracle import o1, o3
    g = gen.random_game(60, 1, 3, 11, levels=3)
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    r = o3.run(gp, max_inner=2, allow_timeout=True)
    val = o3.valuate(gp, r["strat"])
    key = cert.count_vector_keys(gp, val)
    lp = list(val["level_pri"])

    def o1_val(v):
        if val["cls"][v] != o3.FIN:
            return (o1.TOP, {}, 0)
        return (o1.FIN, {int(lp[j]): int(c) for j, c in enumerate(val["counts"][v]) if c}, int(val["depth"][v]))

    vals = [o1_val(v) for v in range(gp["n"])] + [(o1.FIN, {}, 0)]
    for a in range(gp["n"] + 1):
        for b in range(gp["n"] + 1):
            c = o1.compare(vals[a], vals[b])
            assert int(key[a] > key[b]) - int(key[a] < key[b]) == c, (a, b)


@pytest.mark.parametrize("levels", [2, 3, 4])
def test_count_vector_solutions_are_certified(levels):
    from oracle import o3
    g = gen.random_game(5000, 2, 5, 30 + levels, levels=levels)
    gp, res, out = o3.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
    out["dummy_sigma"] = (res["strat"][gp["n_orig"]:] != gp["n"]).astype(np.int8)
    cert.certify_counts(gp, g.offsets, g.targets, out)
    bad = dict(out, val_counts=out["val_counts"].copy())
    bad["val_counts"][7, 0] += 1
    with pytest.raises(AssertionError):
        cert.certify_counts(gp, g.offsets, g.targets, bad)
    r = o3.run(gp, max_inner=2, allow_timeout=True)
    val = o3.valuate(gp, r["strat"])
    bo, be = cert.stopping_violations(gp, r["strat"], val, cert.count_vector_keys(gp, val))
    assert bo.size + be.size > 0
