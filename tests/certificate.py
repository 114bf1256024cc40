"""Checks of a solved profile that hold at any size, with values from the
oracle only.

Algorithm 1 stops when, under the valuation of the current profile, no Odd
vertex has an edge to a strictly smaller value than its current successor's
and no Even vertex has an edge (or the sink) to a strictly greater one
(Section 3, switching rules; Section 4, the loop). Such a profile is optimal
for both players (Theorem 1), so it fixes the winning regions. Given a
profile, the oracle values it (Section 3) and numpy checks the stopping
condition over every vertex and edge.
"""
import numpy as np

from oracle import o2


def profile_to_gprime(gp, offsets, targets, sigma, tau, dummy_sigma):
    """The profile of G' (one successor per id, the sink = n') for a profile
    in original ids as the C ABI reports it: sigma = -1 for the sink, a
    dummy d_w reported as w in tau, dummy_sigma = 1 where a dummy takes its
    edge. G' keeps the edge positions of every original vertex, and only
    Odd vertices' edges are redirected to dummies, so the successor of an Odd
    vertex is the G' target at the position of the reported one."""
    n0, n = gp["n_orig"], gp["n"]
    offsets = np.asarray(offsets, np.int64)
    targets = np.asarray(targets, np.int32)
    m0 = int(offsets[-1])
    assert np.array_equal(gp["off"][: n0 + 1], offsets)
    own = gp["own"][:n0]
    strat = np.empty(n, np.int32)
    sigma = np.asarray(sigma, np.int64)
    strat[:n0] = np.where(sigma < 0, n, sigma)
    src = np.repeat(np.arange(n0, dtype=np.int64), np.diff(offsets))
    hit = (own[src] == 1) & (targets == np.asarray(tau)[src])
    per_vertex = np.bincount(src[hit], minlength=n0)
    assert np.all(per_vertex[own == 1] == 1), "an Odd successor is not one of the vertex's edges"
    strat[src[hit]] = gp["tgt"][:m0][hit]
    k = gp["k"]
    if k:
        dt = gp["tgt"][gp["off"][n0:n]]
        strat[n0:] = np.where(np.asarray(dummy_sigma)[:k] != 0, dt, n)
    return strat


def switch_keys(gp, val):
    """Switching key of every id of G' plus the sink (index n'): the rank in
    the order of valuations (the sink's is its empty valuation's)."""
    n = gp["n"]
    key = np.empty(n + 1, np.int64)
    key[:n] = val["rank"]
    key[n] = val["sink_rank"]
    return key


def count_vector_keys(gp, val):
    """Switching key of every id of G' plus the sink for count-vector
    valuations (Section 3): a dense rank in the order where TOP is above
    every finite valuation and two finite ones compare at the highest
    priority whose counts differ (more is better for an even priority, fewer
    for an odd one); equal count vectors get equal keys."""
    n = gp["n"]
    lp = np.asarray(val["level_pri"], np.int64)
    counts = np.vstack([np.asarray(val["counts"], np.int64), np.zeros((1, lp.size), np.int64)])
    top = np.append(np.asarray(val["cls"]) != o2.FIN, False).astype(np.int64)
    signed = counts * np.where(lp % 2 == 0, 1, -1)[None, :]
    cols = [signed[:, j] for j in range(lp.size)] + [top]  # lexsort: the last key is the primary one
    order = np.lexsort(cols)
    sk = np.stack(cols, axis=1)[order]
    new = np.ones(n + 1, bool)
    new[1:] = np.any(sk[1:] != sk[:-1], axis=1)
    key = np.empty(n + 1, np.int64)
    key[order] = np.cumsum(new) - 1
    return key


def stopping_violations(gp, strat, val, key=None):
    """(Odd vertices with a strictly better edge, Even vertices with a
    strictly better edge or sink) under the valuation ``val`` of ``strat``
    (``key``: switching keys, by default the ranks of ``val``)."""
    n = gp["n"]
    key = switch_keys(gp, val) if key is None else key
    kt = key[gp["tgt"]]
    starts = gp["off"][:-1]
    lo = np.minimum.reduceat(kt, starts)
    hi = np.maximum.reduceat(kt, starts)
    cur = key[strat]
    odd = gp["own"][:n] == 1
    bad_odd = np.nonzero(odd & (lo < cur))[0]
    bad_even = np.nonzero(~odd & (np.maximum(hi, key[n]) > cur))[0]
    return bad_odd, bad_even


def certify(gp, offsets, targets, out):
    """Checks a solution reported in original ids (``out``: win, sigma, tau,
    dummy_sigma, val_class, val_depth, val_rank) against the oracle's
    valuation of the same profile. Returns the oracle's valuation."""
    strat = profile_to_gprime(gp, offsets, targets, out["sigma"], out["tau"], out["dummy_sigma"])
    val = o2.valuate(gp, strat)
    assert not np.any(val["cls"] == o2.ODDCYCLE), "the profile reaches an odd cycle"
    bad_odd, bad_even = stopping_violations(gp, strat, val)
    assert bad_odd.size == 0, "Odd can still switch at %d vertices, first %s" % (bad_odd.size, bad_odd[:5])
    assert bad_even.size == 0, "Even can still switch at %d vertices, first %s" % (bad_even.size, bad_even[:5])
    want = o2.map_back(gp, dict(val, strat=strat))
    for k in ("win", "sigma", "tau", "val_class", "val_depth", "val_rank"):
        a, b = np.asarray(out[k]), np.asarray(want[k])
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0]
            raise AssertionError("%s differs at %d vertices, first %s: got %s want %s" %
                                 (k, bad.size, bad[:5], a[bad[:5]], b[bad[:5]]))
    return val


def certify_counts(gp, offsets, targets, out):
    """certify() for games whose priorities repeat: the oracle's count-vector
    valuation (O-3) of the reported profile, the stopping condition under
    the count-vector order, and the reported count vectors."""
    from oracle import o3
    strat = profile_to_gprime(gp, offsets, targets, out["sigma"], out["tau"], out["dummy_sigma"])
    val = o3.valuate(gp, strat)
    assert val["status"] == o3.OK and not np.any(val["cls"] == o3.ODDCYCLE), "the profile reaches an odd cycle"
    bad_odd, bad_even = stopping_violations(gp, strat, val, count_vector_keys(gp, val))
    assert bad_odd.size == 0, "Odd can still switch at %d vertices, first %s" % (bad_odd.size, bad_odd[:5])
    assert bad_even.size == 0, "Even can still switch at %d vertices, first %s" % (bad_even.size, bad_even[:5])
    want = o3.map_back(gp, dict(val, strat=strat))
    for k in ("win", "sigma", "tau", "val_class", "val_depth", "val_counts"):
        a, b = np.asarray(out[k]), np.asarray(want[k])
        if not np.array_equal(a, b):
            bad = np.nonzero(np.any((a != b).reshape(a.shape[0], -1), axis=1))[0]
            raise AssertionError("%s differs at %d vertices, first %s" % (k, bad.size, bad[:5]))
    return val
