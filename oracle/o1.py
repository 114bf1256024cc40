"""Definitional CPU oracle (O-1) for small games.

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
baseline may use it; the product path never does.

Everything here follows the paper's definitions literally, with no encoding
tricks: a finite valuation is the count vector L(p) of Section 3
("Valuations"), compared by Maxdiff (same paragraph); the switching rules are
the greedy all-switches rule for Even (Section 3, "Switching rules") and
All_Odd (Section 4); the loop is Algorithm 1 (Section 4). Priorities need not
be distinct. Intended for games of at most a few thousand vertices.

Readings of points the paper leaves open (shared with every other solver in
this repository):
  * the preprocessing of Section 3 inserts one dummy Even vertex per vertex of
    Odd's Even-free trap U entered from U (see ``preprocess``);
  * a switch happens only when strictly better; among equally good
    successors the lowest edge-list position wins; Even looks at the sink
    first;
  * the initial Odd strategy takes the first edge of each list;
  * the Odd-switchability condition of Section 4 compares against tau(v)
    (the text writes sigma(v), which Odd vertices do not have).
"""
from __future__ import annotations

import functools

FIN, TOP, ODDCYCLE = 0, 1, 2
INT32_MAX = 2**31 - 1


# ---------------------------------------------------------------------------
# Preprocessing (Section 3, "The algorithm": dummy Even vertices)

def odd_trap(n, off, tgt, own):
    """Greatest set U of Odd vertices each of which has an edge into U: from
    U, Odd can keep the play away from Even vertices forever. Computed as a
    plain greatest fixpoint by repeated removal."""
    U = {v for v in range(n) if own[v] == 1}
    changed = True
    while changed:
        changed = False
        for v in sorted(U):
            if not any(int(tgt[e]) in U for e in range(off[v], off[v + 1])):
                U.discard(v)
                changed = True
    return U


def preprocess(n, off, tgt, own, pri, dummy_zero=None):
    """Builds G' from G: for each w in U that some edge from U enters (W, in
    increasing id order), dummy vertex n + j (j = index of w in W) is an Even
    vertex of priority 2j with the single edge to w; edges U -> w are
    redirected to it; every original priority p becomes p + 2|W|. When the
    priorities repeat (or dummy_zero is set) every dummy gets priority 0 and
    every original priority p becomes p + 2 instead, so that the dummies add
    one priority rather than |W|. Returns a dict with the new CSR arrays as
    Python lists plus ``dummy_of`` and ``k``."""
    if dummy_zero is None:
        dummy_zero = len(set(int(p) for p in pri)) < n
    U = odd_trap(n, off, tgt, own)
    W = sorted({int(tgt[e]) for v in U for e in range(off[v], off[v + 1]) if int(tgt[e]) in U})
    k = len(W)
    index = {w: j for j, w in enumerate(W)}
    noff, ntgt, nown, npri = [0], [], [], []
    for v in range(n):
        for e in range(off[v], off[v + 1]):
            t = int(tgt[e])
            ntgt.append(n + index[t] if (v in U and t in U) else t)
        noff.append(len(ntgt))
        nown.append(int(own[v]))
        npri.append(int(pri[v]) + (2 if dummy_zero else 2 * k))
    for j, w in enumerate(W):
        ntgt.append(w)
        noff.append(len(ntgt))
        nown.append(0)
        npri.append(0 if dummy_zero else 2 * j)
    return dict(n=n + k, off=noff, tgt=ntgt, own=nown, pri=npri, dummy_of=W, k=k, U=U, n_orig=n,
                dummy_zero=bool(dummy_zero))


# ---------------------------------------------------------------------------
# Valuations (Section 3)

def play(strat, sink, v):
    """The play from v under the profile (strat[x] = sigma(x) or tau(x)),
    cut when it reaches the sink or repeats a vertex. Returns (vertices,
    index of the first repeated vertex or None when the sink was reached)."""
    seen = {}
    path = []
    x = v
    while x != sink and x not in seen:
        seen[x] = len(path)
        path.append(x)
        x = strat[x]
    return path, (None if x == sink else seen[x])


def valuation(pri, strat, sink, v):
    """Val(v): TOP for an infinite play, else the count of each priority on
    v_0 .. v_k (v_0 included, the sink excluded). Returned as (kind, L, dom)
    with L a dict priority -> count and dom the largest priority on the cycle
    of an infinite play."""
    path, cyc = play(strat, sink, v)
    if cyc is not None:
        dom = max(pri[x] for x in path[cyc:])
        return (TOP if dom % 2 == 0 else ODDCYCLE, None, dom)
    L = {}
    for x in path:
        L[pri[x]] = L.get(pri[x], 0) + 1
    return (FIN, L, -1)


def maxdiff(L1, L2):
    """Largest priority whose counts differ, or None when L1 = L2."""
    keys = [p for p in set(L1) | set(L2) if L1.get(p, 0) != L2.get(p, 0)]
    return max(keys) if keys else None


def compare(a, b):
    """-1, 0, +1 as valuation a is below, equal to, above b under the order
    of Section 3; TOP is above every finite valuation."""
    (ka, La, _), (kb, Lb, _) = a, b
    if ka != FIN or kb != FIN:
        ta, tb = ka != FIN, kb != FIN
        return (ta > tb) - (ta < tb)
    p = maxdiff(La, Lb)
    if p is None:
        return 0
    if p % 2 == 0:
        return -1 if La.get(p, 0) < Lb.get(p, 0) else 1
    return -1 if La.get(p, 0) > Lb.get(p, 0) else 1


SINK_VAL = (FIN, {}, -1)


def all_valuations(gp, strat):
    sink = gp["n"]
    return [valuation(gp["pri"], strat, sink, v) for v in range(gp["n"])] + [SINK_VAL]


# ---------------------------------------------------------------------------
# Switching rules

def switch(gp, strat, vals, player):
    """Greedy all-switches for ``player`` (0 Even: maximise, sink first;
    1 Odd: minimise). Returns (new strat, number of switched vertices)."""
    n, off, tgt, own = gp["n"], gp["off"], gp["tgt"], gp["own"]
    new = list(strat)
    count = 0
    want = 1 if player == 0 else -1
    for v in range(n):
        if own[v] != player:
            continue
        cands = ([n] if player == 0 else []) + [tgt[e] for e in range(off[v], off[v + 1])]
        best = cands[0]
        for u in cands[1:]:
            if compare(vals[u], vals[best]) == want:
                best = u
        if compare(vals[best], vals[strat[v]]) == want:
            new[v] = best
            count += 1
    return new, count


def initial_profile(gp):
    """sigma_init (every Even vertex to the sink) and the first-edge tau."""
    n = gp["n"]
    return [n if gp["own"][v] == 0 else gp["tgt"][gp["off"][v]] for v in range(n)]


def ranks(gp, vals):
    """Position of each finite valuation (and the sink's) in the total order;
    INT32_MAX for TOP. Returns (rank list for vertices, sink rank)."""
    n = gp["n"]
    fin = [v for v in range(n + 1) if vals[v][0] == FIN]
    fin.sort(key=functools.cmp_to_key(lambda a, b: compare(vals[a], vals[b])))
    r = [INT32_MAX] * (n + 1)
    for i, v in enumerate(fin):
        r[v] = i
    return r[:n], r[n]


def result_of(gp, strat, vals, major, inner):
    rank, sink_rank = ranks(gp, vals)
    cls = [vals[v][0] for v in range(gp["n"])]
    depth = [sum(vals[v][1].values()) if vals[v][0] == FIN else -1 for v in range(gp["n"])]
    dom = [vals[v][2] for v in range(gp["n"])]
    # count vectors over the distinct priorities of G' in ascending order (zeros for top)
    level_pri = sorted(set(gp["pri"]))
    counts = [[vals[v][1].get(p, 0) for p in level_pri] if vals[v][0] == FIN else [0] * len(level_pri)
              for v in range(gp["n"])]
    return dict(strat=list(strat), cls=cls, depth=depth, rank=rank, sink_rank=sink_rank, dom=dom,
                major=major, inner=inner, counts=counts, level_pri=level_pri)


class NotAdmissible(Exception):
    pass


def run(gp, strat=None, mode="solve", max_inner=10**6, trace=None):
    """Algorithm 1 (Section 4). mode "solve" runs both loops; mode
    "best_response" runs the inner loop only; mode "solve_reset" runs both
    loops but starts every best-response computation again from the initial
    Odd strategy (the SI-Reset variant of Section 6). ``trace`` (a list)
    receives (phase, strat, vals) after every valuation, for invariant
    checks."""
    strat = initial_profile(gp) if strat is None else list(strat)
    major = inner = 0
    while True:
        while True:
            if inner >= max_inner:
                raise TimeoutError("inner iteration cap reached")
            vals = all_valuations(gp, strat)
            if any(v[0] == ODDCYCLE for v in vals):
                raise NotAdmissible("odd cycle under the current profile")
            inner += 1
            if trace is not None:
                trace.append(("inner", list(strat), vals))
            strat, count = switch(gp, strat, vals, 1)
            if count == 0:
                break
        if mode == "best_response":
            break
        strat, count = switch(gp, strat, vals, 0)
        if count == 0:
            break
        major += 1
        if mode == "solve_reset":
            init = initial_profile(gp)
            strat = [init[v] if gp["own"][v] == 1 else strat[v] for v in range(gp["n"])]
    return result_of(gp, strat, vals, major, inner)


def valuate(gp, strat):
    vals = all_valuations(gp, strat)
    return result_of(gp, strat, vals, 0, 0)


def map_back(gp, res):
    """Results in original vertex ids: winner (0 Even, 1 Odd), sigma (-1 for
    the sink or Odd vertices), tau (a dummy reported as the vertex it guards;
    -1 for Even vertices), class (1 top, 0 finite), depth, rank."""
    n0, n = gp["n_orig"], gp["n"]
    dummy_of = gp["dummy_of"]
    win, sigma, tau, vc, vd, vr = [], [], [], [], [], []
    for v in range(n0):
        s = res["strat"][v]
        top = res["cls"][v] != FIN
        win.append(0 if top else 1)
        if gp["own"][v] == 0:
            sigma.append(-1 if s == n else s)
            tau.append(-1)
        else:
            sigma.append(-1)
            tau.append(dummy_of[s - n0] if s >= n0 else s)
        vc.append(1 if top else 0)
        vd.append(res["depth"][v])
        vr.append(res["rank"][v])
    return dict(win=win, sigma=sigma, tau=tau, val_class=vc, val_depth=vd, val_rank=vr)


def solve_game(n, off, tgt, own, pri, reset=False):
    """Convenience: preprocess, run Algorithm 1 (SI-Reset with reset=True), map back."""
    gp = preprocess(n, list(off), list(tgt), list(own), list(pri))
    res = run(gp, mode="solve_reset" if reset else "solve")
    out = map_back(gp, res)
    out.update(major=res["major"], inner=res["inner"])
    return gp, res, out
