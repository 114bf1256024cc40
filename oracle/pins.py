"""Independent checks that pin the oracle to the paper and to mathematics.

TEST INFRASTRUCTURE ONLY.

None of these functions reuses the oracle's valuation, comparison or
switching code:
  * ``brute_force_winners``: the winning sets of Section 2 by enumerating
    every pair of positional strategies of the ORIGINAL game (no sink, no
    dummies). Positional determinacy (the theorem of Section 2) and the fact
    that one-player parity games have positional optimal strategies make this
    exact.
  * ``zielonka_winners``: Zielonka's recursive algorithm (the textbook
    algorithm, written from its definition with attractors).
  * ``closed_form_value``: a big-integer encoding of the valuation order of
    Section 3. Priority p contributes sign(p) * L(p) * B**rank(p) where sign is
    +1 for even and -1 for odd priorities, rank(p) orders the priorities used
    by the game, and B exceeds every count. Comparing these integers compares
    the count vectors from their largest differing priority downwards, which is
    exactly the Maxdiff rule.
  * ``bellman_ford_values``: the best-response valuation Val^sigma (Section 3)
    as shortest paths to the sink under that order (Section 4 mentions this
    method), computed with the big-integer encoding.
  * ``euler_tour``: the sequential list construction of Section 5 ("Constructing
    the list ranking instance in parallel") and the list-ranking valuation of the
    formal reduction (up edges weigh A_{-p}, down edges A_{p}).
"""
from __future__ import annotations

import itertools


# ---------------------------------------------------------------------------
# Section 2: plays, MaxIo and the winner, by brute force

def _winner_of_play(start, succ, pri):
    """Winner (0 Even, 1 Odd) of the unique play from ``start`` when every
    vertex follows ``succ``: the parity of the largest priority on the cycle
    that the play eventually repeats forever."""
    seen = {}
    path = []
    x = start
    while x not in seen:
        seen[x] = len(path)
        path.append(x)
        x = succ[x]
    cycle = path[seen[x]:]
    return max(pri[y] for y in cycle) % 2


def brute_force_winners(n, off, tgt, own, pri):
    """W_Even as a sorted list: v is in W_Even iff some positional sigma
    makes every positional tau lose from v."""
    even = [v for v in range(n) if own[v] == 0]
    odd = [v for v in range(n) if own[v] == 1]
    choices = {v: [int(tgt[e]) for e in range(off[v], off[v + 1])] for v in range(n)}
    wins_for_even = [False] * n
    for sig in itertools.product(*[choices[v] for v in even]):
        good = [True] * n
        for tau in itertools.product(*[choices[v] for v in odd]):
            succ = [0] * n
            for v, t in zip(even, sig):
                succ[v] = t
            for v, t in zip(odd, tau):
                succ[v] = t
            for v in range(n):
                if good[v] and _winner_of_play(v, succ, pri) == 1:
                    good[v] = False
        for v in range(n):
            wins_for_even[v] |= good[v]
    return [v for v in range(n) if wins_for_even[v]]


# ---------------------------------------------------------------------------
# Zielonka's recursive algorithm

def _attractor(player, target, alive, succs, preds, own):
    attr = set(target)
    count = {}
    stack = list(target)
    while stack:
        x = stack.pop()
        for y in preds[x]:
            if y not in alive or y in attr:
                continue
            if own[y] == player:
                attr.add(y)
                stack.append(y)
            else:
                if y not in count:
                    count[y] = sum(1 for z in succs[y] if z in alive)
                count[y] -= 1
                if count[y] == 0:
                    attr.add(y)
                    stack.append(y)
    return attr


def zielonka_winners(n, off, tgt, own, pri):
    """(W_Even, W_Odd) as sets, by Zielonka's recursive algorithm."""
    succs = [[int(tgt[e]) for e in range(off[v], off[v + 1])] for v in range(n)]
    preds = [[] for _ in range(n)]
    for v in range(n):
        for u in succs[v]:
            preds[u].append(v)

    def solve(alive):
        if not alive:
            return set(), set()
        p = max(pri[v] for v in alive)
        i = p % 2
        top = {v for v in alive if pri[v] == p}
        A = _attractor(i, top, alive, succs, preds, own)
        W = solve(alive - A)
        if not W[1 - i]:
            res = [set(), set()]
            res[i] = set(alive)
            return res[0], res[1]
        B = _attractor(1 - i, W[1 - i], alive, succs, preds, own)
        W2 = solve(alive - B)
        res = [set(), set()]
        res[1 - i] = W2[1 - i] | B
        res[i] = W2[i]
        return res[0], res[1]

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 10 * n + 1000))
    try:
        return solve(set(range(n)))
    finally:
        sys.setrecursionlimit(old)


# ---------------------------------------------------------------------------
# Closed form of the valuation order and Bellman-Ford best responses

class Encoding:
    """Integer encoding of count vectors: value(L) = sum over p of
    sign(p) * L(p) * B**rank(p)."""

    def __init__(self, pri, max_count):
        prios = sorted(set(int(p) for p in pri))
        self.rank = {p: i for i, p in enumerate(prios)}
        self.B = 2 * max_count + 3

    def unit(self, p):
        return (1 if p % 2 == 0 else -1) * self.B ** self.rank[p]


TOP_VALUE = float("inf")


def closed_form_value(pri, strat, sink, v, enc):
    """Integer value of Val(v) under the profile, or TOP_VALUE for an
    infinite play."""
    seen = set()
    total = 0
    x = v
    while x != sink:
        if x in seen:
            return TOP_VALUE
        seen.add(x)
        total += enc.unit(pri[x])
        x = strat[x]
    return total


def bellman_ford_values(gp, sigma):
    """Val^sigma: for Even vertices the edge is fixed by sigma (the sink is
    id n); Odd vertices minimise. Shortest paths to the sink with
    edge weight = the unit of the vertex left, by Bellman-Ford relaxation
    from TOP everywhere. Returns a list of integers / TOP_VALUE (sink last)."""
    n = gp["n"]
    pri, own, off, tgt = gp["pri"], gp["own"], gp["off"], gp["tgt"]
    enc = Encoding(pri, n)
    dist = [TOP_VALUE] * n + [0]
    for _ in range(n + 1):
        changed = False
        for v in range(n):
            if own[v] == 0:
                best = dist[sigma[v]]
            else:
                best = min(dist[int(tgt[e])] for e in range(off[v], off[v + 1]))
            cand = TOP_VALUE if best == TOP_VALUE else best + enc.unit(pri[v])
            if cand < dist[v]:
                dist[v] = cand
                changed = True
        if not changed:
            break
    return dist


# ---------------------------------------------------------------------------
# Section 5: Euler tour list and the list-ranking valuation

def euler_tour(parent, root, order):
    """The sequential construction of Section 5. Every non-root vertex v owns
    a down element (parent(v), v) and an up element (v, parent(v)); start_v
    initially points at the down element (a head sentinel for the root) and
    end_v at the up element (an end sentinel for the root). Processing v with
    parent u links the element start_u points at to v's down element and then
    sets start_u = end_v; finally every start_v is linked to end_v. Returns the
    list of (x, y) elements from the head sentinel to the end sentinel."""
    HEAD, END = ("head",), ("end",)
    start, end, link = {}, {}, {}
    verts = set(parent) | {root}
    for v in verts:
        if v == root:
            start[v], end[v] = HEAD, END
        else:
            start[v], end[v] = (parent[v], v), (v, parent[v])
    down = {v: (parent[v], v) for v in parent}
    for v in order:
        u = parent[v]
        link[start[u]] = down[v]
        start[u] = end[v]
    for v in verts:
        link[start[v]] = end[v]
    out = []
    x = link[HEAD]
    while x != END:
        out.append(x)
        x = link[x]
    return out


def list_ranking_valuation(parent, root, order, pri):
    """Count vectors of every non-root vertex by list ranking over the Euler
    tour (formal reduction of Section 5): an up element (v, u) weighs A_{-pri(v)},
    a down element (u, v) weighs A_{pri(v)}; the exclusive prefix sum at v's up
    element is v's count vector (the play from v, v included, root excluded)."""
    tour = euler_tour(parent, root, order)
    acc = {}
    out = {}
    for (x, y) in tour:
        if parent.get(x) == y:        # up element (x, parent(x))
            out[x] = {p: c for p, c in acc.items() if c}
            acc[pri[x]] = acc.get(pri[x], 0) - 1
        else:                         # down element (x, y), y a child of x
            acc[pri[y]] = acc.get(pri[y], 0) + 1
    return out
