"""CPU oracle for greedy all-switches strategy improvement on parity games.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call, link or execute anything in
this folder; the CUDA path shares no code with it and never calls it.

Modules:
  o1        definitional oracle: literal count vectors and Maxdiff (Section 3),
            Algorithm 1 step by step (Section 4); any priorities, small games.
  o2        scalable oracle in plain C (o2.c): same algorithm, distinct
            priorities, ranks by Kruskal merge order; used at every size.
  pins      independent checks the oracle is pinned against: brute force over
            positional strategies, Zielonka's recursive algorithm, Bellman-Ford
            under the valuation order, the Euler-tour list of Section 5.
"""
