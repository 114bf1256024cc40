"""Autotuner of the valuation's work partitioning (pg_set_tuning).

For each size bucket it times full solves of a seeded random game (out-degree
U[2,5], owners p = 0.5, permuted priorities) and one valuation of a long
successor chain (an n-vertex play along a random permutation) under
candidate settings, by coordinate descent from the library's defaults:

  walk_cap      steps of a direct nearest-greater walk before pointer jumping
  switch_block  threads per block of the switching passes
  loop_ranks    loop iterations that rank every valuation instead of comparing
  deep_cut      the chain length that hands a call to the ruling-set ranks
  ruler_bits    the ruling set's density (one ruler in 2^ruler_bits)

Every candidate's results (winners, strategies, ranks, depths) must equal the
defaults' bit for bit; a candidate that differs is an error, never a choice.
The winner of each bucket becomes one line of the tuning table that
pg_load_tuning reads (and pg_ctx_create, through PG_TUNING_FILE or the
binding's per-device default); the timings go to a JSON report.

    python -m paper_1705_02313_gb300.tune [--sizes 10000,100000,1000000,10000000]
        [--reps 3] [--table path] [--report path]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CANDIDATES = {
    "walk_cap": [16, 32, 64, 128],
    "switch_block": [128, 256, 512],
    "loop_ranks": [0, 1],
    "deep_cut": [8, 16, 64, 256],
    "ruler_bits": [3, 5, 7],
}
DEFAULTS = {"walk_cap": 64, "switch_block": 256, "loop_ranks": 0, "deep_cut": 64, "ruler_bits": 5}
FIELDS = ("deep_cut", "ruler_bits", "walk_cap", "switch_block", "loop_ranks")


def device_slug(name):
    """File-name form of a device name ("NVIDIA GB300" -> "nvidia_gb300")."""
    return "".join(c if c.isalnum() else "_" for c in name.strip().lower()).strip("_") or "device"


def default_table_path(device_name):
    return os.path.join(HERE, "tuning", device_slug(device_name) + ".txt")


def bucket_bounds(sizes):
    """max_ids of each bucket: the geometric midpoint to the next size (ids of
    G' are about 1.33 n for the random workload), the last one unbounded."""
    ids = [int(1.34 * s) + 2 for s in sizes]
    out = []
    for i in range(len(ids)):
        out.append(int(math.sqrt(ids[i] * ids[i + 1])) if i + 1 < len(ids) else 2**62)
    return out


def table_text(entries, device_name, note=""):
    """The table as pg_load_tuning reads it."""
    lines = ["# tuning table for %s, written by paper_1705_02313_gb300/tune.py%s" % (device_name, note),
             "# max_ids deep_cut ruler_bits walk_cap switch_block loop_ranks"]
    for max_ids, best in entries:
        lines.append("%d %d %d %d %d %d" % (max_ids, best["deep_cut"], best["ruler_bits"], best["walk_cap"],
                                            best["switch_block"], best["loop_ranks"]))
    return "\n".join(lines) + "\n"


def coordinate_descent(measure, passes=2):
    """Minimises measure(setting) one parameter at a time, from DEFAULTS.
    Returns (best setting, best time, {setting key: time})."""
    seen = {}

    def cost(st):
        key = tuple(st[f] for f in FIELDS)
        if key not in seen:
            seen[key] = measure(dict(st))
        return seen[key]

    best = dict(DEFAULTS)
    best_t = cost(best)
    for _ in range(passes):
        changed = False
        for name, values in CANDIDATES.items():
            for v in values:
                if v == best[name]:
                    continue
                st = dict(best)
                st[name] = v
                t = cost(st)
                if t < best_t * 0.98:  # a clear gain only: flat responses keep the defaults
                    best, best_t, changed = st, t, True
        if not changed:
            break
    return best, best_t, {",".join("%s=%d" % (f, k[i]) for i, f in enumerate(FIELDS)): t for k, t in seen.items()}


class Runner:
    """Times solves and chain valuations on the GPU under one setting at a
    time (a one-entry tuning table), checking results against the defaults."""

    def __init__(self, reps=3):
        import torch

        from paper_1705_02313_gb300 import build, pg
        build.build()
        self.torch, self.pg, self.reps = torch, pg, reps
        self.ctx = pg.pg_ctx_create(0, tuning=False)
        self.stream = torch.cuda.Stream()
        pg.pg_set_stream(self.ctx, self.stream)

    def set(self, st):
        self.pg.pg_set_tuning_table(self.ctx, [(2**62, st)])

    def solve_case(self, n, seed=0):
        from paper_1705_02313_gb300 import gen
        torch = self.torch
        g = gen.native_random_game(n, 2, 5, seed)
        d_in = [torch.from_numpy(a).cuda() for a in g.arrays()]
        ref = {}

        def measure(st):
            self.set(st)
            times = []
            out = None
            for _ in range(self.reps + 1):
                game = self.pg.pg_load_csr(self.ctx, g.n, g.m, *d_in)
                try:
                    out = {k: torch.empty(g.n, dtype=dt, device="cuda") for k, dt in
                           (("win", torch.uint8), ("sigma", torch.int32), ("tau", torch.int32),
                            ("val_rank", torch.int32), ("val_depth", torch.int32))}
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(self.stream)
                    self.pg.pg_solve(self.ctx, game, **out)
                    e1.record(self.stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                finally:
                    self.pg.pg_game_free(game)
            if not ref:
                ref.update(out)
            for k, v in out.items():
                if not torch.equal(v, ref[k]):
                    raise RuntimeError("setting %s changed %s: results must not depend on the tuning" % (st, k))
            return float(np.median(times[1:]))

        return measure

    def chain_case(self, n, seed=7):
        from paper_1705_02313_gb300 import gen
        torch = self.torch
        g, sigma = gen.chain_profile(n, seed=seed)
        d_in = [torch.from_numpy(a).cuda() for a in g.arrays()]
        d_sig = torch.from_numpy(sigma).cuda()
        game = self.pg.pg_load_csr(self.ctx, g.n, g.m, *d_in)
        ref = {}

        def measure(st):
            self.set(st)
            times = []
            out = None
            for _ in range(self.reps + 1):
                out = dict(val_rank=torch.empty(n, dtype=torch.int32, device="cuda"),
                           val_depth=torch.empty(n, dtype=torch.int32, device="cuda"))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(self.stream)
                self.pg.pg_valuate(self.ctx, game, d_sig, None, None, **out)
                e1.record(self.stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            if not ref:
                ref.update(out)
            for k, v in out.items():
                if not torch.equal(v, ref[k]):
                    raise RuntimeError("setting %s changed %s: results must not depend on the tuning" % (st, k))
            return float(np.median(times[1:]))

        return measure, game

    def close(self):
        self.pg.pg_ctx_destroy(self.ctx)


def tune(sizes, reps=3, chain=True, log=print):
    """Runs the tuner on the current GPU; returns (report, table entries).
    The objective of a bucket is the time of one full solve of the random
    workload plus (with chain) one valuation of the long chain, so that the
    walk and switch parameters answer to the solve and the ruling-set cutover
    to both: a table entry is chosen by size alone, whatever the game's shape."""
    import torch
    r = Runner(reps)
    name = torch.cuda.get_device_name(0)
    report = {"device": name, "reps": reps, "candidates": CANDIDATES, "defaults": DEFAULTS, "buckets": []}
    entries = []
    try:
        for n, max_ids in zip(sizes, bucket_bounds(sizes)):
            t0 = time.time()
            solve = r.solve_case(n)
            parts = {}
            game = None
            if chain:
                chain_measure, game = r.chain_case(n)
            try:
                def measure(st):
                    ts = solve(st)
                    tc = chain_measure(st) if chain else 0.0
                    parts[",".join("%s=%d" % (f, st[f]) for f in FIELDS)] = {"solve_ms": ts, "chain_ms": tc}
                    return ts + tc
                best, best_t, seen = coordinate_descent(measure)
            finally:
                if game is not None:
                    r.pg.pg_game_free(game)
            dkey = ",".join("%s=%d" % (f, DEFAULTS[f]) for f in FIELDS)
            bkey = ",".join("%s=%d" % (f, best[f]) for f in FIELDS)
            b = {"n": n, "max_ids": max_ids,
                 "objective": "ms of one full solve of a random game (out-degree U[2,5], seed 0)" +
                              (" + one valuation of a successor chain through all n vertices" if chain else ""),
                 "best": best, "best_ms": parts[bkey], "default_ms": parts[dkey], "measured": parts,
                 "tuning_s": round(time.time() - t0, 1)}
            entries.append((max_ids, best))
            report["buckets"].append(b)
            log("n=%d best %s %s (default %s)" % (n, best, parts[bkey], parts[dkey]))
    finally:
        r.close()
    return report, entries


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--sizes", default="10000,100000,1000000,10000000")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--no-chain", action="store_true")
    ap.add_argument("--table", default="", help="table path (default: tuning/<device>.txt next to this file)")
    ap.add_argument("--report", default="", help="JSON report path (default: next to the table)")
    args = ap.parse_args(argv)
    sizes = [int(x) for x in args.sizes.split(",") if x]
    report, entries = tune(sizes, args.reps, chain=not args.no_chain)
    table = args.table or default_table_path(report["device"])
    os.makedirs(os.path.dirname(os.path.abspath(table)), exist_ok=True)
    with open(table, "w") as f:
        f.write(table_text(entries, report["device"]))
    rep = args.report or os.path.splitext(table)[0] + ".json"
    with open(rep, "w") as f:
        json.dump(report, f, indent=1)
        f.write("\n")
    print("wrote", table, "and", rep)
    return 0


if __name__ == "__main__":
    sys.exit(main())
