"""Benchmark: greedy all-switches strategy improvement on one 10M-vertex game.

One step = one whole solve through the C ABI: pg_load_csr from device-resident
input arrays (validation, the admissibility preprocessing and relabelling on
the GPU) followed by pg_solve to device-resident results (every inner and
outer iteration of Algorithm 1). The reported value is best-response edges/s:
input edges times valuations computed, divided by the step time (the whole
step, preprocessing and Even switches included).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (launched by torch.distributed.run): every rank solves its own replica
of the game (a single game does not shard: replicas only); value = edges *
valuations summed over ranks / the slowest rank's time. The batch leg shards
its games over the ranks instead (each rank solves its share alone).
--impl reference times the CPU oracle (oracle/o2.c, single thread) on a
bounded sample of the same workload: each step runs the first iterations of
the same solve.

Beside the headline the line carries: the end-to-end rate from pinned host
memory, the roofline of the inner iteration (B_alg = 8 m' + 20 n' bytes per
valuation + switching pass, over the solve time of the timed steps, against
the measured HBM bandwidth; DRAM traffic from the committed ncu summary while
the kernels' sources are unchanged), the dominant kernel, per-kernel times, SI-Reset, the 4-priority count-vector game, the
4,096-game batch (--batch batch-256 for a small one), a Poisson serving
stream (--serve seconds, 60 by default), an optional long-chain valuation (--chain n), and
the oracle timed on the host cores (one core for the solve; all cores, one
game per process, for the batch and serving samples).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "best-response edges/s (10M-vertex random parity game, full solve)"
UNIT = "edges/s"
WORKLOADS = {
    # name: (generator, kwargs, description)
    "random-10m": ("random_game", dict(n=10_000_000, dmin=2, dmax=5, seed=0),
                   "random game, n=10,000,000, out-degree U[2,5], owners p=0.5, permuted priorities, seed 0"),
    "random-1m": ("random_game", dict(n=1_000_000, dmin=2, dmax=8, seed=0),
                  "random game, n=1,000,000, out-degree U[2,8], owners p=0.5, permuted priorities, seed 0"),
    "random-6m": ("random_game", dict(n=6_000_000, dmin=2, dmax=5, seed=0),
                  "random game, n=6,000,000, out-degree U[2,5], owners p=0.5, permuted priorities, seed 0 "
                  "(profiling case: inputs above L2, about 1 GB on the device)"),
    "ladder-10m": ("ladder_game", dict(n=10_000_000, seed=0),
                   "ladder game, n=10,000,000, i->i+1 plus one back edge, owners p=0.5, permuted priorities"),
    "random-10m-4pri": ("random_game", dict(n=10_000_000, dmin=2, dmax=5, seed=0, levels=4),
                        "random game, n=10,000,000, out-degree U[2,5], owners p=0.5, priorities uniform over 0..3 "
                        "(count-vector mode; the shape of the verification games of Table 1)"),
}


def make_game(name):
    from paper_1705_02313_gb300 import gen
    fn, kw, _ = WORKLOADS[name]
    kw = dict(kw)
    if fn == "random_game":  # the C generator: the same game as gen.random_game
        return gen.native_random_game(kw["n"], kw["dmin"], kw["dmax"], kw["seed"], levels=kw.get("levels", 0))
    return gen.ladder_game(kw["n"], kw["seed"])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# per-kernel algorithmic bytes: the compulsory traffic of each pass (each per-id array once at its element size,
# one gather per edge)

def algorithmic_bytes(name, s):
    """Compulsory bytes of one launch of a kernel class: every per-id array
    read or written once at its element size, one gather per edge, chain and
    walk steps beyond the first not counted (they are the kernels' own cost).
    s: n = ids of G' (vertices, dummies, sink slot), m = edges, and the Odd /
    Even split of both."""
    n, m = s["n"], s["m"]
    table = {
        "walk": 9 * n,         # compare-mode walk (the loop's): strat 4 + flags 1 read; gd32 4 written
        "classify": 10 * n,    # gd32 4 + flags 1 read; top word 4 written; the top's parity 1 gathered
        "chain1": 15 * n,      # gd32 4 + flags 1 read; kind 1, cls 1, slot 4 written; one children-count atomic 4
        "child_scan": 8 * n,   # counts read, offsets written
        "scatter": 33 * n,     # kind 1, sz 4, gd32 4, slot 4, the parent's offset 4 read; entry 8, count 4, sink value 4 written
        "siblings": 20 * n,    # offsets 4, entries 8 read; weight 4, odd total 4 written
        "sink_scan": 8 * n,    # sink values 4 read, weights 4 written (the tile sums come with k_scatter)
        "chain2": 17 * n,      # flags 1, odd total 4, weight 4, gd32 4 read; key 4 written
        # the Odd view: vertex, offset, strategy; target + gather (a full pass: after the first of a solve the
        # pass evaluates only the vertices some of whose successors changed their top word)
        "switch_odd": 12 * s["n_odd"] + 8 * s["m_odd"],
        "switch_even": 12 * s["n_even"] + 8 * s["m_even"],
    }
    return table.get(name)


def kernel_entry(name, v, s, hbm):
    """Per kernel class: device ms over the timed solve, launches, calls, and
    algorithmic GB/s per call against the measured HBM copy bandwidth."""
    ms, launches, calls = v
    e = {"ms": ms, "launches": launches, "calls": calls}
    # the Even pass returns at once in iterations where Odd switched: per call it has no fixed work
    ab = algorithmic_bytes(name, s) if name != "switch_even" else None
    if ab and calls and ms > 0:
        gbs = ab / (ms / calls / 1000.0) / 1e9
        e.update(us_per_call=ms / calls * 1000.0, algorithmic_bytes=ab, achieved_gbs=gbs, frac_of_hbm=gbs / hbm)
    return e


# where each kernel class whose DRAM traffic is recorded is defined
KERNEL_SOURCE = {"chain1": ("pg_iter.cu", "k_chain1("), "classify": ("pg_iter.cu", "k_classify("),
                 "walk": ("pg_iter.cu", "k_walk_cmp("), "switch_odd": ("pg_iter.cu", "k_switch_cmp_pl(")}
# the files holding the kernels of one inner iteration (their traffic is recorded as "iteration")
ITERATION_SOURCES = ("pg_iter.cu", "pg_device.cuh", "pg_scan.cu")


def kernel_text(path, marker):
    """The source from the top of the file to the end of the definition that
    ``marker`` opens (the kernel with the helpers and constants before it)."""
    text = open(path, "rb").read()
    i = text.index(marker.encode())
    j = text.index(b"{", i)
    depth = 0
    for k in range(j, len(text)):
        c = text[k:k + 1]
        if c == b"{":
            depth += 1
        elif c == b"}":
            depth -= 1
            if depth == 0:
                return text[:k + 1]
    return text


def kernel_source_hash(kernel="chain1"):
    """Hash of what the kernel is compiled from: its source up to the end of
    its definition and the compile-time constants of the internal header
    (code after it and host-side structures do not change it)."""
    csrc = os.path.join(ROOT, "paper_1705_02313_gb300", "csrc")
    h = hashlib.sha256()
    if kernel == "iteration":  # every kernel of one inner iteration: the whole files they are compiled from
        for fname in ITERATION_SOURCES:
            with open(os.path.join(csrc, fname), "rb") as fh:
                h.update(fh.read())
    else:
        fname, marker = KERNEL_SOURCE.get(kernel, ("pg_iter.cu", "k_%s(" % kernel))
        h.update(kernel_text(os.path.join(csrc, fname), marker))
    with open(os.path.join(csrc, "pg_internal.cuh"), "rb") as fh:
        for line in fh.read().splitlines():
            if line.strip().startswith(b"constexpr"):
                h.update(line + b"\n")
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload):
    """dram bytes per launch of ``kernel`` from the committed ncu summary, if
    it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        e = t[workload][kernel]
        if e.get("source_hash") != kernel_source_hash(kernel):
            return None
        return e["dram_bytes_per_launch"]
    except Exception:
        return None


# ---------------------------------------------------------------------------
# one long successor chain: the valuation alone (nearest-greater walks that run
# out of steps, pointer jumping, ranks along an n-long list)

def chain_measure(n, ctx, reps=3):
    import torch

    from paper_1705_02313_gb300 import gen, pg
    g, sigma = gen.chain_profile(n, seed=7)
    d_in = [torch.from_numpy(a).cuda() for a in g.arrays()]
    d_sig = torch.from_numpy(sigma).cuda()
    game = pg.pg_load_csr(ctx, g.n, g.m, *d_in)
    try:
        vr = torch.empty(n, dtype=torch.int32, device="cuda")
        pg.pg_valuate(ctx, game, d_sig, None, None, val_rank=vr)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            pg.pg_valuate(ctx, game, d_sig, None, None, val_rank=vr)
        e1.record()
        torch.cuda.synchronize()
        c = pg.pg_game_counters(game)
    finally:
        pg.pg_game_free(game)
    ms = e0.elapsed_time(e1) / reps
    return {"workload": "chain-%d" % n, "description": "one successor chain through all %d vertices (an all-Even game, "
            "chain along a random permutation, one extra random edge per vertex), valuation only" % n,
            "valuation_ms": ms, "pending_walks": c["n_pending"], "jump_rounds": c["jump_rounds"],
            "vertices_per_s": n / (ms / 1000.0)}


# ---------------------------------------------------------------------------
# count-vector mode: games whose priorities repeat

def cv_measure(name, ctx, steps=3):
    """Full solves of a repeated-priority workload: one warm-up, then steps
    solves (load + solve from device arrays, results to device), CUDA events."""
    import torch

    from paper_1705_02313_gb300 import pg
    game = make_game(name)
    n, m = game.n, game.m
    d_in = [torch.from_numpy(a).cuda() for a in game.arrays()]
    win = torch.empty(n, dtype=torch.uint8, device="cuda")
    levels = None

    def one():
        nonlocal levels
        g = pg.pg_load_csr(ctx, n, m, *d_in)
        try:
            levels = pg.pg_game_levels(g)
            cnt = torch.empty(n * max(levels.size, 1), dtype=torch.int32, device="cuda")
            return pg.pg_solve(ctx, g, win=win, val_counts=cnt)
        finally:
            pg.pg_game_free(g)

    one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    inner_total = 0
    for _ in range(steps):
        major, inner = one()
        inner_total += inner
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # best responses two ways (Section 4 and Table 2): one-player strategy
    # improvement against Bellman-Ford, from sigma_init and from the final sigma
    g = pg.pg_load_csr(ctx, n, m, *d_in)
    br = {}
    try:
        sig_final = torch.empty(n, dtype=torch.int32, device="cuda")
        pg.pg_solve(ctx, g, sigma=sig_final)
        for label, sig in [("sigma_init", torch.full((n,), -1, dtype=torch.int32, device="cuda")),
                           ("sigma_final", sig_final)]:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it = pg.pg_best_response(ctx, g, sig)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            rounds = pg.pg_best_response_bf(ctx, g, sig)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            br[label] = {"si_ms": (t1 - t0) * 1e3, "si_iterations": it, "bellman_ford_ms": (t2 - t1) * 1e3,
                         "bellman_ford_rounds": rounds}
    finally:
        pg.pg_game_free(g)
    return {"workload": name, "description": WORKLOADS[name][2], "n": n, "m": m, "levels_of_g_prime": levels.tolist(),
            "major_iterations": major, "valuations_per_solve": inner, "full_solve_ms": ms,
            "edges_per_s": m * inner_total / (ms * steps / 1000.0), "unit": "edges/s",
            "inner_iteration_us": ms * 1000.0 / inner, "best_response": br}


# ---------------------------------------------------------------------------
# batches: pg_solve_batch against a loop of pg_load_csr + pg_solve

BATCHES = {
    # name: (games, size lo, size hi, out-degree lo, hi, description)
    "batch-256": (256, 1_000, 100_000, 2, 6,
                  "256 random games, sizes log-uniform in [1e3, 1e5], out-degree U[2,6], owners p=0.5, permuted "
                  "priorities, game i seeded by SplitMix64(0x5EED ^ i)"),
    "batch-4096": (4096, 1_000, 1_000_000, 2, 6,
                   "4,096 random games, sizes log-uniform in [1e3, 1e6], out-degree U[2,6], owners p=0.5, permuted "
                   "priorities, game i seeded by SplitMix64(0x5EED ^ i)"),
}


def batch_measure(name, cpu_budget=0):
    """Solves the batch three ways, each once after a warm-up on its first
    games: pg_solve_batch with the inputs already in device memory, the same
    from host arrays with results copied back (end to end), and a loop of
    pg_load_csr + pg_solve over the same games one at a time. With several
    ranks every rank takes its share of the games (largest first to the
    least loaded rank) and solves it alone; throughput is all games over the
    slowest rank's time."""
    import torch

    from paper_1705_02313_gb300 import gen, pg, shard
    ws, rank, _ = dist_env()
    count, lo, hi, dmin, dmax, desc = BATCHES[name]
    sizes_all = gen.log_uniform_sizes(count, lo, hi).astype(np.int64)
    mine = shard.shard_of(sizes_all, ws, rank) if ws > 1 else None
    t0 = time.perf_counter()
    vb, eb, off, tgt, own, pri = gen.native_batch(count, lo, hi, dmin, dmax, indices=mine)
    t_gen = time.perf_counter() - t0
    local = count if mine is None else int(mine.size)
    n0, m0 = int(vb[-1]), int(eb[-1])
    dev = [torch.from_numpy(a).cuda() for a in (off, tgt, own, pri)]
    out = dict(win=torch.empty(max(n0, 1), dtype=torch.uint8, device="cuda"),
               sigma=torch.empty(max(n0, 1), dtype=torch.int32, device="cuda"))
    ctx = pg.pg_ctx_create(torch.cuda.current_device())
    try:
        w = min(local, 16)  # warm-up: the first games
        if w:
            pg.pg_solve_batch(ctx, w, vb[:w + 1], eb[:w + 1], *dev, **out)
        torch.cuda.synchronize()
        shard.barrier()
        t0 = time.perf_counter()
        res = pg.pg_solve_batch(ctx, local, vb, eb, *dev, **out) if local else None
        torch.cuda.synchronize()
        t_batch = shard.max_over_ranks(time.perf_counter() - t0)
        win_b = out["win"].cpu().numpy()[:n0]
        sig_b = out["sigma"].cpu().numpy()[:n0]
        # end to end: host inputs, results back in host memory
        hwin = np.empty(n0, np.uint8)
        hsig = np.empty(n0, np.int32)
        shard.barrier()
        t0 = time.perf_counter()
        if local:
            pg.pg_solve_batch(ctx, local, vb, eb, off, tgt, own, pri, win=hwin, sigma=hsig)
        t_e2e = shard.max_over_ranks(time.perf_counter() - t0)
        # one game at a time through the single-game entry points
        o_off, o_tgt, o_own, o_pri = dev
        shard.barrier()
        t0 = time.perf_counter()
        inner_sum = 0
        for i in range(local):
            a, b = int(vb[i]), int(vb[i + 1])
            e0, e1 = int(eb[i]), int(eb[i + 1])
            g = pg.pg_load_csr(ctx, b - a, e1 - e0, o_off[a + i:b + i + 1], o_tgt[e0:e1], o_own[a:b], o_pri[a:b])
            try:
                _, inner = pg.pg_solve(ctx, g, win=out["win"][a:b], sigma=out["sigma"][a:b])
                inner_sum += inner
            finally:
                pg.pg_game_free(g)
        torch.cuda.synchronize()
        t_single = shard.max_over_ranks(time.perf_counter() - t0)
        same = bool(np.array_equal(win_b, out["win"].cpu().numpy()[:n0]) and
                    np.array_equal(sig_b, out["sigma"].cpu().numpy()[:n0]) and
                    np.array_equal(win_b, hwin) and np.array_equal(sig_b, hsig))
    finally:
        pg.pg_ctx_destroy(ctx)
    same = all(shard.gather_to_all(same))
    inner_sum = int(shard.sum_over_ranks(inner_sum))
    its = int(shard.max_over_ranks(res["iterations"] if res else 0))
    inner_lo = int(-shard.max_over_ranks(-(int(res["inner"].min()) if res else 10**9)))
    inner_hi = int(shard.max_over_ranks(int(res["inner"].max()) if res else 0))
    cpu = None
    if cpu_budget > 0 and rank == 0:
        c = cpu_batch(count, lo, hi, dmin, dmax, cpu_budget)
        k = c["games"]
        if mine is None:
            oracle_same = all(np.array_equal(c["win"][i], win_b[vb[i]:vb[i + 1]]) and
                              np.array_equal(c["sigma"][i], sig_b[vb[i]:vb[i + 1]]) for i in range(k))
        else:
            oracle_same = None  # the games of the sample are spread over the ranks
        cpu = {"value": k / c["seconds"], "unit": "games/s", "cores": c["cores"], "kind": "oracle",
               "sample": "games 0..%d of the batch (%d vertices), one game per process on %d processes, %.1f s wall "
                         "(%.1f s of single-thread solves); each worker generates its game before timing the solve"
                         % (k - 1, c["vertices"], c["cores"], c["seconds"], c["solve_seconds"]),
               "identical_to_gpu": oracle_same}
    return {"workload": name, "description": desc, "games": count, "vertices": int(sizes_all.sum()),
            "edges": int(shard.sum_over_ranks(m0)), "ranks": ws,
            "games_per_rank": [int(x) for x in shard.gather_to_all(local)],
            "metric": "batched games/s vs one-at-a-time", "unit": "games/s",
            "batched_games_per_s": count / t_batch, "batched_e2e_games_per_s": count / t_e2e,
            "one_at_a_time_games_per_s": count / t_single, "speedup": t_single / t_batch,
            "batched_s": t_batch, "batched_e2e_s": t_e2e, "one_at_a_time_s": t_single,
            "lockstep_iterations": its, "inner_min": inner_lo,
            "batched_split_ms": ({"load": res["load_ms"], "pack": res["pack_ms"], "loop": res["loop_ms"]}
                                 if res else None),
            "inner_max": inner_hi, "valuations_one_at_a_time": inner_sum,
            "generate_s": t_gen, "identical_results": same, "cpu_baseline": cpu,
            "timing": "wall clock around each call, device synchronised; includes loading and preprocessing; "
                      "with several ranks, the slowest rank's time"}


# ---------------------------------------------------------------------------
# serving: a Poisson stream of games through pg_server_*

SERVE = {
    "serve-200": dict(rate=200.0, lo=10_000, hi=4_000_000, dmin=2, dmax=6, pool=64,
                      desc="Poisson arrivals at 200 games/s; random games with sizes log-uniform in [1e4, 4e6], "
                           "out-degree U[2,6], owners p=0.5, permuted priorities; arrival j is game j mod 64 of a "
                           "pool generated with seeds SplitMix64(0x5EED ^ i)"),
}


def serve_measure(name, seconds, cpu_budget=0):
    """Submits arrivals of a Poisson process for ``seconds`` from one thread,
    polls results from another, then solves the pool one game at a time
    (pg_load_csr + pg_solve from host arrays) for comparison. With several
    ranks the stream shards by arrival (shard.stream_assign: each arrival to
    the rank with the least work submitted so far, decided by every rank alone);
    each rank serves its arrivals on its own GPU, and rank 0 reports all games
    over the slowest rank's time. The queue of waiting games is sampled every
    half second to show whether it stays bounded."""
    import threading

    import torch

    from paper_1705_02313_gb300 import gen, pg, shard
    ws, rank, _ = dist_env()
    cfg = SERVE[name]
    t0 = time.perf_counter()
    vb, eb, off, tgt, own, pri = gen.native_batch(cfg["pool"], cfg["lo"], cfg["hi"], cfg["dmin"], cfg["dmax"])
    t_gen = time.perf_counter() - t0
    P = cfg["pool"]
    pool = [(int(vb[i + 1] - vb[i]), int(eb[i + 1] - eb[i]), off[int(vb[i]) + i:int(vb[i + 1]) + i + 1],
             tgt[int(eb[i]):int(eb[i + 1])], own[int(vb[i]):int(vb[i + 1])], pri[int(vb[i]):int(vb[i + 1])])
            for i in range(P)]
    rng = np.random.default_rng(12345)
    gaps = rng.exponential(1.0 / cfg["rate"], size=int(cfg["rate"] * seconds * 2) + 16)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < seconds]
    owner = shard.stream_assign(np.diff(vb)[np.arange(arrivals.size) % P], ws)
    mine = np.nonzero(owner == rank)[0]
    sv = pg.pg_server_create(torch.cuda.current_device())
    done = {}
    submit_err = []
    queue_trace = []  # (seconds since start, games waiting, games submitted, games completed)
    stop = threading.Event()

    def submitter():
        start = time.perf_counter()
        try:
            for j in mine:
                d = arrivals[j] - (time.perf_counter() - start)
                if d > 0:
                    time.sleep(d)
                n, m, o, t, w, p = pool[j % P]
                pg.pg_server_submit(sv, n, m, o, t, w, p, tag=int(j))
        except Exception as e:  # reported in the result
            submit_err.append(repr(e))

    def sampler():
        while not stop.wait(0.5):
            st = pg.pg_server_get_stats(sv)
            queue_trace.append((round(time.perf_counter() - t_start, 2), int(st["queued"]), int(st["submitted"]),
                                int(st["completed"])))

    shard.barrier()
    th = threading.Thread(target=submitter)
    ts = threading.Thread(target=sampler, daemon=True)
    t_start = time.perf_counter()
    th.start()
    ts.start()
    limit = seconds + 120.0
    while len(done) < len(mine) and time.perf_counter() - t_start < limit:
        for r in pg.pg_server_poll(sv, 256, 50):
            done[r["tag"]] = (r, time.perf_counter())
            pg.pg_server_fetch(sv, r["tag"], r["n"], r["k"], keep=False)
    th.join()
    stop.set()
    t_last = max((x[1] for x in done.values()), default=time.perf_counter())
    stats = pg.pg_server_get_stats(sv)
    pg.pg_server_destroy(sv)
    lat_l = [x[0]["latency_us"] / 1e3 for x in done.values()]
    qus_l = [x[0]["queue_us"] / 1e3 for x in done.values()]
    ok_l = sum(1 for x in done.values() if x[0]["status"] == pg.PG_OK)
    # served over the second half of the window: completions per second against arrivals per second
    half = [x[1] - t_start for x in done.values() if seconds / 2 <= x[1] - t_start <= seconds]
    lat = np.concatenate([np.asarray(x, dtype=np.float64) for x in shard.gather_to_all(lat_l)])
    qus = np.concatenate([np.asarray(x, dtype=np.float64) for x in shard.gather_to_all(qus_l)])
    ok = int(shard.sum_over_ranks(ok_l))
    completed = int(shard.sum_over_ranks(len(done)))
    span = shard.max_over_ranks(t_last - t_start)
    served = completed / span if completed else 0.0
    served_2nd_half = shard.sum_over_ranks(len(half)) / (seconds / 2)
    traces = shard.gather_to_all(queue_trace)
    qmax = max((q for tr in traces for (_, q, _, _) in tr), default=0)
    q_end = sum(tr[-1][1] for tr in traces if tr)
    q_mid = sum(min(tr, key=lambda e: abs(e[0] - seconds / 2))[1] for tr in traces if tr)
    # one at a time over the pool (host arrays, as submitted), on rank 0's GPU
    t_single = None
    if rank == 0:
        ctx = pg.pg_ctx_create(torch.cuda.current_device())
        t0 = time.perf_counter()
        for (n, m, o, t, w, p) in pool:
            g = pg.pg_load_csr(ctx, n, m, o, t, w, p)
            try:
                pg.pg_solve(ctx, g, win=np.empty(n, np.uint8))
            finally:
                pg.pg_game_free(g)
        t_single = time.perf_counter() - t0
        pg.pg_ctx_destroy(ctx)
    torch.cuda.synchronize()
    cpu = None
    if cpu_budget > 0 and rank == 0:
        c = cpu_batch(P, cfg["lo"], cfg["hi"], cfg["dmin"], cfg["dmax"], cpu_budget)
        cpu = {"value": c["games"] / c["seconds"], "unit": "games/s", "cores": c["cores"], "kind": "oracle",
               "sample": "games 0..%d of the pool (%d vertices), one game per process on %d processes, %.1f s wall "
                         "(%.1f s of single-thread solves)"
                         % (c["games"] - 1, c["vertices"], c["cores"], c["seconds"], c["solve_seconds"])}
    offered = len(arrivals) / seconds
    return {"workload": name, "description": cfg["desc"], "seconds": seconds, "arrivals": int(len(arrivals)),
            "ranks": ws, "arrivals_per_rank": [int(x) for x in np.bincount(owner, minlength=ws)],
            "completed": completed, "ok": ok, "metric": "served games/s and latency", "unit": "games/s",
            "served_games_per_s": served, "offered_games_per_s": offered,
            "served_games_per_s_second_half": served_2nd_half,
            "latency_ms_p50": float(np.percentile(lat, 50)) if lat.size else None,
            "latency_ms_p99": float(np.percentile(lat, 99)) if lat.size else None,
            "queue_ms_p50": float(np.percentile(qus, 50)) if qus.size else None,
            "queue": {"waiting_max": int(qmax), "waiting_at_half": int(q_mid), "waiting_at_end": int(q_end),
                      "bounded": bool(served_2nd_half >= 0.95 * offered),
                      "trace_rank0": queue_trace[::4],
                      "note": "games submitted and not yet admitted, sampled every 0.5 s (trace: every 2 s: "
                              "seconds, waiting, submitted, completed); bounded = completions in the second half "
                              "of the window keep up with arrivals (>= 95%)"},
            "one_at_a_time_games_per_s": (P / t_single) if t_single else None, "pool_games": P,
            "pool_vertices": int(vb[-1]), "pool_edges": int(eb[-1]), "generate_s": t_gen,
            "server": stats, "submit_errors": submit_err, "cpu_baseline": cpu,
            "timing": "wall clock; latency from submission to result, measured by the server; with several ranks, "
                      "all ranks' games over the slowest rank's span"}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample

def cpu_sample(game, iters, gp=None):
    """The oracle's first ``iters`` valuations of the solve (the preprocessing
    is outside the timed part; pass ``gp`` to reuse it)."""
    from oracle import o2
    if gp is None:
        gp = o2.preprocess(game.n, game.offsets, game.targets, game.owner, game.pri)
    t0 = time.perf_counter()
    res = o2.run(gp, max_inner=iters, allow_timeout=True)
    dt = time.perf_counter() - t0
    return dict(seconds=dt, iters=res["inner"], edges=game.m)


def _oracle_batch_game(job):
    """One game of a batch solved by the oracle in a pool worker: generated
    from its seed, then preprocessed and solved (O-2, single thread)."""
    i, n, dmin, dmax = job
    from oracle import o2
    from paper_1705_02313_gb300 import gen
    g = gen.native_random_game(n, dmin, dmax, gen.batch_seed(i), nthreads=1)
    t0 = time.perf_counter()
    _, res, out = o2.solve_game(g.n, g.offsets, g.targets, g.owner, g.pri)
    return i, time.perf_counter() - t0, np.asarray(out["win"], np.uint8), np.asarray(out["sigma"], np.int32)


def cpu_batch(count, lo, hi, dmin, dmax, budget_vertices):
    """The oracle on all host cores, one game per process (spawned), over the
    first games of the batch up to ``budget_vertices`` vertices in total."""
    import multiprocessing as mp

    from paper_1705_02313_gb300 import gen
    sizes = gen.log_uniform_sizes(count, lo, hi).astype(np.int64)
    take = max(1, int(np.searchsorted(np.cumsum(sizes), budget_vertices, side="right")))
    take = min(take, count)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    jobs = [(i, int(sizes[i]), dmin, dmax) for i in range(take)]
    jobs.sort(key=lambda j: -j[1])  # largest first: less idle time at the end
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_batch_game, [(0, 1000, dmin, dmax)] * cores)  # start-up and library load
        t0 = time.perf_counter()
        res = pool.map(_oracle_batch_game, jobs, chunksize=1)
        wall = time.perf_counter() - t0
    res.sort(key=lambda r: r[0])
    return dict(games=take, vertices=int(sizes[:take].sum()), cores=cores, seconds=wall,
                solve_seconds=float(sum(r[1] for r in res)), win=[r[2] for r in res], sigma=[r[3] for r in res])


# ---------------------------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import o2
    game = make_game(args.workload)
    gp = o2.preprocess(game.n, game.offsets, game.targets, game.owner, game.pri)
    iters = args.ref_iters
    times = []
    for i in range(args.warmup + args.steps):
        r = cpu_sample(game, iters, gp)
        if i >= args.warmup:
            times.append(r["seconds"])
    tot = sum(times)
    value = game.m * iters * len(times) / tot
    sample = "first %d valuations (of a full solve) of the %s workload per step" % (iters, args.workload)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload][2], "n": game.n, "m": game.m},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    from paper_1705_02313_gb300 import build
    build.build()
    from paper_1705_02313_gb300 import pg

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    game = make_game(args.workload)
    n, m = game.n, game.m
    ctx = pg.pg_ctx_create(local)
    stream = torch.cuda.Stream(device=dev)
    pg.pg_set_stream(ctx, stream)
    d_in = [torch.from_numpy(a).to(dev) for a in game.arrays()]
    torch.cuda.synchronize()
    out = dict(win=torch.empty(n, dtype=torch.uint8, device=dev), sigma=torch.empty(n, dtype=torch.int32, device=dev),
               tau=torch.empty(n, dtype=torch.int32, device=dev), val_class=torch.empty(n, dtype=torch.int8, device=dev),
               val_depth=torch.empty(n, dtype=torch.int32, device=dev),
               val_rank=torch.empty(n, dtype=torch.int32, device=dev))

    def step(inputs, outputs, evs=None):
        """One load + solve; evs: three CUDA events recorded on the library's
        stream before the load, between load and solve, and after the solve."""
        if evs:
            evs[0].record(stream)
        g = pg.pg_load_csr(ctx, n, m, *inputs)
        if evs:
            evs[1].record(stream)
        try:
            _, _, k = pg.pg_game_info(g)
            like = outputs["win"]
            if like.is_cuda:
                ds = torch.empty(max(k, 1), dtype=torch.int8, device=like.device)
            else:
                ds = torch.empty(max(k, 1), dtype=torch.int8).pin_memory()
            major, inner = pg.pg_solve(ctx, g, dummy_sigma=ds, **outputs)
            if evs:
                evs[2].record(stream)
            stats = pg.pg_kernel_stats(g)
            return major, inner, k, stats, pg.pg_last_timing(g)
        finally:
            pg.pg_game_free(g)

    # warm-up (untimed)
    for _ in range(args.warmup):
        step(d_in, out)
    # per-kernel timing pass (untimed): device time of each kernel class
    pg.pg_set_timing(ctx, True)
    major, inner, k, kstats, tinfo = step(d_in, out)
    pg.pg_set_timing(ctx, False)

    # timed region: K steps, inputs resident in HBM, results to HBM
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    launches0 = pg.pg_launch_count(ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    t0 = time.perf_counter()
    inner_total = 0
    step_evs = []
    for _ in range(args.steps):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        _, inner_s, _, _, _ = step(d_in, out, evs)
        step_evs.append(evs)
        inner_total += inner_s
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    dev_ms = ev0.elapsed_time(ev1)
    load_ms = sum(e[0].elapsed_time(e[1]) for e in step_evs)
    solve_ms = sum(e[1].elapsed_time(e[2]) for e in step_evs)
    launches = pg.pg_launch_count(ctx) - launches0
    clk = clocks.stop()
    t_ms = max(dev_ms, 0.0)
    if ws > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_ms, float(inner_total)], device=dev, dtype=torch.float64)
        mx = tt.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = tt.clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        t_ms, inner_sum = float(mx[0]), float(sm[1])
    else:
        inner_sum = float(inner_total)
    value = m * inner_sum / (t_ms / 1000.0)

    # end to end through the C ABI with host buffers: pinned inputs, pinned outputs
    h_in = [torch.from_numpy(a).pin_memory() for a in game.arrays()]
    h_out = {kk: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for kk, v in out.items()}
    step(h_in, h_out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_inner = 0
    for _ in range(args.steps):
        _, i_s, _, _, _ = step(h_in, h_out)
        e_inner += i_s
    torch.cuda.synchronize()
    e_wall = time.perf_counter() - t0
    h2d = sum(a.nbytes for a in game.arrays())
    d2h = sum(v.numel() * v.element_size() for v in h_out.values()) + k
    e2e = {"value": m * e_inner / e_wall, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # roofline: the inner iteration against B_alg = 8 m' + 20 n' (one pass over the edges and a few per-id arrays),
    # its time taken from the timed steps (solve time, CUDA events around pg_solve, over the valuations computed)
    own = game.owner
    deg = np.diff(game.offsets).astype(np.int64)
    s = {"n": n + k, "m": m + k, "n_odd": int(own.sum()), "m_odd": int(deg[own == 1].sum()),
         "n_even": int((own == 0).sum()) + k, "m_even": int(deg[own == 0].sum()) + k}
    per = {nm: (ms, launches_k, calls) for nm, (ms, launches_k, calls) in kstats.items() if calls > 0}
    dom_name = max(per, key=lambda x: per[x][0]) if per else None
    hbm, src = peaks()
    b_alg = 8 * (m + k) + 20 * (n + k)
    iter_s = solve_ms / 1000.0 / max(inner_total, 1)
    roof = {"bound": "hbm", "kernel": "inner iteration (valuation + switching, the CUDA-graph loop of pg_solve)",
            "achieved": b_alg / iter_s / 1e9, "peak": hbm, "unit": "GB/s", "frac": b_alg / iter_s / 1e9 / hbm,
            "peak_source": src + " (hbm_gbs, burst copy)", "traffic": measured_traffic("iteration", args.workload),
            "algorithmic_bytes_per_launch": b_alg, "avg_launch_us": iter_s * 1e6,
            "units": "one inner iteration: B_alg = 8 m' + 20 n' bytes, m' = %d edges and n' = %d vertices of G' "
                     "(the Odd switching pass evaluates only the vertices some of whose successors changed their top "
                     "word, so an iteration moves less)" % (m + k, n + k),
            "timing": "solve time of the timed steps (CUDA events around pg_solve on the library's stream) / "
                      "valuations; the loads (%.2f ms per step) are outside" % (load_ms / args.steps),
            "inner_loop_edges_per_s": m / iter_s}
    dominant = None
    if dom_name:
        ms, _, calls = per[dom_name]
        avg_s = ms / calls / 1000.0
        ab = algorithmic_bytes(dom_name, s)
        ach = ab / avg_s / 1e9 if ab else None
        dominant = {"kernel": dom_name, "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": (ach / hbm if ach else None), "traffic": measured_traffic(dom_name, args.workload),
                    "algorithmic_bytes_per_launch": ab, "avg_launch_us": avg_s * 1e6,
                    "timing": "host-driven timing pass (per-kernel CUDA events)"}
    valuation_path = None
    if tinfo["valuations"]:
        per_iter_s = (tinfo["valuation_ms"] + tinfo["switch_ms"]) / tinfo["valuations"] / 1000.0
        valuation_path = {"inner_iteration_us": per_iter_s * 1e6, "b_alg_bytes": b_alg,
                          "achieved_gbs": b_alg / per_iter_s / 1e9, "frac_of_hbm": b_alg / per_iter_s / 1e9 / hbm,
                          "inner_loop_edges_per_s": m / per_iter_s,
                          "timing": "host-driven timing pass (one launch per kernel, events around each class)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload][2], "n": n, "m": m,
                   "dummies": k, "valuations_per_solve": inner, "major_iterations": major,
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (CSR %.0f MB; no flush)" % (h2d / 1e6)},
        "full_solve_ms": t_ms / args.steps,
        "wall_s": wall,
        "roofline": roof,
        "dominant_kernel": dominant,
        "inner_iteration_host_loop": valuation_path,
        "load_ms": load_ms / args.steps,
        "kernels": {nm: kernel_entry(nm, v, s, hbm) for nm, v in kstats.items() if v[1]},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if rank == 0:  # ablation of Section 6 (Table 2): best responses restarted from the initial Odd strategy
        g = pg.pg_load_csr(ctx, n, m, *d_in)
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r_major, r_inner = pg.pg_solve(ctx, g, win=out["win"], reset_tau=True)
            torch.cuda.synchronize()
            r_ms = (time.perf_counter() - t0) * 1e3
        finally:
            pg.pg_game_free(g)
        line["si_reset"] = {"major_iterations": r_major, "valuations": r_inner, "solve_ms": r_ms,
                            "valuations_plain": inner, "major_plain": major,
                            "note": "SI-Reset: every best response restarts from the first edge of each Odd list"}
    if rank == 0 and args.cv_workload:
        line["count_vector"] = cv_measure(args.cv_workload, ctx)
    if rank == 0 and args.chain > 0:
        line["long_chain"] = chain_measure(args.chain, ctx)
    if not args.no_batch:  # every rank solves its share of the batch's games
        b = batch_measure(args.batch, 0 if args.no_cpu_baseline else args.batch_cpu_vertices)
        if rank == 0:
            line["batch"] = b
    if args.serve > 0:  # every rank serves its share of the stream
        sres = serve_measure("serve-200", args.serve, 0 if args.no_cpu_baseline else args.serve_cpu_vertices)
        if rank == 0:
            line["serve"] = sres
    if rank == 0 and not args.no_cpu_baseline:
        r = cpu_sample(game, args.cpu_iters)
        line["cpu_baseline"] = {"value": r["edges"] * r["iters"] / r["seconds"], "unit": UNIT, "cores": 1,
                                "kind": "oracle",
                                "sample": "first %d valuations of the same solve (%.1f s single-threaded)" %
                                          (r["iters"], r["seconds"])}
    if rank == 0:
        print(json.dumps(line), flush=True)
    pg.pg_ctx_destroy(ctx)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_profile_solves(args):
    """Only W warm-up solves plus ``--profile-solves`` solves of the workload
    (no timing region, no baselines): the command that profiler captures run."""
    import torch

    from paper_1705_02313_gb300 import build
    build.build()
    from paper_1705_02313_gb300 import pg
    game = make_game(args.workload)
    n, m = game.n, game.m
    ctx = pg.pg_ctx_create(0)
    pg.pg_set_timing(ctx, True)
    d_in = [torch.from_numpy(a).cuda() for a in game.arrays()]
    out = dict(win=torch.empty(n, dtype=torch.uint8, device="cuda"))
    res = []
    for i in range(args.profile_solves):
        g = pg.pg_load_csr(ctx, n, m, *d_in)
        try:
            major, inner = pg.pg_solve(ctx, g, **out)
            res.append({"major": major, "inner": inner, "kernels_ms": {k: round(v[0], 3) for k, v in
                                                                       pg.pg_kernel_stats(g).items() if v[1]}})
        finally:
            pg.pg_game_free(g)
    print(json.dumps({"workload": args.workload, "solves": res}), flush=True)
    pg.pg_ctx_destroy(ctx)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile-solves", type=int, default=0,
                    help="run only this many solves (for profiler captures) and exit")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="random-10m")
    ap.add_argument("--cpu-iters", type=int, default=3)
    ap.add_argument("--batch-cpu-vertices", type=int, default=6_000_000,
                    help="vertices of the batch's first games that the all-cores oracle baseline solves")
    ap.add_argument("--serve-cpu-vertices", type=int, default=4_000_000,
                    help="vertices of the serving pool's first games that the all-cores oracle baseline solves")
    ap.add_argument("--ref-iters", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-one-at-a-time measurement")
    ap.add_argument("--chain", type=int, default=0,
                    help="also time pg_valuate on one successor chain of this many vertices (0: skip)")
    ap.add_argument("--cv-workload", default="random-10m-4pri",
                    help="count-vector workload measured beside the main line ('' to skip)")
    ap.add_argument("--serve", type=float, default=60.0,
                    help="seconds of the Poisson serving stream measured beside the main line (0: skip)")
    ap.add_argument("--batch", choices=sorted(BATCHES), default="batch-4096",
                    help="batch workload measured beside the main line")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.profile_solves:
        return run_profile_solves(args)
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
