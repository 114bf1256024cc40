"""Writes tests/golden/full_size_digests.json: the CPU oracle's full solve of
the two 10,000,000-vertex workloads, as SHA-256 digests of every output array
plus a few sampled values, so that the GPU parity test can compare the CUDA
path's final results with the oracle's element for element without running
the oracle for minutes on the GPU machine.

Calls only the oracle (oracle/o2) and the seeded input generators; nothing
here touches the CUDA path. Run it again whenever the generators or the
oracle's arithmetic change:

    python tests/golden/make_full_size_digests.py

It takes about ten minutes (the two solves run in two processes).

Workloads (the benchmark's):
  random-10m  random game, n = 10,000,000, out-degree U[2,5], owners p = 0.5,
              permuted priorities, seed 0 (native generator)
  ladder-10m  ladder game, n = 10,000,000 (i -> i+1 plus one back edge to
              j < i), owners p = 0.5, permuted priorities, seed 0
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "full_size_digests.json")
KEYS = ("win", "sigma", "tau", "val_class", "val_depth", "val_rank", "dummy_sigma")
SAMPLES = 64


def make_game(name):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from paper_1705_02313_gb300 import gen
    if name == "random-10m":
        return gen.native_random_game(10_000_000, 2, 5, 0)
    if name == "ladder-10m":
        return gen.ladder_game(10_000_000, 0)
    raise ValueError(name)


def digest(a):
    a = np.ascontiguousarray(a)
    return hashlib.sha256(a.tobytes()).hexdigest()


def input_digest(g):
    h = hashlib.sha256()
    for a in g.arrays():
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def sample_indices(size, seed=1705):
    rng = np.random.default_rng(seed)
    return np.unique(rng.integers(0, max(size, 1), SAMPLES)) if size else np.zeros(0, np.int64)


def oracle_outputs(gp, res):
    """Output arrays in original ids, as the C ABI reports them."""
    from oracle import o2
    out = o2.map_back(gp, res)
    n0, n = gp["n_orig"], gp["n"]
    out["dummy_sigma"] = (res["strat"][n0:n] != n).astype(np.int8)
    return out


def solve(name):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import o2
    t0 = time.time()
    g = make_game(name)
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    res = o2.run(gp)
    out = oracle_outputs(gp, res)
    rec = {"input_sha256": input_digest(g), "n": g.n, "m": g.m, "k": int(gp["k"]),
           "major": int(res["major"]), "inner": int(res["inner"]), "arrays": {}}
    for key in KEYS:
        a = np.asarray(out[key])
        idx = sample_indices(a.size)
        rec["arrays"][key] = {"dtype": str(a.dtype), "size": int(a.size), "sha256": digest(a),
                              "sample_index": idx.tolist(), "sample_value": a[idx].astype(np.int64).tolist()}
    rec["oracle_seconds"] = round(time.time() - t0, 1)
    return name, rec


def main():
    names = ["random-10m", "ladder-10m"]
    with mp.get_context("spawn").Pool(len(names)) as pool:
        results = dict(pool.map(solve, names))
    doc = {"what": "the CPU oracle's (oracle/o2) full solves of the benchmark's 10M-vertex workloads: digests of "
                   "the outputs in original vertex ids (win, sigma, tau, val_class, val_depth, val_rank, "
                   "dummy_sigma) and sampled values; written by tests/golden/make_full_size_digests.py",
           "workloads": results}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
