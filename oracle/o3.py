"""ctypes wrapper of the count-vector C oracle (O-3, ``o3.c``): Algorithm 1
with valuations as count vectors (Section 3), for games whose priorities may
repeat.

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
baseline may use it; the product path never does.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import o2
from .o2 import OracleError, _p

FIN, TOP, ODDCYCLE = 0, 1, 2
OK, EINVAL, ENOMEM, ETIMEOUT, ENOTADMISSIBLE = 0, 1, 2, 3, 4


def lib():
    L = o2.lib()
    if not getattr(L, "_o3_ready", False):
        P = C.c_void_p
        L.o3_run.argtypes = [C.c_int32, P, P, P, P, P, C.c_int, C.c_int64, P, P, P, P, P, P, P, P]
        L.o3_valuate_profile.argtypes = [C.c_int32, P, P, P, P, P, P, P, P, P, P, P]
        L._o3_ready = True
    return L


def levels(pri):
    """The distinct priorities in ascending order."""
    return np.unique(np.asarray(pri, dtype=np.int32))


def run(gp, strat=None, mode="solve", max_inner=10**9, allow_timeout=False):
    """Algorithm 1 on the preprocessed game ``gp`` (from o2.preprocess or
    o1.preprocess). mode: "solve", "best_response" or "solve_reset"."""
    n = gp["n"]
    off = np.ascontiguousarray(gp["off"], np.int32)
    tgt = np.ascontiguousarray(gp["tgt"], np.int32)
    own = np.ascontiguousarray(gp["own"], np.uint8)
    pri = np.ascontiguousarray(gp["pri"], np.int32)
    strat = o2.initial_profile(dict(gp, off=off, tgt=tgt, own=own)) if strat is None else \
        np.array(strat, dtype=np.int32, copy=True)
    d_max = levels(pri).size
    cls = np.zeros(n, np.int8)
    depth = np.zeros(n, np.int32)
    dom = np.zeros(n, np.int32)
    cnt = np.zeros(max(n * d_max, 1), np.int32)
    lp = np.zeros(max(d_max, 1), np.int32)
    d = C.c_int32(0)
    major, inner = C.c_int64(0), C.c_int64(0)
    rc = lib().o3_run(n, _p(off), _p(tgt), _p(own), _p(pri), _p(strat),
                      {"solve": 0, "best_response": 1, "solve_reset": 2}[mode], int(max_inner), _p(cls), _p(depth),
                      _p(dom), _p(cnt), _p(lp), C.byref(d), C.byref(major), C.byref(inner))
    if rc and not (allow_timeout and rc == ETIMEOUT):
        raise OracleError(rc, "o3_run")
    counts = cnt[: n * d.value].reshape(n, d.value).copy()
    counts[cls != FIN] = 0
    return dict(status=rc, strat=strat, cls=cls, depth=depth, dom=dom, counts=counts, level_pri=lp[: d.value].copy(),
                major=major.value, inner=inner.value)


def valuate(gp, strat):
    """Valuation of one profile (Section 3), no switching."""
    n = gp["n"]
    off = np.ascontiguousarray(gp["off"], np.int32)
    tgt = np.ascontiguousarray(gp["tgt"], np.int32)
    own = np.ascontiguousarray(gp["own"], np.uint8)
    pri = np.ascontiguousarray(gp["pri"], np.int32)
    strat = np.ascontiguousarray(strat, np.int32)
    d_max = levels(pri).size
    cls = np.zeros(n, np.int8)
    depth = np.zeros(n, np.int32)
    dom = np.zeros(n, np.int32)
    cnt = np.zeros(max(n * d_max, 1), np.int32)
    lp = np.zeros(max(d_max, 1), np.int32)
    d = C.c_int32(0)
    rc = lib().o3_valuate_profile(n, _p(off), _p(tgt), _p(own), _p(pri), _p(strat), _p(cls), _p(depth), _p(dom),
                                  _p(cnt), _p(lp), C.byref(d))
    if rc not in (OK, ENOTADMISSIBLE):
        raise OracleError(rc, "o3_valuate_profile")
    counts = cnt[: n * d.value].reshape(n, d.value).copy()
    counts[cls != FIN] = 0
    return dict(status=rc, cls=cls, depth=depth, dom=dom, counts=counts, level_pri=lp[: d.value].copy())


def map_back(gp, res):
    """Results in original vertex ids (as o2.map_back) plus the count vector
    of every original vertex (rows) over the levels of G' (columns)."""
    n0 = gp["n_orig"]
    out = o2.map_back(gp, dict(res, rank=np.zeros(gp["n"], np.int32)))
    out.pop("val_rank", None)
    out["val_counts"] = res["counts"][:n0]
    out["level_pri"] = res["level_pri"]
    return out


def solve_game(n, off, tgt, own, pri, reset=False):
    """Preprocess (dummies at priority 0 when priorities repeat) and solve."""
    gp = o2.preprocess(n, off, tgt, own, pri)
    res = run(gp, mode="solve_reset" if reset else "solve")
    out = map_back(gp, res)
    out.update(major=res["major"], inner=res["inner"])
    return gp, res, out
