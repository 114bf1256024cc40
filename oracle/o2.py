"""ctypes wrapper of the scalable C oracle (O-2, ``o2.c``).

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
baseline may use it; the product path never does.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

FIN, TOP, ODDCYCLE = 0, 1, 2
INT32_MAX = 2**31 - 1
OK, EINVAL, ENOMEM, ETIMEOUT, ENOTADMISSIBLE, ECHECK = 0, 1, 2, 3, 4, 5

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        P = C.c_void_p
        _lib.o2_preprocess.argtypes = [C.c_int32, P, P, P, P, P, P, P, P, P, P, P, C.c_int]
        _lib.o2_run.argtypes = [C.c_int32, P, P, P, P, P, C.c_int, C.c_int64, C.c_int,
                                P, P, P, P, P, P, P, P, C.c_int64]
        _lib.o2_valuate_profile.argtypes = [C.c_int32, P, P, P, P, P, P, P]
        _lib.o2_compare.argtypes = [C.c_int32, P, P, P, C.c_int32, C.c_int32]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed with status %d" % (what, code))
        self.code = code


def preprocess(n, off, tgt, own, pri, dummy_zero=None):
    """P0 of Section 3 (see ``o2_preprocess``). Returns a dict of numpy
    arrays for G' plus ``dummy_of``, ``k`` and ``inU``. dummy_zero (default:
    when priorities repeat) gives every dummy priority 0 and shifts original
    priorities by 2, instead of priorities 2j and a shift of 2k."""
    off = np.ascontiguousarray(off, dtype=np.int32)
    tgt = np.ascontiguousarray(tgt, dtype=np.int32)
    own = np.ascontiguousarray(own, dtype=np.uint8)
    pri = np.ascontiguousarray(pri, dtype=np.int32)
    m = int(off[n])
    o_off = np.zeros(2 * n + 1, np.int32)
    o_tgt = np.zeros(m + n, np.int32)
    o_own = np.zeros(2 * n, np.uint8)
    o_pri = np.zeros(2 * n, np.int32)
    dummy = np.zeros(max(n, 1), np.int32)
    inU = np.zeros(max(n, 1), np.uint8)
    k = C.c_int32(0)
    if dummy_zero is None:
        dummy_zero = np.unique(pri).size < n
    rc = lib().o2_preprocess(n, _p(off), _p(tgt), _p(own), _p(pri), _p(o_off), _p(o_tgt), _p(o_own),
                             _p(o_pri), _p(dummy), C.byref(k), _p(inU), 1 if dummy_zero else 0)
    if rc:
        raise OracleError(rc, "o2_preprocess")
    k = k.value
    np_ = n + k
    mp = int(o_off[np_])
    return dict(n=np_, n_orig=n, k=k, off=o_off[: np_ + 1].copy(), tgt=o_tgt[:mp].copy(),
                own=o_own[:np_].copy(), pri=o_pri[:np_].copy(), dummy_of=dummy[:k].copy(), inU=inU[:n].copy(),
                dummy_zero=bool(dummy_zero))


def initial_profile(gp):
    """sigma_init (Even -> sink, id n') and tau = first edge of each list."""
    n = gp["n"]
    strat = np.where(gp["own"] == 0, n, gp["tgt"][np.minimum(gp["off"][:-1], max(len(gp["tgt"]) - 1, 0))])
    return strat.astype(np.int32)


def run(gp, strat=None, mode="solve", max_inner=10**9, check=False, stats_cap=0, allow_timeout=False):
    """Algorithm 1 (Section 4) on the preprocessed game. mode: "solve",
    "best_response" (inner loop only) or "solve_reset" (every best response
    starts again from the initial Odd strategy: SI-Reset, Section 6). Raises
    OracleError for any non-OK status (except the iteration cap when
    ``allow_timeout``); ``res['status']`` holds the status."""
    n = gp["n"]
    strat = initial_profile(gp) if strat is None else np.array(strat, dtype=np.int32, copy=True)
    cls = np.zeros(n, np.int8)
    depth = np.zeros(n, np.int32)
    rank = np.zeros(n, np.int32)
    dom = np.zeros(n, np.int32)
    sink_rank = C.c_int32(0)
    major = C.c_int64(0)
    inner = C.c_int64(0)
    stats = np.zeros(4 * max(stats_cap, 1), np.int64)
    rc = lib().o2_run(n, _p(gp["off"]), _p(gp["tgt"]), _p(gp["own"]), _p(gp["pri"]), _p(strat),
                      {"solve": 0, "best_response": 1, "solve_reset": 2}[mode], int(max_inner), 1 if check else 0,
                      _p(cls), _p(depth), _p(rank), _p(dom), C.byref(sink_rank), C.byref(major), C.byref(inner),
                      _p(stats) if stats_cap else None, int(stats_cap))
    if rc and not (allow_timeout and rc == ETIMEOUT):
        raise OracleError(rc, "o2_run")
    res = dict(status=rc, strat=strat, cls=cls, depth=depth, rank=rank, dom=dom, sink_rank=sink_rank.value,
               major=major.value, inner=inner.value)
    if stats_cap:
        res["stats"] = stats[: 4 * min(inner.value, stats_cap)].reshape(-1, 4)
    return res


def valuate(gp, strat):
    """Valuation of one profile (Section 3), no switching."""
    n = gp["n"]
    strat = np.ascontiguousarray(strat, dtype=np.int32)
    cls = np.zeros(n, np.int8)
    depth = np.zeros(n, np.int32)
    rank = np.zeros(n, np.int32)
    dom = np.zeros(n, np.int32)
    sink_rank = C.c_int32(0)
    rc = lib().o2_valuate_profile(n, _p(gp["pri"]), _p(strat), _p(cls), _p(depth), _p(rank), _p(dom),
                                  C.byref(sink_rank))
    if rc:
        raise OracleError(rc, "o2_valuate_profile")
    return dict(strat=strat, cls=cls, depth=depth, rank=rank, dom=dom, sink_rank=sink_rank.value)


def compare(gp, strat, depth, u, w):
    """Literal comparison of two finite valuations by walking both plays."""
    return lib().o2_compare(gp["n"], _p(gp["pri"]), _p(np.ascontiguousarray(strat, np.int32)),
                            _p(np.ascontiguousarray(depth, np.int32)), int(u), int(w))


def map_back(gp, res):
    """Results in original vertex ids (see the C ABI's result arrays)."""
    n0, n = gp["n_orig"], gp["n"]
    own = gp["own"][:n0]
    s = res["strat"][:n0].astype(np.int64)
    top = res["cls"][:n0] != FIN
    win = np.where(top, 0, 1).astype(np.uint8)
    sigma = np.where(own == 0, np.where(s == n, -1, s), -1).astype(np.int32)
    tau_raw = np.where(s >= n0, gp["dummy_of"][np.clip(s - n0, 0, max(gp["k"] - 1, 0))] if gp["k"] else s, s)
    tau = np.where(own == 1, tau_raw, -1).astype(np.int32)
    return dict(win=win, sigma=sigma, tau=tau, val_class=top.astype(np.int8),
                val_depth=res["depth"][:n0].copy(), val_rank=res["rank"][:n0].copy())


def solve_game(n, off, tgt, own, pri, check=False, reset=False):
    """Preprocess and solve; reset=True runs the SI-Reset variant (Section 6)."""
    gp = preprocess(n, off, tgt, own, pri)
    res = run(gp, check=check, mode="solve_reset" if reset else "solve")
    out = map_back(gp, res)
    out.update(major=res["major"], inner=res["inner"])
    return gp, res, out
