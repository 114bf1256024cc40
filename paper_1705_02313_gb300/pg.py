"""Python binding of libpg (include/pg.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does
nothing but convert arguments: arrays may be numpy arrays or torch tensors
(CPU tensors and numpy arrays are passed as host memory, CUDA tensors as
device memory). All computation happens in the CUDA library; if libpg.so is
missing or fails to load, every call raises ``PgUnavailable``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# PG_LIBPG may name another build of the same library (for example a debug build)
LIB_PATH = os.environ.get("PG_LIBPG") or os.path.join(HERE, "libpg.so")

PG_OK, PG_EINVAL, PG_ENOMEM, PG_ETIMEOUT, PG_ENOTADMISSIBLE, PG_ECUDA, PG_EUNSUPPORTED = range(7)
PG_MEM_HOST, PG_MEM_DEVICE = 0, 1
STATUS_NAMES = {0: "PG_OK", 1: "PG_EINVAL", 2: "PG_ENOMEM", 3: "PG_ETIMEOUT", 4: "PG_ENOTADMISSIBLE",
                5: "PG_ECUDA", 6: "PG_EUNSUPPORTED"}
INT32_MAX = 2**31 - 1


class PgUnavailable(RuntimeError):
    pass


class PgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, str(code)), msg))
        self.code = code


class pg_result(C.Structure):
    _fields_ = [("win", C.c_void_p), ("sigma", C.c_void_p), ("tau", C.c_void_p), ("val_class", C.c_void_p),
                ("val_depth", C.c_void_p), ("val_rank", C.c_void_p), ("dummy_sigma", C.c_void_p),
                ("mem_kind", C.c_int32), ("major", C.c_int64), ("inner", C.c_int64), ("val_counts", C.c_void_p)]


class pg_solve_opts(C.Structure):
    _fields_ = [("sigma_init", C.c_void_p), ("tau_init", C.c_void_p), ("dummy_sigma_init", C.c_void_p),
                ("mem_kind", C.c_int32), ("max_inner", C.c_int64), ("reset_tau", C.c_int32)]


class pg_valuation(C.Structure):
    _fields_ = [("val_class", C.c_void_p), ("val_depth", C.c_void_p), ("val_rank", C.c_void_p),
                ("dom", C.c_void_p), ("mem_kind", C.c_int32), ("val_counts", C.c_void_p)]


class pg_result_batch(C.Structure):
    _fields_ = [("win", C.c_void_p), ("sigma", C.c_void_p), ("tau", C.c_void_p), ("val_class", C.c_void_p),
                ("val_depth", C.c_void_p), ("val_rank", C.c_void_p), ("dummy_sigma", C.c_void_p),
                ("mem_kind", C.c_int32), ("major", C.c_void_p), ("inner", C.c_void_p), ("status", C.c_void_p),
                ("dummy_base", C.c_void_p), ("iterations", C.c_int64), ("load_ms", C.c_double),
                ("pack_ms", C.c_double), ("loop_ms", C.c_double)]


class pg_server_opts(C.Structure):
    _fields_ = [("max_vertices", C.c_int64), ("max_edges", C.c_int64), ("max_games", C.c_int32),
                ("round_iters", C.c_int32), ("max_inner", C.c_int64), ("wide_offsets", C.c_int32)]


TUNING_FIELDS = ("deep_cut", "ruler_bits", "walk_cap", "switch_block", "loop_ranks")


class pg_tuning(C.Structure):
    _fields_ = [(f, C.c_int32) for f in TUNING_FIELDS]


class pg_tuning_entry(C.Structure):
    _fields_ = [("max_ids", C.c_int64), ("t", pg_tuning)]


class pg_served(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("status", C.c_int32), ("n", C.c_int32), ("k", C.c_int32),
                ("major", C.c_int64), ("inner", C.c_int64), ("queue_us", C.c_double), ("latency_us", C.c_double)]


class pg_server_stats(C.Structure):
    _fields_ = [(nm, C.c_int64) for nm in ["submitted", "admitted", "completed", "queued", "admitted_while_busy",
                                           "rounds", "iterations", "max_resident", "capacity_vertices",
                                           "capacity_edges"]] + \
               [(nm, C.c_double) for nm in ["loop_ms", "repack_ms", "collect_ms"]]


class pg_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("ms", C.c_double), ("launches", C.c_int64), ("calls", C.c_int64)]


_lib = None


def lib():
    """The loaded libpg.so (built by paper_1705_02313_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise PgUnavailable("libpg.so is not built: run __graft_entry__.build() or python -m "
                            "paper_1705_02313_gb300.build")
    try:
        L = C.CDLL(LIB_PATH)
    except OSError as e:
        raise PgUnavailable("libpg.so failed to load: %s" % e)
    P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
    L.pg_ctx_create.argtypes = [C.POINTER(P), C.c_int]
    L.pg_ctx_destroy.argtypes = [P]
    L.pg_ctx_destroy.restype = None
    L.pg_set_stream.argtypes = [P, P]
    L.pg_last_error.argtypes = [P]
    L.pg_last_error.restype = C.c_char_p
    L.pg_load_csr.argtypes = [P, I32, I64, P, P, P, P, I32, C.POINTER(P)]
    L.pg_game_free.argtypes = [P]
    L.pg_game_free.restype = None
    L.pg_game_info.argtypes = [P, C.POINTER(I32), C.POINTER(I64), C.POINTER(I32)]
    L.pg_game_dummies.argtypes = [P, P]
    L.pg_game_levels.argtypes = [P, C.POINTER(I32), P]
    L.pg_game_counters.argtypes = [P, C.POINTER(pg_counters)]
    L.pg_best_response_bf.argtypes = [P, P, P, P, I32, C.POINTER(pg_valuation), C.POINTER(I64)]
    L.pg_solve.argtypes = [P, C.POINTER(pg_solve_opts), C.POINTER(pg_result)]
    L.pg_best_response.argtypes = [P, P, P, P, I32, C.POINTER(pg_valuation), C.POINTER(I64)]
    L.pg_valuate.argtypes = [P, P, P, P, I32, C.POINTER(pg_valuation)]
    L.pg_set_timing.argtypes = [P, I32]
    L.pg_set_graphs.argtypes = [P, I32]
    L.pg_set_loop_ranks.argtypes = [P, I32]
    L.pg_set_wide_offsets.argtypes = [P, I32]
    L.pg_set_tuning.argtypes = [P, C.POINTER(pg_tuning)]
    L.pg_get_tuning.argtypes = [P, C.POINTER(pg_tuning)]
    L.pg_set_tuning_table.argtypes = [P, C.POINTER(pg_tuning_entry), I32]
    L.pg_load_tuning.argtypes = [P, C.c_char_p]
    L.pg_device_name.argtypes = [C.c_int, C.c_char_p, I32]
    L.pg_release_cached_memory.argtypes = [C.c_int]
    L.pg_last_loop.argtypes = [P, C.POINTER(I32), C.POINTER(I64)]
    L.pg_last_timing.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                 C.POINTER(I64)]
    L.pg_valuate_static.argtypes = [I32, P, P, P, P, P, P]
    L.pg_solve_batch.argtypes = [P, I32, P, P, P, P, P, P, I32, I64, C.POINTER(pg_result_batch)]
    L.pg_server_create.argtypes = [C.c_int, C.POINTER(pg_server_opts), C.POINTER(P)]
    L.pg_server_destroy.argtypes = [P]
    L.pg_server_destroy.restype = None
    L.pg_server_submit.argtypes = [P, I32, I64, P, P, P, P, C.c_uint64]
    L.pg_server_poll.argtypes = [P, C.POINTER(pg_served), I32, I32, C.POINTER(I32)]
    L.pg_server_fetch.argtypes = [P, C.c_uint64, P, P, P, P, P, P, P]
    L.pg_server_get_stats.argtypes = [P, C.POINTER(pg_server_stats)]
    L.pg_server_error.argtypes = [P]
    L.pg_server_error.restype = C.c_char_p
    L.pg_kernel_stats.argtypes = [P, C.POINTER(pg_kernel_stat), I32, C.POINTER(I32)]
    L.pg_reset_stats.argtypes = [P]
    L.pg_launch_count.argtypes = [P, C.POINTER(I64)]
    for name in ["pg_solve_batch", "pg_valuate_static", "pg_kernel_stats", "pg_reset_stats", "pg_launch_count", "pg_ctx_create", "pg_set_stream", "pg_load_csr", "pg_game_info", "pg_game_dummies", "pg_solve",
                 "pg_best_response", "pg_valuate", "pg_set_timing", "pg_last_timing", "pg_set_graphs", "pg_set_loop_ranks", "pg_set_wide_offsets", "pg_set_tuning", "pg_get_tuning", "pg_set_tuning_table", "pg_load_tuning", "pg_device_name", "pg_last_loop", "pg_release_cached_memory", "pg_server_create", "pg_server_submit", "pg_server_poll",
                 "pg_server_fetch", "pg_server_get_stats", "pg_game_levels", "pg_game_counters", "pg_best_response_bf"]:
        getattr(L, name).restype = I32
    _lib = L
    return L


# ---------------------------------------------------------------------------
# marshalling helpers

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr_kind(x):
    """(pointer, mem_kind) of an array; None gives (None, None)."""
    if x is None:
        return None, None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), (PG_MEM_DEVICE if x.is_cuda else PG_MEM_HOST)
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, PG_MEM_HOST
    raise TypeError("expected a numpy array or a torch tensor, got %r" % type(x))


def _same_kind(*arrays):
    kinds = {k for _, k in (_ptr_kind(a) for a in arrays if a is not None)}
    if len(kinds) > 1:
        raise ValueError("arrays mix host and device memory")
    return kinds.pop() if kinds else PG_MEM_HOST


def _check(ctx, rc, what):
    if rc != PG_OK:
        msg = lib().pg_last_error(ctx).decode(errors="replace") if ctx else what
        raise PgError(rc, msg)


def _dtype_check(x, np_dtype, name):
    if x is None:
        return
    if _is_torch(x):
        import torch
        want = {np.int32: torch.int32, np.uint8: torch.uint8, np.int8: torch.int8, np.int64: torch.int64}[np_dtype]
        if x.dtype != want:
            raise TypeError("%s must be %s" % (name, want))
    elif x.dtype != np_dtype:
        raise TypeError("%s must be %s" % (name, np.dtype(np_dtype)))


# ---------------------------------------------------------------------------
# entry points (same names as include/pg.h)

def pg_device_name(device=0):
    buf = C.create_string_buffer(256)
    rc = lib().pg_device_name(int(device), buf, 256)
    if rc != PG_OK:
        raise PgError(rc, "pg_device_name")
    return buf.value.decode(errors="replace")


def pg_ctx_create(device=0, tuning=True):
    """A context on ``device``. With tuning (and no PG_TUNING_FILE, which the
    library itself loads) the autotuner's table for this device model is
    loaded when the package holds one (tuning/<device>.txt, see tune.py)."""
    h = C.c_void_p()
    rc = lib().pg_ctx_create(C.byref(h), device)
    if rc != PG_OK:
        raise PgError(rc, "pg_ctx_create(%d) failed" % device)
    if tuning and not os.environ.get("PG_TUNING_FILE"):
        from . import tune
        path = tune.default_table_path(pg_device_name(device))
        if os.path.exists(path):
            pg_load_tuning(h, path)
    elif not tuning:
        pg_set_tuning_table(h, [])
    return h


def pg_ctx_destroy(ctx):
    lib().pg_ctx_destroy(ctx)


def pg_set_stream(ctx, stream):
    """stream: a torch.cuda.Stream, a raw cudaStream_t handle (int), or None."""
    handle = getattr(stream, "cuda_stream", stream)
    _check(ctx, lib().pg_set_stream(ctx, C.c_void_p(handle or None)), "pg_set_stream")


def pg_last_error(ctx):
    return lib().pg_last_error(ctx).decode(errors="replace")


def pg_load_csr(ctx, n, m, offsets, targets, owner, pri):
    for a, dt, nm in [(offsets, np.int32, "offsets"), (targets, np.int32, "targets"), (owner, np.uint8, "owner"),
                      (pri, np.int32, "pri")]:
        _dtype_check(a, dt, nm)
    kind = _same_kind(offsets, targets, owner, pri)
    g = C.c_void_p()
    rc = lib().pg_load_csr(ctx, int(n), int(m), _ptr_kind(offsets)[0], _ptr_kind(targets)[0], _ptr_kind(owner)[0],
                           _ptr_kind(pri)[0], kind, C.byref(g))
    _check(ctx, rc, "pg_load_csr")
    return g


def pg_game_free(game):
    lib().pg_game_free(game)


def pg_game_info(game):
    n, m, k = C.c_int32(), C.c_int64(), C.c_int32()
    rc = lib().pg_game_info(game, C.byref(n), C.byref(m), C.byref(k))
    if rc != PG_OK:
        raise PgError(rc, "pg_game_info")
    return n.value, m.value, k.value


class pg_counters(C.Structure):
    _fields_ = [(nm, C.c_int32) for nm in ["n_pending", "jump_rounds", "n_fin", "n_odd", "n_big", "n_huge",
                                           "n_switch", "deep", "n_rulers", "deep_rounds", "rs_rounds"]]


def pg_game_counters(game):
    """Counters of the last valuation on game (dict)."""
    c = pg_counters()
    rc = lib().pg_game_counters(game, C.byref(c))
    if rc != PG_OK:
        raise PgError(rc, "pg_game_counters")
    return {f: getattr(c, f) for f, _ in pg_counters._fields_}


def pg_game_levels(game):
    """Count-vector mode: the distinct priorities of G' in ascending order
    (an empty array for a game with distinct priorities)."""
    d = C.c_int32(0)
    lp = np.zeros(8, np.int32)
    rc = lib().pg_game_levels(game, C.byref(d), lp.ctypes.data)
    if rc != PG_OK:
        raise PgError(rc, "pg_game_levels")
    return lp[: d.value].copy()


def pg_game_dummies(game):
    n, m, k = pg_game_info(game)
    out = np.zeros(max(k, 1), np.int32)
    rc = lib().pg_game_dummies(game, out.ctypes.data)
    if rc != PG_OK:
        raise PgError(rc, "pg_game_dummies")
    return out[:k]


def pg_solve(ctx, game, win=None, sigma=None, tau=None, val_class=None, val_depth=None, val_rank=None,
             dummy_sigma=None, sigma_init=None, tau_init=None, dummy_sigma_init=None, max_inner=0, reset_tau=False,
             val_counts=None):
    """Fills the given output arrays (all in host memory or all in device
    memory); returns (major, inner). val_counts (n x d int32) is filled in
    count-vector mode (games whose priorities repeat)."""
    _dtype_check(win, np.uint8, "win")
    for a, nm in [(sigma, "sigma"), (tau, "tau"), (val_depth, "val_depth"), (val_rank, "val_rank"),
                  (val_counts, "val_counts")]:
        _dtype_check(a, np.int32, nm)
    _dtype_check(val_class, np.int8, "val_class")
    _dtype_check(dummy_sigma, np.int8, "dummy_sigma")
    res = pg_result(_ptr_kind(win)[0], _ptr_kind(sigma)[0], _ptr_kind(tau)[0], _ptr_kind(val_class)[0],
                    _ptr_kind(val_depth)[0], _ptr_kind(val_rank)[0], _ptr_kind(dummy_sigma)[0],
                    _same_kind(win, sigma, tau, val_class, val_depth, val_rank, dummy_sigma, val_counts), 0, 0,
                    _ptr_kind(val_counts)[0])
    opts = pg_solve_opts(_ptr_kind(sigma_init)[0], _ptr_kind(tau_init)[0], _ptr_kind(dummy_sigma_init)[0],
                         _same_kind(sigma_init, tau_init, dummy_sigma_init), int(max_inner), 1 if reset_tau else 0)
    rc = lib().pg_solve(game, C.byref(opts), C.byref(res))
    _check(ctx, rc, "pg_solve")
    return res.major, res.inner


def pg_best_response(ctx, game, sigma, tau_inout=None, dummy_sigma=None, val_class=None, val_depth=None,
                     val_rank=None, dom=None, val_counts=None):
    _dtype_check(sigma, np.int32, "sigma")
    _dtype_check(tau_inout, np.int32, "tau_inout")
    val = pg_valuation(_ptr_kind(val_class)[0], _ptr_kind(val_depth)[0], _ptr_kind(val_rank)[0], _ptr_kind(dom)[0],
                       _same_kind(val_class, val_depth, val_rank, dom, val_counts), _ptr_kind(val_counts)[0])
    iters = C.c_int64(0)
    rc = lib().pg_best_response(game, _ptr_kind(sigma)[0], _ptr_kind(dummy_sigma)[0], _ptr_kind(tau_inout)[0],
                                _same_kind(sigma, tau_inout, dummy_sigma), C.byref(val), C.byref(iters))
    _check(ctx, rc, "pg_best_response")
    return iters.value


def pg_best_response_bf(ctx, game, sigma, tau_out=None, dummy_sigma=None, val_class=None, val_depth=None,
                        val_rank=None, dom=None, val_counts=None):
    """Bellman-Ford best response (count-vector mode); returns the rounds run."""
    _dtype_check(sigma, np.int32, "sigma")
    _dtype_check(tau_out, np.int32, "tau_out")
    val = pg_valuation(_ptr_kind(val_class)[0], _ptr_kind(val_depth)[0], _ptr_kind(val_rank)[0], _ptr_kind(dom)[0],
                       _same_kind(val_class, val_depth, val_rank, dom, val_counts), _ptr_kind(val_counts)[0])
    rounds = C.c_int64(0)
    rc = lib().pg_best_response_bf(game, _ptr_kind(sigma)[0], _ptr_kind(dummy_sigma)[0], _ptr_kind(tau_out)[0],
                                   _same_kind(sigma, tau_out, dummy_sigma), C.byref(val), C.byref(rounds))
    _check(ctx, rc, "pg_best_response_bf")
    return rounds.value


def pg_valuate(ctx, game, sigma=None, tau=None, dummy_sigma=None, val_class=None, val_depth=None, val_rank=None,
               dom=None, val_counts=None):
    """Returns the status code (PG_OK or PG_ENOTADMISSIBLE; outputs are filled in both cases)."""
    val = pg_valuation(_ptr_kind(val_class)[0], _ptr_kind(val_depth)[0], _ptr_kind(val_rank)[0], _ptr_kind(dom)[0],
                       _same_kind(val_class, val_depth, val_rank, dom, val_counts), _ptr_kind(val_counts)[0])
    rc = lib().pg_valuate(game, _ptr_kind(sigma)[0], _ptr_kind(dummy_sigma)[0], _ptr_kind(tau)[0],
                          _same_kind(sigma, tau, dummy_sigma), C.byref(val))
    if rc not in (PG_OK, PG_ENOTADMISSIBLE):
        _check(ctx, rc, "pg_valuate")
    return rc


def pg_solve_batch(ctx, ngames, vtx_base, edge_base, offsets, targets, owner, pri, max_inner=0, win=None,
                   sigma=None, tau=None, val_class=None, val_depth=None, val_rank=None, dummy_sigma=None):
    """vtx_base, edge_base: int64 numpy arrays (ngames + 1). Returns a dict with
    per-game major, inner, status (numpy), dummy_base and iterations; the given
    output arrays are filled."""
    vtx_base = np.ascontiguousarray(vtx_base, dtype=np.int64)
    edge_base = np.ascontiguousarray(edge_base, dtype=np.int64)
    for a, dt, nm in [(offsets, np.int32, "offsets"), (targets, np.int32, "targets"), (owner, np.uint8, "owner"),
                      (pri, np.int32, "pri")]:
        _dtype_check(a, dt, nm)
    kind = _same_kind(offsets, targets, owner, pri)
    major = np.zeros(ngames, np.int64)
    inner = np.zeros(ngames, np.int64)
    status = np.zeros(ngames, np.int32)
    dbase = np.zeros(ngames + 1, np.int64)
    res = pg_result_batch(_ptr_kind(win)[0], _ptr_kind(sigma)[0], _ptr_kind(tau)[0], _ptr_kind(val_class)[0],
                          _ptr_kind(val_depth)[0], _ptr_kind(val_rank)[0], _ptr_kind(dummy_sigma)[0],
                          _same_kind(win, sigma, tau, val_class, val_depth, val_rank, dummy_sigma),
                          major.ctypes.data, inner.ctypes.data, status.ctypes.data, dbase.ctypes.data, 0)
    rc = lib().pg_solve_batch(ctx, int(ngames), vtx_base.ctypes.data, edge_base.ctypes.data, _ptr_kind(offsets)[0],
                              _ptr_kind(targets)[0], _ptr_kind(owner)[0], _ptr_kind(pri)[0], kind, int(max_inner),
                              C.byref(res))
    if rc not in (PG_OK, PG_ETIMEOUT, PG_ENOTADMISSIBLE):
        _check(ctx, rc, "pg_solve_batch")
    return dict(rc=rc, major=major, inner=inner, status=status, dummy_base=dbase, iterations=res.iterations,
                load_ms=res.load_ms, pack_ms=res.pack_ms, loop_ms=res.loop_ms)


def pack_games(games):
    """Packs generator games into the pg_solve_batch input layout (host arrays)."""
    nv = np.array([g.n for g in games], np.int64)
    ne = np.array([g.m for g in games], np.int64)
    vtx_base = np.zeros(len(games) + 1, np.int64)
    edge_base = np.zeros(len(games) + 1, np.int64)
    np.cumsum(nv, out=vtx_base[1:])
    np.cumsum(ne, out=edge_base[1:])
    offsets = np.concatenate([g.offsets for g in games]).astype(np.int32)
    targets = np.concatenate([g.targets for g in games]).astype(np.int32)
    owner = np.concatenate([g.owner for g in games]).astype(np.uint8)
    pri = np.concatenate([g.pri for g in games]).astype(np.int32)
    return vtx_base, edge_base, offsets, targets, owner, pri


def pg_server_create(device=0, max_vertices=0, max_edges=0, max_games=0, round_iters=0, max_inner=0,
                     wide_offsets=False):
    opts = pg_server_opts(int(max_vertices), int(max_edges), int(max_games), int(round_iters), int(max_inner),
                          1 if wide_offsets else 0)
    sv = C.c_void_p()
    rc = lib().pg_server_create(int(device), C.byref(opts), C.byref(sv))
    if rc != PG_OK:
        raise PgError(rc, "pg_server_create")
    return sv


def pg_server_destroy(server):
    lib().pg_server_destroy(server)


def pg_server_submit(server, n, m, offsets, targets, owner, pri, tag):
    """Queues a game (host arrays, copied before the call returns)."""
    arrs = [np.ascontiguousarray(offsets, np.int32), np.ascontiguousarray(targets, np.int32),
            np.ascontiguousarray(owner, np.uint8), np.ascontiguousarray(pri, np.int32)]
    rc = lib().pg_server_submit(server, int(n), int(m), *[a.ctypes.data for a in arrs], int(tag))
    if rc != PG_OK:
        raise PgError(rc, "pg_server_submit")


def pg_server_poll(server, max_results=64, timeout_ms=0):
    """Finished games in completion order: a list of dicts."""
    buf = (pg_served * max(1, int(max_results)))()
    cnt = C.c_int32(0)
    rc = lib().pg_server_poll(server, buf, int(max_results), int(timeout_ms), C.byref(cnt))
    if rc != PG_OK:
        raise PgError(rc, "pg_server_poll: " + pg_server_error(server))
    return [{f: getattr(buf[i], f) for f, _ in pg_served._fields_} for i in range(cnt.value)]


def pg_server_fetch(server, tag, n, k, keep=True):
    """Results of a reported game as numpy arrays (and releases them); with
    keep=False they are only released."""
    if not keep:
        rc = lib().pg_server_fetch(server, int(tag), *([None] * 7))
        if rc != PG_OK:
            raise PgError(rc, "pg_server_fetch")
        return None
    out = dict(win=np.empty(n, np.uint8), sigma=np.empty(n, np.int32), tau=np.empty(n, np.int32),
               val_class=np.empty(n, np.int8), val_depth=np.empty(n, np.int32), val_rank=np.empty(n, np.int32),
               dummy_sigma=np.empty(max(k, 1), np.int8))
    rc = lib().pg_server_fetch(server, int(tag), *[out[x].ctypes.data for x in
                                                   ["win", "sigma", "tau", "val_class", "val_depth", "val_rank",
                                                    "dummy_sigma"]])
    if rc != PG_OK:
        raise PgError(rc, "pg_server_fetch")
    out["dummy_sigma"] = out["dummy_sigma"][:k]
    return out


def pg_server_get_stats(server):
    st = pg_server_stats()
    rc = lib().pg_server_get_stats(server, C.byref(st))
    if rc != PG_OK:
        raise PgError(rc, "pg_server_get_stats")
    return {f: getattr(st, f) for f, _ in pg_server_stats._fields_}


def pg_server_error(server):
    return lib().pg_server_error(server).decode()


def pg_valuate_static(n, succ, odd, val_class=None, val_depth=None, val_rank=None, stream=None):
    """Allocation-free valuation of a successor function whose vertex ids are
    priority ranks (device arrays only). Returns the status code (PG_OK or
    PG_ENOTADMISSIBLE; any other status raises PgError)."""
    arrays = [succ, odd, val_class, val_depth, val_rank]
    if any(a is not None and _ptr_kind(a)[1] != PG_MEM_DEVICE for a in arrays):
        raise ValueError("pg_valuate_static takes device arrays only")
    _dtype_check(succ, np.int32, "succ")
    _dtype_check(odd, np.uint8, "odd")
    _dtype_check(val_class, np.int8, "val_class")
    _dtype_check(val_depth, np.int32, "val_depth")
    _dtype_check(val_rank, np.int32, "val_rank")
    handle = getattr(stream, "cuda_stream", stream)
    rc = lib().pg_valuate_static(int(n), _ptr_kind(succ)[0], _ptr_kind(odd)[0], _ptr_kind(val_class)[0],
                                 _ptr_kind(val_depth)[0], _ptr_kind(val_rank)[0], C.c_void_p(handle or None))
    if rc not in (PG_OK, PG_ENOTADMISSIBLE):
        raise PgError(rc, "pg_valuate_static failed")
    return rc


def pg_set_timing(ctx, enable):
    _check(ctx, lib().pg_set_timing(ctx, 1 if enable else 0), "pg_set_timing")


def pg_set_graphs(ctx, enable):
    _check(ctx, lib().pg_set_graphs(ctx, 1 if enable else 0), "pg_set_graphs")


def pg_set_tuning(ctx, deep_cut=0, ruler_bits=0, walk_cap=0, switch_block=0, loop_ranks=0):
    """Sets the work partitioning of the valuation (zero keeps a value)."""
    t = pg_tuning(int(deep_cut), int(ruler_bits), int(walk_cap), int(switch_block), int(loop_ranks))
    _check(ctx, lib().pg_set_tuning(ctx, C.byref(t)), "pg_set_tuning")


def pg_get_tuning(ctx):
    t = pg_tuning()
    _check(ctx, lib().pg_get_tuning(ctx, C.byref(t)), "pg_get_tuning")
    return {f: getattr(t, f) for f in TUNING_FIELDS}


def pg_set_tuning_table(ctx, entries):
    """entries: [(max_ids, {field: value})] by increasing max_ids; [] clears."""
    arr = (pg_tuning_entry * max(len(entries), 1))()
    for i, (m, d) in enumerate(entries):
        arr[i].max_ids = int(m)
        arr[i].t = pg_tuning(*[int(d.get(f, 0)) for f in TUNING_FIELDS])
    _check(ctx, lib().pg_set_tuning_table(ctx, arr, len(entries)), "pg_set_tuning_table")


def pg_load_tuning(ctx, path):
    _check(ctx, lib().pg_load_tuning(ctx, str(path).encode()), "pg_load_tuning")


def pg_set_wide_offsets(ctx, enable):
    _check(ctx, lib().pg_set_wide_offsets(ctx, 1 if enable else 0), "pg_set_wide_offsets")


def pg_set_loop_ranks(ctx, enable):
    _check(ctx, lib().pg_set_loop_ranks(ctx, 1 if enable else 0), "pg_set_loop_ranks")


def pg_release_cached_memory(device=0):
    """Returns the game memory pool's cached memory on ``device`` to the driver."""
    rc = lib().pg_release_cached_memory(int(device))
    if rc != PG_OK:
        raise PgError(rc, "pg_release_cached_memory")


def pg_last_loop(game):
    """(ran_as_graph, iterations) of the last loop on game."""
    gr, it = C.c_int32(), C.c_int64()
    rc = lib().pg_last_loop(game, C.byref(gr), C.byref(it))
    if rc != PG_OK:
        raise PgError(rc, "pg_last_loop")
    return bool(gr.value), it.value


def pg_last_timing(game):
    t, v, s, k = C.c_double(), C.c_double(), C.c_double(), C.c_int64()
    lib().pg_last_timing(game, C.byref(t), C.byref(v), C.byref(s), C.byref(k))
    return dict(total_ms=t.value, valuation_ms=v.value, switch_ms=s.value, valuations=k.value)


def pg_kernel_stats(game):
    """{name: (ms, launches, calls)} per kernel class since pg_reset_stats."""
    arr = (pg_kernel_stat * 32)()
    cnt = C.c_int32(0)
    rc = lib().pg_kernel_stats(game, arr, 32, C.byref(cnt))
    if rc != PG_OK:
        raise PgError(rc, "pg_kernel_stats")
    return {arr[i].name.decode(): (arr[i].ms, arr[i].launches, arr[i].calls) for i in range(min(cnt.value, 32))}


def pg_reset_stats(game):
    rc = lib().pg_reset_stats(game)
    if rc != PG_OK:
        raise PgError(rc, "pg_reset_stats")


def pg_launch_count(ctx):
    out = C.c_int64(0)
    _check(ctx, lib().pg_launch_count(ctx, C.byref(out)), "pg_launch_count")
    return out.value


# ---------------------------------------------------------------------------
# convenience: one call from arrays to results (still marshalling only)

def solve_arrays(ctx, n, offsets, targets, owner, pri, device_outputs=False):
    """Loads, solves and frees a game; returns a dict of numpy (host) or torch
    (device) arrays plus 'major' and 'inner'."""
    game = pg_load_csr(ctx, n, int(offsets[-1]), offsets, targets, owner, pri)
    try:
        _, _, k = pg_game_info(game)
        if device_outputs:
            import torch
            dev = torch.device("cuda")
            out = dict(win=torch.empty(n, dtype=torch.uint8, device=dev),
                       sigma=torch.empty(n, dtype=torch.int32, device=dev),
                       tau=torch.empty(n, dtype=torch.int32, device=dev),
                       val_class=torch.empty(n, dtype=torch.int8, device=dev),
                       val_depth=torch.empty(n, dtype=torch.int32, device=dev),
                       val_rank=torch.empty(n, dtype=torch.int32, device=dev),
                       dummy_sigma=torch.empty(max(k, 1), dtype=torch.int8, device=dev))
        else:
            out = dict(win=np.empty(n, np.uint8), sigma=np.empty(n, np.int32), tau=np.empty(n, np.int32),
                       val_class=np.empty(n, np.int8), val_depth=np.empty(n, np.int32),
                       val_rank=np.empty(n, np.int32), dummy_sigma=np.empty(max(k, 1), np.int8))
        major, inner = pg_solve(ctx, game, **out)
        out["dummy_sigma"] = out["dummy_sigma"][:k]
        out.update(major=major, inner=inner, k=k)
        return out
    finally:
        pg_game_free(game)
