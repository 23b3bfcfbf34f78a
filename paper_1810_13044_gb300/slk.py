"""ctypes binding of the C-ABI in ``include/slk.h`` (argument marshalling only).

Every function has the name of its C entry point without the ``slk_`` prefix
and takes torch CUDA tensors for device arrays; all work runs in the CUDA
library on the tensors' device, on torch's current stream.  There is no CPU
fallback: if the library is missing or no GPU is usable, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libslk_gb300.so")

SLK_OK, SLK_NOT_CONVERGED = 0, 1
STATUS = {0: "SLK_OK", 1: "SLK_NOT_CONVERGED", -1: "SLK_ERR_INVALID_ARG", -2: "SLK_ERR_CUDA",
          -3: "SLK_ERR_OOM", -4: "SLK_ERR_TIMEOUT", -5: "SLK_ERR_NO_DEVICE",
          -6: "SLK_ERR_SCRATCH_LIMIT"}
NOALLOC_MAX_ELEMS = 4 << 20   # SLK_NOALLOC_MAX_ELEMS
AFFINITY = {"binary": 0, "heat": 1}
PRECISION = {"fp32": 0, "bf16_rerank": 1}
SIGMA_RULE = {"median": 0, "meansq": 1}

# Every symbol include/slk.h declares (checked by the CPU tests).
EXPORTS = ["slk_version", "slk_create", "slk_destroy", "slk_set_stream", "slk_last_error",
           "slk_knn_graph", "slk_sigma", "slk_unary", "slk_bound_iterate", "slk_mode_update",
           "slk_energy", "slk_default_params", "slk_solve", "slk_solve_host", "slk_profile",
           "slk_profile_read", "slk_bound_iterate_noalloc", "slk_solve_batched", "slk_server_create",
           "slk_server_destroy", "slk_server_submit", "slk_server_step", "slk_server_poll",
           "slk_server_request_bytes", "slk_unary_vec", "slk_mean_shift", "slk_energy_vec",
           "slk_solve_ms", "slk_initial_modes", "slk_barrier_selftest", "slk_kmeanspp",
           "slk_symmetrize", "slk_knn_stage_rows"]
PHASES = ["knn_prep", "knn_cand", "knn_rerank", "knn_fallback", "sigma", "unary", "bound", "mode",
          "energy", "mean_shift", "transfer"]


class SlkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("max_outer", ctypes.c_int32), ("max_inner", ctypes.c_int32),
                ("tol_inner", ctypes.c_float), ("sigma_rule", ctypes.c_int32),
                ("affinity", ctypes.c_int32), ("knn_precision", ctypes.c_int32),
                ("refine_init", ctypes.c_int32), ("reorder", ctypes.c_int32),
                ("max_ms", ctypes.c_int32), ("tol_ms", ctypes.c_float), ("tol_modes", ctypes.c_float),
                ("symmetrize", ctypes.c_int32)]


class Instance(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("N", ctypes.c_int64), ("D", ctypes.c_int32),
                ("L", ctypes.c_int32), ("k", ctypes.c_int32), ("lam", ctypes.c_float),
                ("sigma", ctypes.c_float), ("init_modes", ctypes.c_void_p), ("Z", ctypes.c_void_p),
                ("labels", ctypes.c_void_p), ("modes", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("quantum", ctypes.c_int32),
                ("memory_bytes", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int32), ("inner_iters_total", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("sigma", ctypes.c_float),
                ("energy", ctypes.c_double), ("knn_fallback_rows", ctypes.c_int64),
                ("ms_iters_total", ctypes.c_int32), ("knn_float32_rows", ctypes.c_int64),
                ("knn_exact_rows", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P, i32, i64, f32, f64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                             ctypes.c_double)
    sig = {
        "slk_version": (ctypes.c_char_p, []),
        "slk_create": (i32, [ctypes.POINTER(P), ctypes.c_int, P]),
        "slk_destroy": (i32, [P]),
        "slk_set_stream": (i32, [P, P]),
        "slk_last_error": (ctypes.c_char_p, [P]),
        "slk_knn_graph": (i32, [P, P, i64, i32, i32, i32, i32, f32, P, P, P, P, P]),
        "slk_sigma": (i32, [P, P, i64, i32, P]),
        "slk_unary": (i32, [P, P, i64, i32, P, i32, f32, P, P]),
        "slk_bound_iterate": (i32, [P, P, P, P, P, i64, i32, f32, P, P, i32, f32, P, P]),
        "slk_mode_update": (i32, [P, P, P, P, P, P, i64, i32, f32, P, P, P, P]),
        "slk_energy": (i32, [P, P, i32, P, P, P, P, i64, i32, P, f32, f32, P]),
        "slk_default_params": (None, [ctypes.POINTER(Params)]),
        "slk_solve": (i32, [P, P, i64, i32, i32, i32, f32, f32, P, ctypes.POINTER(Params), P, P, P,
                            ctypes.POINTER(Stats)]),
        "slk_solve_host": (i32, [P, P, i64, i32, i32, i32, f32, f32, P, ctypes.POINTER(Params), P, P,
                                 P, ctypes.POINTER(Stats)]),
        "slk_profile": (i32, [P, i32]),
        "slk_bound_iterate_noalloc": (i32, [P, P, P, P, P, i64, i32, f32, P, i32, f32, P, P]),
        "slk_solve_batched": (i32, [P, ctypes.POINTER(Instance), i32, ctypes.POINTER(Params),
                                    ctypes.POINTER(Stats)]),
        "slk_server_create": (i32, [P, ctypes.POINTER(ServerConfig), ctypes.POINTER(Params),
                                    ctypes.POINTER(P)]),
        "slk_server_destroy": (i32, [P]),
        "slk_server_submit": (i32, [P, ctypes.POINTER(Instance), ctypes.POINTER(i64)]),
        "slk_server_step": (i32, [P, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "slk_server_poll": (i32, [P, i64, ctypes.POINTER(i32), ctypes.POINTER(Stats)]),
        "slk_server_request_bytes": (i32, [P, ctypes.POINTER(Instance), ctypes.POINTER(i64)]),
        "slk_profile_read": (i32, [P, P, P, P]),
        "slk_unary_vec": (i32, [P, P, i64, i32, P, i32, f32, P, P]),
        "slk_mean_shift": (i32, [P, P, i32, P, P, P, P, P, i64, i32, f32, f32, P, i32, f32, P, P, P]),
        "slk_energy_vec": (i32, [P, P, i32, P, P, P, P, i64, i32, P, f32, f32, P]),
        "slk_solve_ms": (i32, [P, P, i64, i32, i32, i32, f32, f32, P, ctypes.POINTER(Params), P, P, P,
                               ctypes.POINTER(Stats)]),
        "slk_initial_modes": (i32, [P, P, i64, i32, P, i32, f32, P, P, P, ctypes.POINTER(i64)]),
        "slk_barrier_selftest": (i32, [P, i32]),
        "slk_kmeanspp": (i32, [P, P, i64, i32, i32, i32, P, P]),
        "slk_symmetrize": (i32, [P, P, P, P, i64, P, P, P, ctypes.POINTER(i64)]),
        "slk_knn_stage_rows": (i32, [P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def version() -> str:
    return load().slk_version().decode()


def default_params(**overrides) -> Params:
    p = Params()
    load().slk_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "sigma_rule" and isinstance(v, str):
            v = SIGMA_RULE[v]
        if k == "affinity" and isinstance(v, str):
            v = AFFINITY[v]
        if k == "knn_precision" and isinstance(v, str):
            v = PRECISION[v]
        setattr(p, k, v)
    return p


class Context:
    """One library context per (device, stream)."""

    def __init__(self, device: int | None = None, stream: torch.cuda.Stream | None = None):
        lib = load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        stream = stream or torch.cuda.current_stream(device)
        self.handle = ctypes.c_void_p()
        st = lib.slk_create(ctypes.byref(self.handle), device, ctypes.c_void_p(stream.cuda_stream))
        if st != SLK_OK:
            raise SlkError(st, f"slk_create(device={device}) failed")
        self._lib = lib

    def set_stream(self, stream: torch.cuda.Stream):
        self._lib.slk_set_stream(self.handle, ctypes.c_void_p(stream.cuda_stream))

    def profile(self, enable: bool):
        """Start (clearing the totals) or stop phase profiling."""
        self.check(self._lib.slk_profile(self.handle, 1 if enable else 0), "slk_profile")

    def profile_read(self):
        """-> ({phase: ms}, {phase: calls}, kernel launches since profiling was enabled)."""
        n = len(PHASES)
        ms = (ctypes.c_double * n)()
        calls = (ctypes.c_int64 * n)()
        launches = ctypes.c_int64(0)
        self.check(self._lib.slk_profile_read(self.handle, ms, calls, ctypes.byref(launches)),
                   "slk_profile_read")
        return dict(zip(PHASES, list(ms))), dict(zip(PHASES, list(calls))), launches.value

    def close(self):
        if self.handle:
            self._lib.slk_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st, what):
        if st not in (SLK_OK, SLK_NOT_CONVERGED):
            msg = self._lib.slk_last_error(self.handle).decode()
            raise SlkError(st, f"{what}: {msg}")
        return st


_ctx_cache: dict = {}


def context(device: int | None = None) -> Context:
    """A cached context bound to torch's current stream of ``device``."""
    if device is None:
        device = torch.cuda.current_device()
    ctx = _ctx_cache.get(device)
    if ctx is None:
        ctx = Context(device)
        _ctx_cache[device] = ctx
    ctx.set_stream(torch.cuda.current_stream(device))
    return ctx


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _need(t, dtype, shape, name):
    if t.dtype != dtype:
        raise TypeError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")


@dataclass
class Graph:
    row_ptr: torch.Tensor   # int64 [N+1]
    col_idx: torch.Tensor   # int32 [N*k]
    dist2: torch.Tensor     # float32 [N*k]
    w: torch.Tensor | None  # float32 [N*k] or None (binary)
    k: int
    fallback_rows: int = -1
    # rows left open by the first certificate, sent to the float32 stage, rescanned exactly
    stage_rows: tuple = (-1, -1, -1)


def knn_graph(X: torch.Tensor, k: int, affinity="binary", precision="fp32", sigma=0.0,
              ctx: Context | None = None) -> Graph:
    ctx = ctx or context(X.device.index)
    N, D = X.shape
    _need(X, torch.float32, (N, D), "X")
    dev = X.device
    row_ptr = torch.empty(N + 1, dtype=torch.int64, device=dev)
    col = torch.empty(N * k, dtype=torch.int32, device=dev)
    d2 = torch.empty(N * k, dtype=torch.float32, device=dev)
    w = torch.empty(N * k, dtype=torch.float32, device=dev) if affinity == "heat" else None
    fb = ctypes.c_int64(-1)
    ctx.check(ctx._lib.slk_knn_graph(ctx.handle, _ptr(X), N, D, k, AFFINITY[affinity],
                                     PRECISION[precision], float(sigma), _ptr(row_ptr), _ptr(col),
                                     _ptr(d2), _ptr(w), ctypes.byref(fb)), "slk_knn_graph")
    return Graph(row_ptr, col, d2, w, k, fb.value, knn_stage_rows(ctx))


def knn_stage_rows(ctx: Context | None = None) -> tuple:
    """(rows the first certificate left open, rows sent to the float32 stage,
    rows rescanned exactly) of the last kNN graph built on ctx."""
    ctx = ctx or context()
    rows = (ctypes.c_int64 * 3)()
    ctx.check(ctx._lib.slk_knn_stage_rows(ctx.handle, rows), "slk_knn_stage_rows")
    return tuple(int(r) for r in rows)


def sigma(dist2: torch.Tensor, rule="median", ctx: Context | None = None) -> float:
    ctx = ctx or context(dist2.device.index)
    _need(dist2, torch.float32, (dist2.numel(),), "dist2")
    out = ctypes.c_float(0.0)
    ctx.check(ctx._lib.slk_sigma(ctx.handle, _ptr(dist2), dist2.numel(), SIGMA_RULE[rule],
                                 ctypes.byref(out)), "slk_sigma")
    return out.value


def unary(X: torch.Tensor, modes: torch.Tensor, sig: float, with_z0=True,
          ctx: Context | None = None):
    ctx = ctx or context(X.device.index)
    N, D = X.shape
    L = modes.numel()
    _need(X, torch.float32, (N, D), "X")
    _need(modes, torch.int32, (L,), "modes")
    A = torch.empty(N, L, dtype=torch.float32, device=X.device)
    Z0 = torch.empty_like(A) if with_z0 else None
    ctx.check(ctx._lib.slk_unary(ctx.handle, _ptr(X), N, D, _ptr(modes), L, float(sig), _ptr(A),
                                 _ptr(Z0)), "slk_unary")
    return A, Z0


def bound_iterate(A, row_ptr, col_idx, w, lam, Z, Z_prev, max_iters, tol=-1.0,
                  ctx: Context | None = None):
    """In place on Z (last iterate) and Z_prev; returns (iters_done, last_delta)."""
    ctx = ctx or context(A.device.index)
    N, L = A.shape
    for t, n in ((Z, "Z"), (Z_prev, "Z_prev")):
        _need(t, torch.float32, (N, L), n)
    it = ctypes.c_int32(0)
    dl = ctypes.c_float(0.0)
    ctx.check(ctx._lib.slk_bound_iterate(ctx.handle, _ptr(A), _ptr(row_ptr), _ptr(col_idx), _ptr(w),
                                         N, L, float(lam), _ptr(Z), _ptr(Z_prev), int(max_iters),
                                         float(tol), ctypes.byref(it), ctypes.byref(dl)),
              "slk_bound_iterate")
    return it.value, dl.value


def mode_update(A, Z_prev, row_ptr, col_idx, w, lam, modes, want_labels=True,
                ctx: Context | None = None):
    """In place on modes; returns (changed, labels, mode_key)."""
    ctx = ctx or context(A.device.index)
    N, L = A.shape
    _need(modes, torch.int32, (L,), "modes")
    labels = torch.empty(N, dtype=torch.int32, device=A.device) if want_labels else None
    key = torch.empty(L, dtype=torch.float32, device=A.device)
    ch = ctypes.c_int32(0)
    ctx.check(ctx._lib.slk_mode_update(ctx.handle, _ptr(A), _ptr(Z_prev), _ptr(row_ptr),
                                       _ptr(col_idx), _ptr(w), N, L, float(lam), _ptr(modes),
                                       _ptr(labels), _ptr(key), ctypes.byref(ch)), "slk_mode_update")
    return ch.value, labels, key


def energy(X, labels, row_ptr, col_idx, w, L, modes, sig, lam, ctx: Context | None = None) -> float:
    ctx = ctx or context(X.device.index)
    N, D = X.shape
    E = ctypes.c_double(0.0)
    ctx.check(ctx._lib.slk_energy(ctx.handle, _ptr(X), D, _ptr(labels), _ptr(row_ptr), _ptr(col_idx),
                                  _ptr(w), N, int(L), _ptr(modes), float(sig), float(lam),
                                  ctypes.byref(E)), "slk_energy")
    return E.value


def solve(X: torch.Tensor, L: int, k: int, lam: float, init_modes: torch.Tensor, sigma=0.0,
          params: Params | None = None, ctx: Context | None = None, out=None):
    """Whole SLK-BO on device tensors -> (Z, labels, modes, stats dict)."""
    ctx = ctx or context(X.device.index)
    N, D = X.shape
    _need(X, torch.float32, (N, D), "X")
    _need(init_modes, torch.int32, (L,), "init_modes")
    if out is None:
        Z = torch.empty(N, L, dtype=torch.float32, device=X.device)
        labels = torch.empty(N, dtype=torch.int32, device=X.device)
        modes = torch.empty(L, dtype=torch.int32, device=X.device)
    else:
        Z, labels, modes = out
    st = Stats()
    p = params or default_params()
    ctx.check(ctx._lib.slk_solve(ctx.handle, _ptr(X), N, D, L, k, float(lam), float(sigma),
                                 _ptr(init_modes), ctypes.byref(p), _ptr(Z), _ptr(labels),
                                 _ptr(modes), ctypes.byref(st)), "slk_solve")
    return Z, labels, modes, st.as_dict()


def solve_host(X, L: int, k: int, lam: float, init_modes, sigma=0.0, params: Params | None = None,
               ctx: Context | None = None, want_z=False, out=None):
    """slk_solve_host on host (CPU, ideally pinned) tensors -> (Z, labels, modes, stats)."""
    ctx = ctx or context()
    N, D = X.shape
    if X.is_cuda or X.dtype != torch.float32 or not X.is_contiguous():
        raise ValueError("X must be a contiguous float32 CPU tensor")
    init = init_modes.to(torch.int32).contiguous()
    if out is None:
        labels = torch.empty(N, dtype=torch.int32)
        modes = torch.empty(L, dtype=torch.int32)
        Z = torch.empty(N, L, dtype=torch.float32) if want_z else None
    else:
        Z, labels, modes = out
    st = Stats()
    p = params or default_params()
    hp = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    ctx.check(ctx._lib.slk_solve_host(ctx.handle, hp(X), N, D, L, k, float(lam), float(sigma),
                                      hp(init), ctypes.byref(p), hp(Z), hp(labels), hp(modes),
                                      ctypes.byref(st)), "slk_solve_host")
    return Z, labels, modes, st.as_dict()


def initial_modes(X: torch.Tensor, seeds: torch.Tensor, sig: float, want_assign=True,
                  ctx: Context | None = None, stats: dict | None = None):
    """slk_initial_modes -> (modes int32 [L], assign int32 [N] or None, density list [L]).
    stats (optional dict) receives the number of exactly recomputed sums."""
    ctx = ctx or context(X.device.index)
    N, D = X.shape
    L = seeds.numel()
    _need(X, torch.float32, (N, D), "X")
    _need(seeds, torch.int32, (L,), "seeds")
    modes = torch.empty(L, dtype=torch.int32, device=X.device)
    assign = torch.empty(N, dtype=torch.int32, device=X.device) if want_assign else None
    dens = (ctypes.c_double * L)()
    ncand = ctypes.c_int64(0)
    ctx.check(ctx._lib.slk_initial_modes(ctx.handle, _ptr(X), N, D, _ptr(seeds), L, float(sig),
                                         _ptr(modes), _ptr(assign), dens, ctypes.byref(ncand)),
              "slk_initial_modes")
    if stats is not None:
        stats["candidates"] = ncand.value
    return modes, assign, list(dens)


# ---------------------------------------------------------------- SLK-MS

def unary_vec(X: torch.Tensor, M: torch.Tensor, sig: float, with_z0=True,
              ctx: Context | None = None):
    """slk_unary_vec: unary term with vector modes M [L, D] -> (A, Z0)."""
    ctx = ctx or context(X.device.index)
    N, D = X.shape
    L = M.shape[0]
    _need(X, torch.float32, (N, D), "X")
    _need(M, torch.float32, (L, D), "M")
    A = torch.empty(N, L, dtype=torch.float32, device=X.device)
    Z0 = torch.empty_like(A) if with_z0 else None
    ctx.check(ctx._lib.slk_unary_vec(ctx.handle, _ptr(X), N, D, _ptr(M), L, float(sig), _ptr(A),
                                     _ptr(Z0)), "slk_unary_vec")
    return A, Z0


def mean_shift(X, A, Z_prev, row_ptr, col_idx, w, lam, sig, M, max_iters, tol=-1.0,
               want_labels=True, ctx: Context | None = None):
    """slk_mean_shift, in place on M [L, D]; returns (iters_done, last_shift, labels)."""
    ctx = ctx or context(X.device.index)
    N, D = X.shape
    L = A.shape[1]
    _need(X, torch.float32, (N, D), "X")
    _need(A, torch.float32, (N, L), "A")
    _need(M, torch.float32, (L, D), "M")
    if Z_prev is not None:
        _need(Z_prev, torch.float32, (N, L), "Z_prev")
    labels = torch.empty(N, dtype=torch.int32, device=X.device) if want_labels else None
    it = ctypes.c_int32(0)
    sh = ctypes.c_float(0.0)
    ctx.check(ctx._lib.slk_mean_shift(ctx.handle, _ptr(X), D, _ptr(A), _ptr(Z_prev), _ptr(row_ptr),
                                      _ptr(col_idx), _ptr(w), N, L, float(lam), float(sig), _ptr(M),
                                      int(max_iters), float(tol), _ptr(labels), ctypes.byref(it),
                                      ctypes.byref(sh)), "slk_mean_shift")
    return it.value, sh.value, labels


def energy_vec(X, labels, row_ptr, col_idx, w, M, sig, lam, ctx: Context | None = None) -> float:
    """slk_energy_vec: Eq. (1) with vector modes M [L, D]."""
    ctx = ctx or context(X.device.index)
    N, D = X.shape
    E = ctypes.c_double(0.0)
    ctx.check(ctx._lib.slk_energy_vec(ctx.handle, _ptr(X), D, _ptr(labels), _ptr(row_ptr),
                                      _ptr(col_idx), _ptr(w), N, M.shape[0], _ptr(M), float(sig),
                                      float(lam), ctypes.byref(E)), "slk_energy_vec")
    return E.value


def solve_ms(X: torch.Tensor, L: int, k: int, lam: float, init_modes: torch.Tensor, sigma=0.0,
             params: Params | None = None, ctx: Context | None = None, out=None):
    """Whole SLK-MS on device tensors -> (Z, labels, M [L, D], stats dict)."""
    ctx = ctx or context(X.device.index)
    N, D = X.shape
    _need(X, torch.float32, (N, D), "X")
    _need(init_modes, torch.int32, (L,), "init_modes")
    if out is None:
        Z = torch.empty(N, L, dtype=torch.float32, device=X.device)
        labels = torch.empty(N, dtype=torch.int32, device=X.device)
        M = torch.empty(L, D, dtype=torch.float32, device=X.device)
    else:
        Z, labels, M = out
    st = Stats()
    p = params or default_params()
    ctx.check(ctx._lib.slk_solve_ms(ctx.handle, _ptr(X), N, D, L, k, float(lam), float(sigma),
                                    _ptr(init_modes), ctypes.byref(p), _ptr(Z), _ptr(labels),
                                    _ptr(M), ctypes.byref(st)), "slk_solve_ms")
    return Z, labels, M, st.as_dict()


def symmetrize(row_ptr, col_idx, w, N: int, ctx: Context | None = None):
    """slk_symmetrize: (K + K^t) / 2 of a device CSR K (w None: binary) ->
    (row_ptr int64 [N+1], col_idx int32 [nnz'], w float32 [nnz'])."""
    ctx = ctx or context(row_ptr.device.index)
    nnz = col_idx.numel()
    dev = row_ptr.device
    out_rp = torch.empty(N + 1, dtype=torch.int64, device=dev)
    out_ci = torch.empty(max(2 * nnz, 1), dtype=torch.int32, device=dev)
    out_w = torch.empty(max(2 * nnz, 1), dtype=torch.float32, device=dev)
    n_out = ctypes.c_int64(0)
    ctx.check(ctx._lib.slk_symmetrize(ctx.handle, _ptr(row_ptr), _ptr(col_idx), _ptr(w), int(N),
                                      _ptr(out_rp), _ptr(out_ci), _ptr(out_w), ctypes.byref(n_out)),
              "slk_symmetrize")
    return out_rp, out_ci[:n_out.value], out_w[:n_out.value]


def kmeanspp(X: torch.Tensor, L: int, first: int, u, ctx: Context | None = None) -> torch.Tensor:
    """slk_kmeanspp: K-means++ seeds of X from the draws (first index, L - 1
    uniforms in [0, 1), e.g. inputs.kmeanspp_draws) -> int32 CUDA tensor [L]."""
    import numpy as np
    ctx = ctx or context(X.device.index)
    N, D = X.shape
    _need(X, torch.float32, (N, D), "X")
    uh = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1))
    seeds = torch.empty(L, dtype=torch.int32, device=X.device)
    ctx.check(ctx._lib.slk_kmeanspp(ctx.handle, _ptr(X), N, D, int(L), int(first),
                                    uh.ctypes.data_as(ctypes.c_void_p) if uh.size else None,
                                    _ptr(seeds)), "slk_kmeanspp")
    return seeds


def barrier_selftest(timeout_ms=50, ctx: Context | None = None):
    """slk_barrier_selftest: the bounded device-wide wait must give up; raises
    SlkError (SLK_ERR_TIMEOUT when the failure path works)."""
    ctx = ctx or context()
    ctx.check(ctx._lib.slk_barrier_selftest(ctx.handle, int(timeout_ms)), "slk_barrier_selftest")


def bound_iterate_noalloc(A, row_ptr, col_idx, w, lam, Z, max_iters, tol=-1.0):
    """slk_bound_iterate_noalloc: the z-updates with the library's static
    scratch (no allocation, no context), on torch's current stream of Z's
    device.  In place on Z; returns (iters_done, last_delta)."""
    lib = load()
    N, L = A.shape
    _need(Z, torch.float32, (N, L), "Z")
    it = ctypes.c_int32(0)
    dl = ctypes.c_float(0.0)
    with torch.cuda.device(Z.device):
        stream = torch.cuda.current_stream(Z.device)
        st = lib.slk_bound_iterate_noalloc(ctypes.c_void_p(stream.cuda_stream), _ptr(A), _ptr(row_ptr),
                                           _ptr(col_idx), _ptr(w), N, L, float(lam), _ptr(Z),
                                           int(max_iters), float(tol), ctypes.byref(it),
                                           ctypes.byref(dl))
    if st != SLK_OK:
        raise SlkError(st, "slk_bound_iterate_noalloc")
    return it.value, dl.value


def solve_batched(problems, params: Params | None = None, ctx: Context | None = None, outs=None):
    """slk_solve_batched.  ``problems``: list of dicts with X (CUDA float32
    N x D), L, k, lam, init_modes (CUDA int32 [L]) and optional sigma.
    Returns a list of (Z, labels, modes, stats dict)."""
    if not problems:
        return []
    ctx = ctx or context(problems[0]["X"].device.index)
    n = len(problems)
    arr = (Instance * n)()
    stats = (Stats * n)()
    keep = []
    for i, pr in enumerate(problems):
        X = pr["X"]
        N, D = X.shape
        L = int(pr["L"])
        _need(X, torch.float32, (N, D), "X")
        _need(pr["init_modes"], torch.int32, (L,), "init_modes")
        if outs is not None:
            Z, lab, modes = outs[i]
        else:
            Z = torch.empty(N, L, dtype=torch.float32, device=X.device)
            lab = torch.empty(N, dtype=torch.int32, device=X.device)
            modes = torch.empty(L, dtype=torch.int32, device=X.device)
        keep.append((Z, lab, modes))
        arr[i] = Instance(X.data_ptr(), N, D, L, int(pr["k"]), float(pr["lam"]), float(pr.get("sigma", 0.0)),
                          pr["init_modes"].data_ptr(), Z.data_ptr(), lab.data_ptr(), modes.data_ptr())
    p = params or default_params()
    ctx.check(ctx._lib.slk_solve_batched(ctx.handle, arr, n, ctypes.byref(p), stats), "slk_solve_batched")
    return [(z, l, m, stats[i].as_dict()) for i, (z, l, m) in enumerate(keep)]


class Server:
    """Continuous-batching server (slk_server_*).  ``submit`` takes a problem
    dict like :func:`solve_batched`'s and returns a ticket; ``step`` admits and
    advances; ``poll`` returns (state, result) with result = (Z, labels, modes,
    stats) once done (state 3)."""

    QUEUED, BUILDING, ITERATING, DONE = 0, 1, 2, 3

    def __init__(self, max_slots=64, quantum=10, memory_bytes=8 << 30, params: Params | None = None,
                 ctx: Context | None = None):
        self.ctx = ctx or context()
        self._lib = self.ctx._lib
        cfg = ServerConfig(int(max_slots), int(quantum), int(memory_bytes))
        self.params = params or default_params()
        self.handle = ctypes.c_void_p()
        self.ctx.check(self._lib.slk_server_create(self.ctx.handle, ctypes.byref(cfg), ctypes.byref(self.params),
                                                   ctypes.byref(self.handle)), "slk_server_create")
        self._live = {}

    def submit(self, pr, out=None) -> int:
        X = pr["X"]
        N, D = X.shape
        L = int(pr["L"])
        _need(X, torch.float32, (N, D), "X")
        _need(pr["init_modes"], torch.int32, (L,), "init_modes")
        if out is None:
            out = (torch.empty(N, L, dtype=torch.float32, device=X.device),
                   torch.empty(N, dtype=torch.int32, device=X.device),
                   torch.empty(L, dtype=torch.int32, device=X.device))
        Z, lab, modes = out
        inst = Instance(X.data_ptr(), N, D, L, int(pr["k"]), float(pr["lam"]), float(pr.get("sigma", 0.0)),
                        pr["init_modes"].data_ptr(), Z.data_ptr(), lab.data_ptr(), modes.data_ptr())
        t = ctypes.c_int64(0)
        self.ctx.check(self._lib.slk_server_submit(self.handle, ctypes.byref(inst), ctypes.byref(t)),
                       "slk_server_submit")
        self._live[t.value] = (pr, out)
        return t.value

    def request_bytes(self, pr) -> int:
        X = pr["X"]
        N, D = X.shape
        inst = Instance(X.data_ptr(), N, D, int(pr["L"]), int(pr["k"]), float(pr["lam"]), 0.0,
                        pr["init_modes"].data_ptr(), 0, 0, 0)
        b = ctypes.c_int64(0)
        self.ctx.check(self._lib.slk_server_request_bytes(self.handle, ctypes.byref(inst), ctypes.byref(b)),
                       "slk_server_request_bytes")
        return b.value

    def step(self):
        r, q = ctypes.c_int32(0), ctypes.c_int32(0)
        self.ctx.check(self._lib.slk_server_step(self.handle, ctypes.byref(r), ctypes.byref(q)),
                       "slk_server_step")
        return r.value, q.value

    def poll(self, ticket):
        st = ctypes.c_int32(0)
        stats = Stats()
        self.ctx.check(self._lib.slk_server_poll(self.handle, int(ticket), ctypes.byref(st), ctypes.byref(stats)),
                       "slk_server_poll")
        if st.value != self.DONE:
            return st.value, None
        _, out = self._live.pop(ticket)
        return st.value, (*out, stats.as_dict())

    def run_until_done(self, tickets, max_steps=100000):
        """Step until every ticket is done; returns {ticket: result}."""
        results, pending = {}, set(tickets)
        for _ in range(max_steps):
            if not pending:
                break
            self.step()
            for t in list(pending):
                st, res = self.poll(t)
                if st == self.DONE:
                    results[t] = res
                    pending.discard(t)
        if pending:
            raise RuntimeError(f"{len(pending)} requests not done after {max_steps} steps")
        return results

    def close(self):
        if self.handle:
            self._lib.slk_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
