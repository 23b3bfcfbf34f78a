"""FP64 CPU oracle for Scalable Laplacian K-modes (SLK-BO, SLK-MS) -- ctypes front end.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import this package.  It is
independent of the CUDA path: it shares no code with it and never takes an
input that the CUDA path produced.

The arithmetic lives in ``slk_oracle.c`` (plain C, double precision); this
module only builds it with gcc (with OpenMP where the compiler has it: rows
that are independent run on all host cores, with results identical to one
thread) and marshals numpy arrays.
Parity of each function is pinned by the ``-m "not gpu"`` tests under
``tests/`` (brute force, closed forms, invariants, library special cases).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slk_oracle.c")
_HDR = os.path.join(_HERE, "slk_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None

# -ffp-contract=off: no fused multiply-add, so x86 and Arm builds round alike.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (idempotent; rebuilds when the source is newer).
    OpenMP is used when gcc accepts -fopenmp, else the loops run on one thread."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    src_m = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR), os.path.getmtime(__file__))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < src_m:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        try:
            subprocess.check_call(["gcc", *CFLAGS, "-fopenmp", "-o", tmp, _SRC, "-lm"],
                                  stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "oracle_threads": (i32, [i32]),
        "oracle_pair_d2": (i32, [P, i64, i32, P, P, i64, P]),
        "oracle_knn_rows": (i32, [P, i64, i32, i32, P, i64, P, P]),
        "oracle_knn": (i32, [P, i64, i32, i32, P, P]),
        "oracle_sigma": (f64, [P, i64, i32]),
        "oracle_gauss": (f64, [f64, f64]),
        "oracle_heat_weights": (None, [P, i64, f64, P]),
        "oracle_unary": (i32, [P, i64, i32, P, i32, f64, P]),
        "oracle_softmax_rows": (None, [P, i64, i32, P]),
        "oracle_pairwise": (None, [P, P, P, i64, i32, P, P]),
        "oracle_logits": (None, [P, P, P, P, i64, i32, f64, P, P]),
        "oracle_bound_iterate": (i32, [P, P, P, P, i64, i32, f64, P, i32, f64, P, P, P]),
        "oracle_log_z": (None, [P, i64, i32, P]),
        "oracle_mode_update": (None, [P, i64, i32, P, P]),
        "oracle_labels": (None, [P, i64, i32, P]),
        "oracle_energy": (f64, [P, i32, P, P, P, P, i64, i32, P, f64, f64]),
        "oracle_relaxed": (f64, [P, P, P, P, P, i64, i32, f64]),
        "oracle_solve_graph": (i32, [P, i64, i32, i32, P, P, P, f64, f64, P, i32, i32, f64,
                                     P, P, P, P, P]),
        "oracle_unary_vec": (i32, [P, i64, i32, P, i32, f64, P]),
        "oracle_mean_shift": (i32, [P, i64, i32, P, i32, f64, P, i32, f64, P, P]),
        "oracle_energy_vec": (f64, [P, i32, P, P, P, P, i64, i32, P, f64, f64]),
        "oracle_solve_ms_graph": (i32, [P, i64, i32, i32, P, P, P, f64, f64, P, i32, i32, f64,
                                        i32, f64, f64, P, P, P, P, P, P]),
        "oracle_initial_modes": (i32, [P, i64, i32, P, i32, f64, P, P, P]),
        "oracle_cluster_density": (i32, [P, i64, i32, P, i32, f64, P, i64, P]),
        "oracle_kmeanspp": (i32, [P, i64, i32, i32, i32, P, P]),
        "oracle_symmetrize": (i32, [P, P, P, i64, P, P, P, i64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc < 0:
        raise ValueError(f"oracle {what}: invalid arguments (code {rc})")


def threads(n: int = 0) -> int:
    """Threads of the oracle's row-parallel loops (n > 0 sets the count first)."""
    return int(_load().oracle_threads(int(n)))


def pair_d2(X, p, q):
    """||x_p - x_q||^2 (float64, the kNN scan's own sums) for the pairs (p[i], q[i])."""
    lib = _load()
    X = _c(X, np.float32)
    p = _c(p, np.int64).reshape(-1)
    q = _c(q, np.int64).reshape(-1)
    out = np.empty(p.size, np.float64)
    _check(lib.oracle_pair_d2(_p(X), X.shape[0], X.shape[1], _p(p), _p(q), p.size, _p(out)), "pair_d2")
    return out


def knn(X, k, rows=None):
    """Exact kNN (Section 4.2) -> (idx int32 [n,k], d2 float64 [n,k])."""
    lib = _load()
    X = _c(X, np.float32)
    N, D = X.shape
    rows = np.arange(N, dtype=np.int64) if rows is None else _c(rows, np.int64)
    idx = np.empty((len(rows), k), np.int32)
    d2 = np.empty((len(rows), k), np.float64)
    _check(lib.oracle_knn_rows(_p(X), N, D, k, _p(rows), len(rows), _p(idx), _p(d2)), "knn")
    return idx, d2


def sigma(d2, rule="median"):
    """Kernel width (Section 4.2): 'median' of sqrt(d2) or the paper's 'meansq'."""
    lib = _load()
    d2 = _c(d2, np.float64).reshape(-1)
    return float(lib.oracle_sigma(_p(d2), d2.size, 0 if rule == "median" else 1))


def gauss(d2, sig):
    return float(_load().oracle_gauss(float(d2), float(sig)))


def heat_weights(d2, sig):
    lib = _load()
    d2 = _c(d2, np.float64).reshape(-1)
    w = np.empty_like(d2)
    lib.oracle_heat_weights(_p(d2), d2.size, float(sig), _p(w))
    return w


def unary(X, modes, sig):
    """a_{p,l} = k(x_p, x_{modes[l]}) (Eq. general-second) -> float64 [N, L]."""
    lib = _load()
    X = _c(X, np.float32)
    modes = _c(modes, np.int32)
    N, D = X.shape
    A = np.empty((N, len(modes)), np.float64)
    _check(lib.oracle_unary(_p(X), N, D, _p(modes), len(modes), float(sig), _p(A)), "unary")
    return A


def softmax_rows(S):
    lib = _load()
    S = _c(S, np.float64)
    Z = np.empty_like(S)
    lib.oracle_softmax_rows(_p(S), S.shape[0], S.shape[1], _p(Z))
    return Z


def _graph(row_ptr, col_idx, w):
    return (_c(row_ptr, np.int64), _c(col_idx, np.int32),
            None if w is None else _c(w, np.float64))


def pairwise(row_ptr, col_idx, w, Z):
    lib = _load()
    rp, ci, ww = _graph(row_ptr, col_idx, w)
    Z = _c(Z, np.float64)
    B = np.empty_like(Z)
    lib.oracle_pairwise(_p(rp), _p(ci), _p(ww), Z.shape[0], Z.shape[1], _p(Z), _p(B))
    return B


def logits(A, row_ptr, col_idx, w, lam, Z):
    lib = _load()
    rp, ci, ww = _graph(row_ptr, col_idx, w)
    A = _c(A, np.float64)
    Z = _c(Z, np.float64)
    S = np.empty_like(A)
    lib.oracle_logits(_p(A), _p(rp), _p(ci), _p(ww), A.shape[0], A.shape[1], float(lam), _p(Z), _p(S))
    return S


def bound_iterate(A, row_ptr, col_idx, w, lam, Z0, max_iters, tol=-1.0):
    """Inner z-updates of Algorithm 1 -> (Z, Zprev, iters, last_delta)."""
    lib = _load()
    rp, ci, ww = _graph(row_ptr, col_idx, w)
    A = _c(A, np.float64)
    Z = np.array(Z0, dtype=np.float64, order="C", copy=True)
    Zp = np.empty_like(Z)
    it = ctypes.c_int(0)
    dl = ctypes.c_double(0.0)
    _check(lib.oracle_bound_iterate(_p(A), _p(rp), _p(ci), _p(ww), A.shape[0], A.shape[1], float(lam),
                                    _p(Z), int(max_iters), float(tol), _p(Zp),
                                    ctypes.byref(it), ctypes.byref(dl)), "bound_iterate")
    return Z, Zp, it.value, dl.value


def log_z(S):
    lib = _load()
    S = _c(S, np.float64)
    out = np.empty_like(S)
    lib.oracle_log_z(_p(S), S.shape[0], S.shape[1], _p(out))
    return out


def mode_update(S):
    """Eq. (mode_byproduct) on logits S -> (modes int32 [L], best log z [L])."""
    lib = _load()
    S = _c(S, np.float64)
    N, L = S.shape
    m = np.empty(L, np.int32)
    key = np.empty(L, np.float64)
    lib.oracle_mode_update(_p(S), N, L, _p(m), _p(key))
    return m, key


def labels(S):
    lib = _load()
    S = _c(S, np.float64)
    out = np.empty(S.shape[0], np.int32)
    lib.oracle_labels(_p(S), S.shape[0], S.shape[1], _p(out))
    return out


def energy(X, labels_, row_ptr, col_idx, w, L, modes, sig, lam):
    """Discrete energy, Eq. (1), at one-hot labels and modes."""
    lib = _load()
    X = _c(X, np.float32)
    rp, ci, ww = _graph(row_ptr, col_idx, w)
    lab = _c(labels_, np.int32)
    modes = _c(modes, np.int32)
    return float(lib.oracle_energy(_p(X), X.shape[1], _p(lab), _p(rp), _p(ci), _p(ww),
                                   X.shape[0], int(L), _p(modes), float(sig), float(lam)))


def relaxed(A, Z, row_ptr, col_idx, w, lam_pair):
    """Relaxed objective, Eq. (2), with pairwise weight ``lam_pair``."""
    lib = _load()
    rp, ci, ww = _graph(row_ptr, col_idx, w)
    A = _c(A, np.float64)
    Z = _c(Z, np.float64)
    return float(lib.oracle_relaxed(_p(A), _p(Z), _p(rp), _p(ci), _p(ww), A.shape[0], A.shape[1],
                                    float(lam_pair)))


def knn_graph(X, k, affinity="binary", sig=None):
    """Exact kNN graph in CSR form: (row_ptr, col_idx, w or None, d2)."""
    idx, d2 = knn(X, k)
    N = X.shape[0]
    row_ptr = np.arange(N + 1, dtype=np.int64) * k
    w = None
    if affinity == "heat":
        w = heat_weights(d2, sig)
    return row_ptr, idx.reshape(-1), w, d2.reshape(-1)


def solve_graph(X, L, row_ptr, col_idx, w, sig, lam, init_modes,
                max_outer=50, max_inner=100, tol=1e-6):
    """Algorithm 1 (SLK-BO) on a given graph -> dict of results."""
    lib = _load()
    X = _c(X, np.float32)
    N, D = X.shape
    rp, ci, ww = _graph(row_ptr, col_idx, w)
    modes = np.array(init_modes, dtype=np.int32, copy=True)
    Z = np.empty((N, L), np.float64)
    lab = np.empty(N, np.int32)
    E = ctypes.c_double(0.0)
    od = ctypes.c_int(0)
    it = ctypes.c_int(0)
    rc = lib.oracle_solve_graph(_p(X), N, D, int(L), _p(rp), _p(ci), _p(ww), float(sig), float(lam),
                                _p(modes), int(max_outer), int(max_inner), float(tol),
                                _p(Z), _p(lab), ctypes.byref(E), ctypes.byref(od), ctypes.byref(it))
    _check(rc, "solve_graph")
    return dict(Z=Z, labels=lab, modes=modes, E=E.value, outer=od.value, inner_total=it.value,
                converged=(rc == 0))


def solve(X, L, k, lam, init_modes, sigma_rule="median", affinity="binary", sig=None,
          max_outer=50, max_inner=100, tol=1e-6, symmetric=False):
    """Whole SLK-BO: exact kNN graph, kernel width, Algorithm 1 (on the
    symmetric affinity (K + K^t) / 2 when ``symmetric``)."""
    t0 = time.perf_counter()
    idx, d2 = knn(X, k)
    if sig is None:
        sig = sigma(d2, sigma_rule)
    N = X.shape[0]
    row_ptr = np.arange(N + 1, dtype=np.int64) * k
    w = heat_weights(d2.reshape(-1), sig) if affinity == "heat" else None
    col = idx.reshape(-1)
    if symmetric:
        row_ptr, col, w = symmetrize(row_ptr, col, w, N)
    out = solve_graph(X, L, row_ptr, col, w, sig, lam, init_modes,
                      max_outer, max_inner, tol)
    out.update(knn_idx=idx, knn_d2=d2, sigma=sig, row_ptr=row_ptr, w=w,
               seconds=time.perf_counter() - t0)
    return out


# ---------------------------------------------------------------- SLK-MS

def unary_vec(X, M, sig):
    """a_{p,l} = k(x_p, m_l) with vector modes M [L, D] -> float64 [N, L]."""
    lib = _load()
    X = _c(X, np.float32)
    M = _c(M, np.float64)
    N, D = X.shape
    A = np.empty((N, M.shape[0]), np.float64)
    _check(lib.oracle_unary_vec(_p(X), N, D, _p(M), M.shape[0], float(sig), _p(A)), "unary_vec")
    return A


def mean_shift(X, logZ, M0, sig, max_iters, tol=-1.0):
    """Eq. (mean-shift) with z fixed (given as log z) -> (M, iters, last_shift)."""
    lib = _load()
    X = _c(X, np.float32)
    logZ = _c(logZ, np.float64)
    M = np.array(M0, dtype=np.float64, order="C", copy=True)
    N, D = X.shape
    it = ctypes.c_int(0)
    sh = ctypes.c_double(0.0)
    _check(lib.oracle_mean_shift(_p(X), N, D, _p(logZ), M.shape[0], float(sig), _p(M),
                                 int(max_iters), float(tol), ctypes.byref(it), ctypes.byref(sh)),
           "mean_shift")
    return M, it.value, sh.value


def energy_vec(X, labels_, row_ptr, col_idx, w, M, sig, lam):
    """Discrete energy, Eq. (1), at one-hot labels and vector modes M [L, D]."""
    lib = _load()
    X = _c(X, np.float32)
    rp, ci, ww = _graph(row_ptr, col_idx, w)
    lab = _c(labels_, np.int32)
    M = _c(M, np.float64)
    return float(lib.oracle_energy_vec(_p(X), X.shape[1], _p(lab), _p(rp), _p(ci), _p(ww),
                                       X.shape[0], M.shape[0], _p(M), float(sig), float(lam)))


def solve_ms_graph(X, L, row_ptr, col_idx, w, sig, lam, init_M, max_outer=50, max_inner=100,
                   tol=1e-6, max_ms=100, tol_ms=1e-5, tol_outer=1e-3):
    """Algorithm 1 (SLK-MS) on a given graph -> dict of results (modes as vectors)."""
    lib = _load()
    X = _c(X, np.float32)
    N, D = X.shape
    rp, ci, ww = _graph(row_ptr, col_idx, w)
    M = np.array(init_M, dtype=np.float64, order="C", copy=True).reshape(L, D)
    Z = np.empty((N, L), np.float64)
    lab = np.empty(N, np.int32)
    E = ctypes.c_double(0.0)
    od, it, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    rc = lib.oracle_solve_ms_graph(_p(X), N, D, int(L), _p(rp), _p(ci), _p(ww), float(sig),
                                   float(lam), _p(M), int(max_outer), int(max_inner), float(tol),
                                   int(max_ms), float(tol_ms), float(tol_outer), _p(Z), _p(lab),
                                   ctypes.byref(E), ctypes.byref(od), ctypes.byref(it),
                                   ctypes.byref(ms))
    _check(rc, "solve_ms_graph")
    return dict(Z=Z, labels=lab, M=M, E=E.value, outer=od.value, inner_total=it.value,
                ms_total=ms.value, converged=(rc == 0))


def solve_ms(X, L, k, lam, init_modes, sigma_rule="median", affinity="binary", sig=None,
             max_outer=50, max_inner=100, tol=1e-6, max_ms=100, tol_ms=1e-5, tol_outer=1e-3):
    """Whole SLK-MS: exact kNN graph, kernel width, Algorithm 1 with mean-shift modes
    starting from the points x_{init_modes[l]}."""
    t0 = time.perf_counter()
    idx, d2 = knn(X, k)
    if sig is None:
        sig = sigma(d2, sigma_rule)
    N = X.shape[0]
    row_ptr = np.arange(N + 1, dtype=np.int64) * k
    w = heat_weights(d2.reshape(-1), sig) if affinity == "heat" else None
    M0 = np.asarray(X, np.float64)[np.asarray(init_modes)]
    out = solve_ms_graph(X, L, row_ptr, idx.reshape(-1), w, sig, lam, M0, max_outer, max_inner,
                         tol, max_ms, tol_ms, tol_outer)
    out.update(knn_idx=idx, knn_d2=d2, sigma=sig, row_ptr=row_ptr, w=w,
               seconds=time.perf_counter() - t0)
    return out


# ---------------------------------------------------------------- starting modes

def initial_modes(X, seeds, sig):
    """Section 4.2 starting modes: nearest-seed assignment, then the mode
    definition of Eq. (1) -> (modes int32 [L], assign int32 [N], density [L])."""
    lib = _load()
    X = _c(X, np.float32)
    seeds = _c(seeds, np.int32)
    N, D = X.shape
    L = len(seeds)
    modes = np.empty(L, np.int32)
    assign = np.empty(N, np.int32)
    dens = np.empty(L, np.float64)
    _check(lib.oracle_initial_modes(_p(X), N, D, _p(seeds), L, float(sig), _p(modes), _p(assign),
                                    _p(dens)), "initial_modes")
    return modes, assign, dens


def cluster_density(X, assign, l, sig, ys):
    """sum_{p: assign[p] = l} k(x_p, x_y) for each y in ys."""
    lib = _load()
    X = _c(X, np.float32)
    assign = _c(assign, np.int32)
    ys = _c(ys, np.int64)
    out = np.empty(len(ys), np.float64)
    _check(lib.oracle_cluster_density(_p(X), X.shape[0], X.shape[1], _p(assign), int(l), float(sig),
                                      _p(ys), len(ys), _p(out)), "cluster_density")
    return out


# ---------------------------------------------------------------- K-means++ seeds

def kmeanspp(X, L, first, u):
    """K-means++ seeds from the given draws (first index, L - 1 uniforms in
    [0, 1)) -> int32 [L]."""
    lib = _load()
    X = _c(X, np.float32)
    u = _c(u, np.float64).reshape(-1)
    if u.size != max(L - 1, 0):
        raise ValueError("need L - 1 uniform draws")
    seeds = np.empty(L, np.int32)
    _check(lib.oracle_kmeanspp(_p(X), X.shape[0], X.shape[1], int(L), int(first),
                               _p(u) if u.size else None, _p(seeds)), "kmeanspp")
    return seeds


# ---------------------------------------------------------------- symmetric affinity

def symmetrize(row_ptr, col_idx, w, N):
    """(K + K^t) / 2 of a CSR K -> (row_ptr, col_idx, w float64); w None: binary K."""
    lib = _load()
    rp, ci, ww = _graph(row_ptr, col_idx, w)
    out_rp = np.empty(int(N) + 1, np.int64)
    _check(lib.oracle_symmetrize(_p(rp), _p(ci), _p(ww), int(N), _p(out_rp), None, None, 0),
           "symmetrize")
    nnz = int(out_rp[-1])
    out_ci = np.empty(max(nnz, 1), np.int32)
    out_w = np.empty(max(nnz, 1), np.float64)
    _check(lib.oracle_symmetrize(_p(rp), _p(ci), _p(ww), int(N), _p(out_rp), _p(out_ci), _p(out_w),
                                 nnz), "symmetrize")
    return out_rp, out_ci[:nnz], out_w[:nnz]
