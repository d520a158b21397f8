"""Build and ctypes wrapper of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use this.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from functools import lru_cache

import numpy as np

from . import tables

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fkt_oracle.c")
_SO = os.path.join(_HERE, "liborc_fkt.so")
_lock = threading.Lock()

KERNELS = {
    "gaussian": 0,
    "exponential": 1,
    "matern32": 2,
    "matern52": 3,
    "cauchy": 4,
    "ratquad": 5,
    "laplace": 6,
}


def build(force: bool = False) -> str:
    """Compile fkt_oracle.c with gcc (FP64, OpenMP, no FP contraction)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                   "-fno-fast-math", "-o", _SO + ".tmp", _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(_SO + ".tmp", _SO)
    return _SO


_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_i64p = ctypes.POINTER(ctypes.c_int64)


@lru_cache(maxsize=1)
def lib() -> ctypes.CDLL:
    L = ctypes.CDLL(build())
    L.orc_basis_new.restype = ctypes.c_void_p
    L.orc_basis_new.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_int), _dp]
    L.orc_basis_free.argtypes = [ctypes.c_void_p]
    L.orc_basis_nterms.argtypes = [ctypes.c_void_p]
    L.orc_harmonics.argtypes = [ctypes.c_void_p, _dp, _dp]
    L.orc_expansion_pairs.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, ctypes.c_int64, _dp]
    L.orc_expansion_pairs_gegenbauer.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_int64, _dp]
    L.orc_kernel_value.restype = ctypes.c_double
    L.orc_kernel_value.argtypes = [_dp, ctypes.c_double]
    L.orc_kernel_derivs.argtypes = [_dp, ctypes.c_double, ctypes.c_int, _dp]
    L.orc_gegenbauer.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double, _dp]
    L.orc_dense.argtypes = [_fp, ctypes.c_int64, ctypes.c_int, _dp, _dp, ctypes.c_int, _i64p, ctypes.c_int64, _dp]
    L.orc_fkt_new.restype = ctypes.c_void_p
    L.orc_fkt_new.argtypes = [_fp, ctypes.c_int64, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p]
    L.orc_fkt_free.argtypes = [ctypes.c_void_p]
    L.orc_fkt_num_nodes.restype = ctypes.c_int64
    L.orc_fkt_num_nodes.argtypes = [ctypes.c_void_p]
    L.orc_fkt_nodes.argtypes = [ctypes.c_void_p, _i64p, _i64p, ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_int32), _i64p, _dp, _dp]
    L.orc_fkt_perm.argtypes = [ctypes.c_void_p, _i64p, ctypes.POINTER(ctypes.c_uint64), _dp]
    L.orc_fkt_s2m.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int]
    L.orc_fkt_eval.argtypes = [ctypes.c_void_p, _i64p, ctypes.c_int64, _dp]
    L.orc_fkt_target_lists.argtypes = [ctypes.c_void_p, ctypes.c_int64, _i64p, _i64p, _i64p, _i64p]
    L.orc_num_threads.restype = ctypes.c_int
    L.orc_fkt_get_multipoles.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int64]
    L.orc_fkt_set_multipoles.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int64]
    return L


def _p(a, t):
    return a.ctypes.data_as(t)


def kparams(kernel: str, ell: float = 1.0, alpha: float = 1.0, scale: float = 1.0) -> np.ndarray:
    return np.array([KERNELS[kernel], ell, alpha, scale], dtype=np.float64)


def kernel_value(kp: np.ndarray, r: float) -> float:
    return lib().orc_kernel_value(_p(kp, _dp), float(r))


def kernel_derivs(kp: np.ndarray, r: float, n: int) -> np.ndarray:
    out = np.zeros(n + 1)
    lib().orc_kernel_derivs(_p(kp, _dp), float(r), int(n), _p(out, _dp))
    return out


def gegenbauer(alpha: float, n: int, x: float) -> np.ndarray:
    out = np.zeros(n + 1)
    lib().orc_gegenbauer(float(alpha), int(n), float(x), _p(out, _dp))
    return out


def zonal_points(d: int, p: int, seed: int = 12345):
    """Unit vectors v_{k,i} for the zonal harmonic basis of each degree k <= p.

    For degree k, D_k = |H_k| points are picked greedily (pivoted Cholesky of the
    Gram matrix C_k^alpha(v_i . v_j), T_k(v_i . v_j) for d = 2) from a seeded random pool so the Gram
    matrix is well conditioned.  Any points in general position give a valid
    basis (Sec. A.1 addition theorem); the choice only affects rounding.
    """
    from scipy.special import eval_chebyt, eval_gegenbauer

    rng = np.random.default_rng(seed)
    a = d / 2.0 - 1.0
    Dk = [tables.harmonic_dim(k, d) for k in range(p + 1)]
    blocks = []
    for k in range(p + 1):
        npool = 4 * Dk[k] + 16
        pool = rng.normal(size=(npool, d))
        pool /= np.linalg.norm(pool, axis=1, keepdims=True)
        cosg = np.clip(pool @ pool.T, -1.0, 1.0)
        G = eval_chebyt(k, cosg) if d == 2 else eval_gegenbauer(k, a, cosg)  # zonal function of degree k
        diag = G.diagonal().copy()
        chosen = []
        Lrows = np.zeros((Dk[k], npool))
        for t in range(Dk[k]):
            i = int(np.argmax(diag))
            chosen.append(i)
            row = (G[i] - Lrows[:t, i] @ Lrows[:t]) / np.sqrt(diag[i])
            Lrows[t] = row
            diag = diag - row * row
            diag[chosen] = -np.inf
        blocks.append(pool[chosen])
    return np.ascontiguousarray(np.concatenate(blocks, axis=0)), Dk


class Basis:
    """Zonal-Gram harmonic basis plus Tbar table for dimension d, order p."""

    def __init__(self, d: int, p: int, seed: int = 12345):
        self.d, self.p = d, p
        self.T = np.ascontiguousarray(tables.tbar_array(p, d))
        self.v, Dk = zonal_points(d, p, seed)
        self.Dk = np.array(Dk, dtype=np.int32)
        h = lib().orc_basis_new(d, p, _p(self.T, _dp), self.Dk.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                _p(self.v, _dp))
        if not h:
            raise RuntimeError("oracle basis: Gram matrix not positive definite")
        self.h = ctypes.c_void_p(h)
        self.nterms = lib().orc_basis_nterms(self.h)

    def __del__(self):
        try:
            lib().orc_basis_free(self.h)
        except Exception:
            pass

    def harmonics(self, u: np.ndarray) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.zeros(int(self.Dk.sum()))
        lib().orc_harmonics(self.h, _p(u, _dp), _p(out, _dp))
        return out

    def expansion(self, kp, X, XP) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float64)
        XP = np.ascontiguousarray(XP, dtype=np.float64)
        out = np.zeros(len(X))
        lib().orc_expansion_pairs(self.h, _p(kp, _dp), _p(X, _dp), _p(XP, _dp), len(X), _p(out, _dp))
        return out


def expansion_gegenbauer(d, p, kp, X, XP) -> np.ndarray:
    T = np.ascontiguousarray(tables.tbar_array(p, d))
    X = np.ascontiguousarray(X, dtype=np.float64)
    XP = np.ascontiguousarray(XP, dtype=np.float64)
    out = np.zeros(len(X))
    lib().orc_expansion_pairs_gegenbauer(d, p, _p(T, _dp), _p(kp, _dp), _p(X, _dp), _p(XP, _dp), len(X),
                                         _p(out, _dp))
    return out


def dense(points: np.ndarray, kp: np.ndarray, w: np.ndarray, targets=None) -> np.ndarray:
    """FP64 dense z = K w at the given targets. points [N][d] float32, w [nrhs][N]; out [nrhs][nt]."""
    X = np.ascontiguousarray(points, dtype=np.float32)
    N, d = X.shape
    W = np.ascontiguousarray(np.atleast_2d(w), dtype=np.float64)
    nrhs = W.shape[0]
    if targets is None:
        targets = np.arange(N, dtype=np.int64)
    T = np.ascontiguousarray(targets, dtype=np.int64)
    out = np.zeros((nrhs, len(T)))
    lib().orc_dense(_p(X, _fp), N, d, _p(kp, _dp), _p(W, _dp), nrhs, _p(T, _i64p), len(T), _p(out, _dp))
    return out


class FKT:
    """Step-by-step FP64 FKT (Algorithm 1) with per-target traversal."""

    def __init__(self, points, kp, p, leaf_size, theta, basis: Basis | None = None):
        self.X = np.ascontiguousarray(points, dtype=np.float32)
        self.N, self.d = self.X.shape
        self.kp = np.ascontiguousarray(kp, dtype=np.float64)
        self.basis = basis if basis is not None else Basis(self.d, p)
        h = lib().orc_fkt_new(_p(self.X, _fp), self.N, self.d, _p(self.kp, _dp), p, leaf_size, float(theta),
                              self.basis.h)
        if not h:
            raise ValueError("oracle FKT: invalid arguments")
        self.h = ctypes.c_void_p(h)
        self.p, self.leaf_size, self.theta = p, leaf_size, theta

    def __del__(self):
        try:
            lib().orc_fkt_free(self.h)
        except Exception:
            pass

    def tree(self):
        n = lib().orc_fkt_num_nodes(self.h)
        begin = np.zeros(n, np.int64)
        end = np.zeros(n, np.int64)
        level = np.zeros(n, np.int32)
        leaf = np.zeros(n, np.int32)
        child = np.zeros((n, 2), np.int64)
        centre = np.zeros((n, self.d))
        rho2 = np.zeros(n)
        lib().orc_fkt_nodes(self.h, _p(begin, _i64p), _p(end, _i64p), level.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                            leaf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _p(child, _i64p), _p(centre, _dp),
                            _p(rho2, _dp))
        perm = np.zeros(self.N, np.int64)
        codes = np.zeros(self.N, np.uint64)
        loL = np.zeros(self.d + 1)
        lib().orc_fkt_perm(self.h, _p(perm, _i64p), codes.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _p(loL, _dp))
        return dict(begin=begin, end=end, level=level, leaf=leaf.astype(bool), child=child, centre=centre, rho2=rho2,
                    perm=perm, codes=codes, lo=loL[:-1], L=loL[-1])

    def mvm(self, w, targets=None) -> np.ndarray:
        W = np.ascontiguousarray(np.atleast_2d(w), dtype=np.float64)
        nrhs = W.shape[0]
        if lib().orc_fkt_s2m(self.h, _p(W, _dp), nrhs) != 0:
            raise ValueError("oracle FKT: bad nrhs")
        if targets is None:
            targets = np.arange(self.N, dtype=np.int64)
        T = np.ascontiguousarray(targets, dtype=np.int64)
        out = np.zeros((nrhs, len(T)))
        lib().orc_fkt_eval(self.h, _p(T, _i64p), len(T), _p(out, _dp))
        return out

    def s2m(self, w) -> None:
        """Multipoles of every node for weights w [nrhs][N] (orc_fkt_s2m), kept for eval()."""
        W = np.ascontiguousarray(np.atleast_2d(w), dtype=np.float64)
        if lib().orc_fkt_s2m(self.h, _p(W, _dp), W.shape[0]) != 0:
            raise ValueError("oracle FKT: bad nrhs")
        self._nrhs = W.shape[0]

    def multipoles(self) -> np.ndarray:
        n = lib().orc_fkt_num_nodes(self.h) * self._nrhs * self.basis.nterms
        out = np.zeros(n)
        if lib().orc_fkt_get_multipoles(self.h, _p(out, _dp), n) != 0:
            raise ValueError("oracle FKT: no multipoles")
        return out

    def set_multipoles(self, M: np.ndarray) -> None:
        M = np.ascontiguousarray(M, dtype=np.float64)
        if lib().orc_fkt_set_multipoles(self.h, _p(M, _dp), len(M)) != 0:
            raise ValueError("oracle FKT: multipole count mismatch")

    def eval(self, targets) -> np.ndarray:
        """z at the given original target indices with the current multipoles and weights."""
        T = np.ascontiguousarray(targets, dtype=np.int64)
        out = np.zeros((self._nrhs, len(T)))
        lib().orc_fkt_eval(self.h, _p(T, _i64p), len(T), _p(out, _dp))
        return out

    def target_lists(self, t: int):
        n = lib().orc_fkt_num_nodes(self.h)
        far = np.zeros(n, np.int64)
        near = np.zeros(n, np.int64)
        nf = np.zeros(1, np.int64)
        nn = np.zeros(1, np.int64)
        lib().orc_fkt_target_lists(self.h, int(t), _p(far, _i64p), _p(nf, _i64p), _p(near, _i64p), _p(nn, _i64p))
        return far[: nf[0]], near[: nn[0]]


def num_threads() -> int:
    return lib().orc_num_threads()
