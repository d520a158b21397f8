"""Thin ctypes binding of libfkt.so (include/fkt.h).

Argument marshalling only: every step of the MVM runs in the library's CUDA
kernels.  The module-level functions carry the C names (``fkt_plan``,
``fkt_mvm``, ...) and take torch CUDA tensors; ``Plan`` wraps them.  If the
library is missing this module raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfkt.so")

FKT_OK, FKT_ERR_INVALID_ARG, FKT_ERR_CUDA, FKT_ERR_OOM = 0, 1, 2, 3
FKT_ERR_NOT_CONVERGED, FKT_ERR_TIMEOUT, FKT_ERR_UNSUPPORTED, FKT_ERR_INTERNAL = 4, 5, 6, 7
FKT_ERR_SCRATCH_LIMIT = 8

KERNELS = {"gaussian": 0, "exponential": 1, "matern32": 2, "matern52": 3, "cauchy": 4, "ratquad": 5, "laplace": 6}

# Every entry point declared in include/fkt.h.
EXPORTS = ["fkt_plan", "fkt_mvm", "fkt_mvm_host", "fkt_dense_mvm", "fkt_set_option", "fkt_plan_stats",
           "fkt_plan_tree", "fkt_plan_lists", "fkt_destroy", "fkt_error_string", "fkt_mvm_noalloc",
           "fkt_check", "fkt_precond_setup", "fkt_precond_apply", "fkt_solve", "fkt_solve_f64", "fkt_batch_plan", "fkt_batch_mvm",
           "fkt_batch_set_option", "fkt_batch_info", "fkt_batch_check", "fkt_batch_destroy", "fkt_autotune_leaf",
           "fkt_precond_learn", "fkt_learn_params", "fkt_learn_eval", "fkt_learn_teacher", "fkt_spectral_sample",
           "fkt_shard_partition", "fkt_shard_block_work", "fkt_shard_set", "fkt_shard_info", "fkt_mvm_shard_begin",
           "fkt_mvm_shard_end", "fkt_probe_pipe_rate", "fkt_batch_autotune"]


class FktError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {lib().fkt_error_string(status).decode()} (status {status})")


class fkt_kernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("lengthscale", ctypes.c_double), ("alpha", ctypes.c_double),
                ("scale", ctypes.c_double)]


class fkt_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("used_fallback", ctypes.c_int),
                ("pad", ctypes.c_int), ("rel_residual", ctypes.c_double), ("true_rel_residual", ctypes.c_double)]


class fkt_learn_opts(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int), ("hidden", ctypes.c_int), ("steps", ctypes.c_int), ("lr", ctypes.c_float),
                ("train_blocks", ctypes.c_int), ("seed", ctypes.c_int), ("install_teacher", ctypes.c_int)]


class fkt_learn_info(ctypes.Structure):
    _fields_ = [("nparams", ctypes.c_int), ("ntrain", ctypes.c_int), ("loss_initial", ctypes.c_double),
                ("loss_final", ctypes.c_double), ("train_ms", ctypes.c_double)]


class fkt_problem(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("N", ctypes.c_int64), ("kernel", fkt_kernel)]


class fkt_stats(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("d", ctypes.c_int32), ("p", ctypes.c_int32), ("nterms", ctypes.c_int32),
                ("leaf_size", ctypes.c_int32), ("depth", ctypes.c_int32), ("nodes", ctypes.c_int64),
                ("leaves", ctypes.c_int64), ("target_blocks", ctypes.c_int64), ("far_entries", ctypes.c_int64),
                ("near_entries", ctypes.c_int64), ("masks", ctypes.c_int64), ("far_pairs", ctypes.c_int64),
                ("near_pairs", ctypes.c_int64), ("s2m_pairs", ctypes.c_int64), ("s2m_nodes", ctypes.c_int64),
                ("plan_ms", ctypes.c_double), ("last_near_ms", ctypes.c_double), ("last_far_ms", ctypes.c_double),
                ("last_s2m_ms", ctypes.c_double), ("last_total_ms", ctypes.c_double),
                ("coarse_columns", ctypes.c_int32), ("coarse_dropped", ctypes.c_int32)]


_LIB = None


def lib() -> ctypes.CDLL:
    """Load libfkt.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libfkt.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    L.fkt_plan.argtypes = [vp, i64, ctypes.c_int, fkt_kernel, ctypes.c_int, ctypes.c_int, ctypes.c_double, vp,
                           ctypes.POINTER(vp)]
    L.fkt_mvm.argtypes = [vp, vp, vp, ctypes.c_int]
    L.fkt_mvm_host.argtypes = [vp, vp, vp, ctypes.c_int]
    L.fkt_mvm_noalloc.argtypes = [vp, vp, vp, ctypes.c_int]
    L.fkt_dense_mvm.argtypes = [vp, vp, vp, ctypes.c_int]
    L.fkt_set_option.argtypes = [vp, ctypes.c_char_p, ctypes.c_char_p]
    L.fkt_plan_stats.argtypes = [vp, ctypes.POINTER(fkt_stats)]
    L.fkt_plan_tree.argtypes = [vp] + [vp] * 8
    L.fkt_plan_lists.argtypes = [vp] + [vp] * 8
    L.fkt_check.argtypes = [vp]
    L.fkt_precond_learn.argtypes = [vp, ctypes.c_double, ctypes.POINTER(fkt_learn_opts), ctypes.POINTER(fkt_learn_info)]
    L.fkt_learn_params.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int)]
    L.fkt_learn_eval.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double), vp]
    L.fkt_learn_teacher.argtypes = [vp, vp, vp]
    L.fkt_batch_plan.argtypes = [ctypes.c_int, ctypes.POINTER(fkt_problem), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, vp, ctypes.POINTER(vp)]
    L.fkt_batch_mvm.argtypes = [vp, vp, vp, ctypes.c_int]
    L.fkt_batch_set_option.argtypes = [vp, ctypes.c_char_p, ctypes.c_char_p]
    L.fkt_batch_info.argtypes = [vp, vp, vp, ctypes.POINTER(fkt_stats)]
    L.fkt_batch_check.argtypes = [vp]
    L.fkt_batch_autotune.argtypes = [vp, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]
    L.fkt_batch_destroy.argtypes = [vp]
    L.fkt_batch_destroy.restype = None
    L.fkt_autotune_leaf.argtypes = [vp, i64, ctypes.c_int, fkt_kernel, ctypes.c_int, ctypes.c_double, ctypes.c_int, vp,
                                    ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.fkt_precond_setup.argtypes = [vp, ctypes.c_double]
    L.fkt_precond_apply.argtypes = [vp, vp, vp, ctypes.c_int]
    L.fkt_solve.argtypes = [vp, ctypes.c_double, vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                            ctypes.POINTER(fkt_solve_info)]
    L.fkt_solve_f64.argtypes = L.fkt_solve.argtypes
    L.fkt_spectral_sample.argtypes = [fkt_kernel, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, vp, vp]
    L.fkt_shard_partition.argtypes = [i64, vp, ctypes.c_int, vp]
    L.fkt_shard_block_work.argtypes = [vp, vp]
    L.fkt_shard_set.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.fkt_shard_info.argtypes = [vp, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int64)] * 5
    L.fkt_mvm_shard_begin.argtypes = [vp, vp, vp, ctypes.c_int]
    L.fkt_mvm_shard_end.argtypes = [vp, vp, vp, ctypes.c_int]
    L.fkt_probe_pipe_rate.argtypes = [ctypes.c_int, i64, ctypes.POINTER(ctypes.c_double)]
    L.fkt_destroy.argtypes = [vp]
    L.fkt_destroy.restype = None
    L.fkt_error_string.argtypes = [ctypes.c_int]
    L.fkt_error_string.restype = ctypes.c_char_p
    for name in EXPORTS:
        if not hasattr(L, name):
            raise RuntimeError(f"libfkt.so lacks {name}")
    _LIB = L
    return L


def _check(status: int, where: str):
    if status != FKT_OK:
        raise FktError(status, where)


def _ptr(a) -> ctypes.c_void_p:
    if a is None:
        return ctypes.c_void_p(0)
    if isinstance(a, np.ndarray):
        return ctypes.c_void_p(a.ctypes.data)
    return ctypes.c_void_p(a.data_ptr())


def _stream_ptr(stream) -> ctypes.c_void_p:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_kernel(kernel: str, lengthscale: float = 1.0, alpha: float = 1.0, scale: float = 1.0) -> fkt_kernel:
    return fkt_kernel(KERNELS[kernel], float(lengthscale), float(alpha), float(scale))


# ---------------------------------------------------------------- C names
def fkt_plan(points, kernel: fkt_kernel, p: int, leaf_size: int, theta: float, stream=None) -> ctypes.c_void_p:
    """points: CUDA float32 tensor [N][d] (contiguous)."""
    N, d = points.shape
    h = ctypes.c_void_p()
    _check(lib().fkt_plan(_ptr(points), N, d, kernel, p, leaf_size, float(theta), _stream_ptr(stream),
                          ctypes.byref(h)), "fkt_plan")
    return h


def fkt_mvm(plan, w, y, nrhs: int):
    _check(lib().fkt_mvm(plan, _ptr(w), _ptr(y), nrhs), "fkt_mvm")


def fkt_mvm_noalloc(plan, w, y, nrhs: int):
    """fkt_mvm with its work buffers in the library's fixed device scratch (no allocation)."""
    _check(lib().fkt_mvm_noalloc(plan, _ptr(w), _ptr(y), nrhs), "fkt_mvm_noalloc")


def fkt_mvm_host(plan, w_host, y_host, nrhs: int):
    _check(lib().fkt_mvm_host(plan, _ptr(w_host), _ptr(y_host), nrhs), "fkt_mvm_host")


def fkt_dense_mvm(plan, w, y, nrhs: int):
    _check(lib().fkt_dense_mvm(plan, _ptr(w), _ptr(y), nrhs), "fkt_dense_mvm")


def fkt_set_option(plan, key: str, value: str):
    _check(lib().fkt_set_option(plan, key.encode(), value.encode()), "fkt_set_option")


def fkt_plan_stats(plan) -> dict:
    s = fkt_stats()
    _check(lib().fkt_plan_stats(plan, ctypes.byref(s)), "fkt_plan_stats")
    return {k: getattr(s, k) for k, _ in fkt_stats._fields_}


def fkt_precond_setup(plan, sigma2: float):
    _check(lib().fkt_precond_setup(plan, float(sigma2)), "fkt_precond_setup")


def fkt_precond_apply(plan, r, z, nrhs: int):
    _check(lib().fkt_precond_apply(plan, _ptr(r), _ptr(z), nrhs), "fkt_precond_apply")


def fkt_solve(plan, sigma2: float, b, x, nrhs: int, tol: float, max_iter: int, raise_on_not_converged=True,
              f64: bool = False) -> dict:
    """fkt_solve (x float32) or fkt_solve_f64 (x float64)."""
    info = fkt_solve_info()
    fn = lib().fkt_solve_f64 if f64 else lib().fkt_solve
    st = fn(plan, float(sigma2), _ptr(b), _ptr(x), nrhs, float(tol), int(max_iter), ctypes.byref(info))
    if st != FKT_OK and not (st == FKT_ERR_NOT_CONVERGED and not raise_on_not_converged):
        raise FktError(st, "fkt_solve_f64" if f64 else "fkt_solve")
    out = {k: getattr(info, k) for k, _ in fkt_solve_info._fields_ if k != "pad"}
    out["status"] = st
    return out


def fkt_spectral_sample(kernel: fkt_kernel, d: int, R: int, seed: int = 1):
    """Random Fourier frequencies (host only): returns (omega [R][d], phase [R]) float64."""
    omega = np.zeros((R, d), np.float64)
    phase = np.zeros(R, np.float64)
    _check(lib().fkt_spectral_sample(kernel, int(d), int(R), int(seed), _ptr(omega), _ptr(phase)),
           "fkt_spectral_sample")
    return omega, phase


def fkt_shard_partition(work, nranks: int) -> np.ndarray:
    """Host only: first block of each of nranks contiguous ranges balancing work, plus nblocks."""
    w = np.ascontiguousarray(work, dtype=np.float64)
    bounds = np.zeros(nranks + 1, np.int64)
    _check(lib().fkt_shard_partition(len(w), _ptr(w), int(nranks), _ptr(bounds)), "fkt_shard_partition")
    return bounds


PIPE_OPS = {"ffma": 0, "ex2": 1, "rsqrt": 2, "sqrt": 3, "rcp": 4, "ffma2": 5}


def fkt_probe_pipe_rate(op: str, iters: int = 1 << 16) -> float:
    """Lane operations per second of one arithmetic pipe on the current device."""
    v = ctypes.c_double()
    _check(lib().fkt_probe_pipe_rate(PIPE_OPS[op], int(iters), ctypes.byref(v)), "fkt_probe_pipe_rate")
    return v.value


def fkt_check(plan):
    """Raise FktError(FKT_ERR_TIMEOUT) if a bounded device-side wait ran out since the last check."""
    _check(lib().fkt_check(plan), "fkt_check")


def fkt_destroy(plan):
    lib().fkt_destroy(plan)


def fkt_error_string(status: int) -> str:
    return lib().fkt_error_string(status).decode()


# ------------------------------------------------------------- convenience
class Plan:
    """An FKT plan over fixed points: ``Plan(points, "matern32", lengthscale=0.2, p=6).mvm(w)``."""

    def __init__(self, points, kernel: str = "gaussian", lengthscale: float = 1.0, alpha: float = 1.0,
                 scale: float = 1.0, p: int = 4, leaf_size: int = 512, theta: float = 0.5, stream=None):
        import torch

        pts = points if isinstance(points, torch.Tensor) else torch.as_tensor(points)
        self.points = pts.to(device="cuda", dtype=torch.float32).contiguous()
        self.N, self.d = self.points.shape
        self.kernel = make_kernel(kernel, lengthscale, alpha, scale)
        self.p, self.leaf_size, self.theta = p, leaf_size, theta
        self.stream = stream
        self.h = fkt_plan(self.points, self.kernel, p, leaf_size, theta, stream)

    def close(self):
        if getattr(self, "h", None):
            fkt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _io(self, w, out):
        import torch

        w2 = w if w.dim() == 2 else w[None]
        w2 = w2.to(device="cuda", dtype=torch.float32).contiguous()
        if w2.shape[1] != self.N:
            raise ValueError(f"w has {w2.shape[1]} points, plan has {self.N}")
        y = out if out is not None else torch.empty_like(w2)
        return w2, y

    def mvm(self, w, out=None):
        """y = Ktilde w for w of shape [N] or [nrhs][N] (CUDA float32)."""
        w2, y = self._io(w, out)
        fkt_mvm(self.h, w2, y, w2.shape[0])
        return y if w.dim() == 2 else y[0]

    def dense(self, w, out=None):
        """Exact O(N^2) product on the GPU (float32)."""
        w2, y = self._io(w, out)
        fkt_dense_mvm(self.h, w2, y, w2.shape[0])
        return y if w.dim() == 2 else y[0]

    def mvm_host(self, w_host: np.ndarray, y_host: np.ndarray | None = None) -> np.ndarray:
        """Host buffers in and out: the call copies to and from the device itself."""
        w2 = np.ascontiguousarray(np.atleast_2d(w_host), dtype=np.float32)
        y = y_host if y_host is not None else np.empty_like(w2)
        fkt_mvm_host(self.h, w2, y, w2.shape[0])
        return y

    def set_option(self, key: str, value: str):
        fkt_set_option(self.h, key, value)

    def stats(self) -> dict:
        return fkt_plan_stats(self.h)

    def check(self):
        fkt_check(self.h)

    def solve(self, sigma2: float, b, tol: float = 1e-6, max_iter: int = 1000, raise_on_not_converged=True,
              f64: bool = False):
        """x with (Ktilde + sigma2 I) x = b by preconditioned CG; returns (x, info dict).
        f64: x in float64 (fkt_solve_f64), otherwise float32."""
        import torch

        b2 = b if b.dim() == 2 else b[None]
        b2 = b2.to(device="cuda", dtype=torch.float32).contiguous()
        x = torch.empty(b2.shape, dtype=torch.float64 if f64 else torch.float32, device=b2.device)
        info = fkt_solve(self.h, sigma2, b2, x, b2.shape[0], tol, max_iter, raise_on_not_converged, f64)
        return (x if b.dim() == 2 else x[0]), info

    def learn_precond(self, sigma2: float, rank=8, hidden=32, steps=300, lr=3e-3, train_blocks=512, seed=1,
                      install_teacher=False) -> dict:
        """Train the low-rank correction of the block-Jacobi preconditioner on the GPU and install it."""
        o = fkt_learn_opts(rank, hidden, steps, lr, train_blocks, seed, int(install_teacher))
        info = fkt_learn_info()
        _check(lib().fkt_precond_learn(self.h, float(sigma2), ctypes.byref(o), ctypes.byref(info)), "fkt_precond_learn")
        return {k: getattr(info, k) for k, _ in fkt_learn_info._fields_}

    def learn_params(self) -> np.ndarray:
        n = ctypes.c_int()
        _check(lib().fkt_learn_params(self.h, None, ctypes.byref(n)), "fkt_learn_params")
        out = np.zeros(n.value, np.float32)
        _check(lib().fkt_learn_params(self.h, _ptr(out), ctypes.byref(n)), "fkt_learn_params")
        return out

    def learn_eval(self, params: np.ndarray):
        """(loss, gradient) of the learning objective at params, computed by the GPU kernels."""
        params = np.ascontiguousarray(params, dtype=np.float32)
        loss = ctypes.c_double()
        grad = np.zeros_like(params)
        _check(lib().fkt_learn_eval(self.h, _ptr(params), ctypes.byref(loss), _ptr(grad)), "fkt_learn_eval")
        return loss.value, grad

    def learn_teacher(self, ntrain: int):
        blocks = np.zeros(ntrain, np.int64)
        D = np.zeros((ntrain, 128, 128), np.float32)
        _check(lib().fkt_learn_teacher(self.h, _ptr(blocks), _ptr(D)), "fkt_learn_teacher")
        return blocks, D

    def precond(self, sigma2: float, r):
        """z = M^{-1} r with the block-Jacobi preconditioner for sigma2."""
        import torch

        fkt_precond_setup(self.h, sigma2)
        r2 = (r if r.dim() == 2 else r[None]).to(device="cuda", dtype=torch.float32).contiguous()
        z = torch.empty_like(r2)
        fkt_precond_apply(self.h, r2, z, r2.shape[0])
        return z if r.dim() == 2 else z[0]

    # ---- target-sharded product (one rank's share; the caller sums mult over the ranks) ----
    def shard_set(self, nranks: int, rank: int) -> dict:
        _check(lib().fkt_shard_set(self.h, int(nranks), int(rank)), "fkt_shard_set")
        return self.shard_info(1)

    def shard_info(self, nrhs: int) -> dict:
        v = [ctypes.c_int64() for _ in range(5)]
        _check(lib().fkt_shard_info(self.h, int(nrhs), *[ctypes.byref(x) for x in v]), "fkt_shard_info")
        return dict(zip(("block_lo", "block_hi", "target_lo", "target_hi", "mult_floats"), [x.value for x in v]))

    def block_work(self) -> np.ndarray:
        w = np.zeros(self.stats()["target_blocks"], np.float64)
        _check(lib().fkt_shard_block_work(self.h, _ptr(w)), "fkt_shard_block_work")
        return w

    def shard_begin(self, w, mult=None):
        """Phase 1: this rank's partial multipoles (a new or given float32 device tensor)."""
        import torch

        w2 = (w if w.dim() == 2 else w[None]).contiguous()
        n = self.shard_info(w2.shape[0])["mult_floats"]
        if mult is None:
            mult = torch.empty(n, dtype=torch.float32, device=w2.device)
        _check(lib().fkt_mvm_shard_begin(self.h, _ptr(w2), _ptr(mult), w2.shape[0]), "fkt_mvm_shard_begin")
        return mult

    def shard_end(self, mult, y):
        """Phase 2 after the multipoles were summed over the ranks: y ([nrhs][N]) gets this rank's targets."""
        _check(lib().fkt_mvm_shard_end(self.h, _ptr(mult), _ptr(y), y.shape[0] if y.dim() == 2 else 1),
               "fkt_mvm_shard_end")
        return y

    def tree(self) -> dict:
        s = self.stats()
        n, N, d = s["nodes"], self.N, self.d
        out = dict(perm=np.zeros(N, np.int64), begin=np.zeros(n, np.int64), end=np.zeros(n, np.int64),
                   level=np.zeros(n, np.int32), leaf=np.zeros(n, np.int32), child=np.zeros((n, 2), np.int64),
                   centre=np.zeros((n, d)), rho2=np.zeros(n))
        _check(lib().fkt_plan_tree(self.h, *[_ptr(out[k]) for k in
                                             ("perm", "begin", "end", "level", "leaf", "child", "centre", "rho2")]),
               "fkt_plan_tree")
        out["leaf"] = out["leaf"].astype(bool)
        return out

    def lists(self) -> dict:
        s = self.stats()
        nb, nf, nn, nm = s["target_blocks"], s["far_entries"], s["near_entries"], s["masks"]
        out = dict(block_range=np.zeros((nb, 2), np.int64), far_off=np.zeros(nb + 1, np.int64),
                   far_node=np.zeros(nf, np.int32), far_mask=np.zeros(nf, np.int32),
                   near_off=np.zeros(nb + 1, np.int64), near_leaf=np.zeros(nn, np.int32),
                   near_mask=np.zeros(nn, np.int32), masks=np.zeros((max(nm, 1), 4), np.uint32))
        _check(lib().fkt_plan_lists(self.h, *[_ptr(out[k]) for k in
                                              ("block_range", "far_off", "far_node", "far_mask", "near_off",
                                               "near_leaf", "near_mask", "masks")]), "fkt_plan_lists")
        return out

    def target_sets(self, lists: dict | None = None):
        """Per sorted target position: (far node set, near leaf set), decoded from the block lists."""
        L = lists or self.lists()
        far, near = {}, {}
        for b, (lo, hi) in enumerate(L["block_range"]):
            for t in range(lo, hi):
                far[t], near[t] = [], []
            for kind, off, ids, msk, dst in (("far", L["far_off"], L["far_node"], L["far_mask"], far),
                                             ("near", L["near_off"], L["near_leaf"], L["near_mask"], near)):
                for e in range(off[b], off[b + 1]):
                    m = msk[e]
                    for t in range(lo, hi):
                        i = t - lo
                        if m < 0 or (L["masks"][m][i >> 5] >> np.uint32(i & 31)) & np.uint32(1):
                            dst[t].append(int(ids[e]))
        return far, near


def fkt_autotune_leaf(points, kernel: fkt_kernel, p: int, theta: float, nrhs: int = 8, candidates=(64, 128, 256, 512),
                      stream=None):
    """(best leaf size, its MVM time in ms) among the candidates, timed on the device."""
    N, d = points.shape
    cand = np.asarray(candidates, dtype=np.int32)
    best = ctypes.c_int()
    ms = ctypes.c_double()
    _check(lib().fkt_autotune_leaf(_ptr(points), N, d, kernel, p, float(theta), nrhs, _ptr(cand), len(cand),
                                   _stream_ptr(stream), ctypes.byref(best), ctypes.byref(ms)), "fkt_autotune_leaf")
    return best.value, ms.value


class Batch:
    """Independent problems [(points [N_i][d], kernel, lengthscale, alpha, scale), ...] sharing d, p, theta."""

    def __init__(self, problems, p: int = 4, leaf_size: int = 512, theta: float = 0.5, stream=None):
        import torch

        self.points = [torch.as_tensor(x).to(device="cuda", dtype=torch.float32).contiguous() for x, *_ in problems]
        arr = (fkt_problem * len(problems))()
        for i, (x, *k) in enumerate(problems):
            arr[i] = fkt_problem(self.points[i].data_ptr(), self.points[i].shape[0], make_kernel(*k))
        d = self.points[0].shape[1]
        self.h = ctypes.c_void_p()
        _check(lib().fkt_batch_plan(len(problems), arr, d, p, leaf_size, float(theta), _stream_ptr(stream),
                                    ctypes.byref(self.h)), "fkt_batch_plan")
        n = len(problems)
        self.offsets = np.zeros(n + 1, np.int64)
        self.leaf_sizes = np.zeros(n, np.int32)
        st = fkt_stats()
        _check(lib().fkt_batch_info(self.h, _ptr(self.offsets), _ptr(self.leaf_sizes), ctypes.byref(st)),
               "fkt_batch_info")
        self.totals = {k: getattr(st, k) for k, _ in fkt_stats._fields_}
        self.N = int(self.offsets[-1])

    def mvm(self, w, out=None):
        """w: CUDA float32 [nrhs][N_total]; returns y of the same shape."""
        y = out if out is not None else w.new_empty(w.shape)
        _check(lib().fkt_batch_mvm(self.h, _ptr(w), _ptr(y), w.shape[0]), "fkt_batch_mvm")
        return y

    def set_option(self, key: str, value: str):
        _check(lib().fkt_batch_set_option(self.h, key.encode(), value.encode()), "fkt_batch_set_option")

    def check(self):
        _check(lib().fkt_batch_check(self.h), "fkt_batch_check")

    def autotune(self, nrhs: int) -> str:
        """Pick the fastest kernel variants for nrhs right-hand sides (fkt_batch_autotune)."""
        buf = ctypes.create_string_buffer(256)
        _check(lib().fkt_batch_autotune(self.h, int(nrhs), buf, len(buf)), "fkt_batch_autotune")
        return buf.value.decode()

    def close(self):
        if getattr(self, "h", None):
            lib().fkt_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
