"""Benchmark: FKT MVMs/s on one GB300.

Default workload (the headline): N = 1M, d = 3 Gaussian-mixture points, Matern-3/2 (l = 0.2), p = 6,
32 right-hand sides, in the precision form (near-field contraction on the tensor cores with TF32
hi/lo operands, far-field contraction on the tensor cores with BF16 hi/lo operands, float32 kernel
values and accumulation), with the plain float32 form (near and far on the CUDA cores) timed on the
same plan beside it, the Cauchy kernel (l = 0.05) as a second line, and the error of every form
against the float64 dense product on a 10,000-target subsample.

Other workloads (--workload): gauss20k (20k uniform points, Gaussian l = 0.1, p = 4, 1 RHS),
laplace16m (16M points half uniform / half in 100 tight clusters, Laplace 1/(4 pi r), p = 8, 4 RHS,
BF16 far field) and batch256 (256 independent problems of 2k-200k points in the unit ball, mixed
Gaussian / Laplace / rational-quadratic kernels, 8 RHS, one CUDA-graph launch) and gpsolve (the GP
solve (Ktilde + sigma2 I) x = b of fkt_solve: d = 4, 100k mixture points, Matern-5/2 l = 0.3,
sigma2 = 1e-2, 8 RHS; one step = one solve with the two-level coarse space, the solves without a
preconditioner and with block-Jacobi run once beside it).

One step = one product over all right-hand sides (all stages of Algorithm 1: permute, s2m, near
field, m2t, combine) on resident device buffers; one MVM = one right-hand side of one problem.  L2
is flushed between timed steps (a 256 MiB write outside the timed events).  Prints ONE JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload matern1m|gauss20k|laplace16m|batch256|gpsolve]
                    [--kernel matern32|cauchy] [--p P] [--theta T] [--leaf M] [--nrhs R]
                    [--far-precision bf16x3|tf32|bf16|fp32] [--near-precision tf32x3|fp32]
                    [--compare fp32|none]

--impl reference times the CPU float64 oracle (the slow reference program) on a bounded sample of
the same workload.  Multi-GPU runs are independent replicas (one plan per rank, no collective):
the value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2106_04487_gb300 import inputs  # noqa: E402

KERNELS = {"matern32": ("matern32", 0.2, 1.0, 1.0), "cauchy": ("cauchy", 0.05, 1.0, 1.0)}
PASS = 32  # right-hand sides per pass of the library

# Workloads: points, kernel (name, lengthscale, alpha, scale), order, opening parameter, leaf size,
# right-hand sides, near / far arithmetic of the headline form, weight distribution, error targets.
WORKLOADS = {
    "matern1m": dict(desc="d=3 N=1000000 gaussian-mixture(10 comps, std 0.05)", n=1_000_000,
                     points=lambda n: inputs.gaussian_mixture(n, 3, 10, 0.05), kernel=KERNELS["matern32"],
                     p=6, theta=0.375, leaf=256, nrhs=32, near="tf32x3", far="bf16x3", weights="normal",
                     err_targets=10000),
    "cauchy2d": dict(desc="d=2 N=20000 uniform square", n=20000, points=lambda n: inputs.uniform_cube(n, 2),
                     kernel=("cauchy", 0.05, 1.0, 1.0), p=4, theta=0.5, leaf=512, nrhs=1, near="fp32", far="fp32",
                     weights="normal", err_targets=20000, d=2),
    "gauss20k": dict(desc="d=3 N=20000 uniform cube", n=20000, points=lambda n: inputs.uniform_cube(n, 3),
                     kernel=("gaussian", 0.1, 1.0, 1.0), p=4, theta=0.5, leaf=512, nrhs=1, near="fp32",
                     far="fp32", weights="normal", err_targets=20000),
    "laplace16m": dict(desc="d=3 N=16000000 half uniform cube + half 100 clusters (std 0.005)", n=16_000_000,
                       points=lambda n: inputs.uniform_plus_clusters(n, 3, 100, 0.005),
                       kernel=("laplace", 1.0, 1.0, 1.0 / (4.0 * np.pi)), p=8, theta=0.5, leaf=512, nrhs=4,
                       near="fp32", far="bf16", weights="uniform", err_targets=400),
    "batch256": dict(desc="256 problems, N log-uniform [2000, 200000], unit ball, kernels gaussian l=0.1 / "
                          "laplace 1/r / ratquad alpha=1 l=0.2", n=0, points=None, kernel=None, p=4, theta=0.5,
                     leaf=0, nrhs=8, near="fp32", far="bf16x3", weights="normal", err_targets=150),
    "pipes": dict(desc="arithmetic pipe rates", n=0, points=None, kernel=None, p=0, theta=0.5, leaf=1, nrhs=1,
                  near="fp32", far="fp32", weights="normal", err_targets=0),
    "gpsolve": dict(desc="d=4 N=100000 gaussian-mixture(20 comps, std 0.05)", n=100_000,
                    points=lambda n: inputs.gaussian_mixture(n, 4, 20, 0.05), kernel=("matern52", 0.3, 1.0, 1.0),
                    p=6, theta=0.3, leaf=256, nrhs=8, near="fp32", far="fp32", weights="normal", err_targets=0),
}
BATCH_KERNELS = [("gaussian", 0.1, 1.0, 1.0), ("laplace", 1.0, 1.0, 1.0), ("ratquad", 0.2, 1.0, 1.0)]
GP_SIGMA2 = 1e-2

# DRAM bytes (read + write) per launch of a kernel from one ncu capture, keyed by kernel and
# workload (kernel, p, theta, leaf, nrhs, N); see profiles/.  Any other workload reports null.
PROFILED_TRAFFIC = {
    ("near_tc_kernel<3,matern32>", "matern32", 6, 0.375, 256, 32, 1_000_000): 2.8022e9 + 0.1303e9,
    ("far_tc2_kernel<6,bf16x3>", "matern32", 6, 0.375, 256, 32, 1_000_000): 1.4582e9 + 0.1308e9,
}

# Per-SM lane rates of GB300 used by the ALU rooflines, measured by fkt_probe_pipe_rate
# (bench.py --workload pipes; profiles/pipe_rates_gb300.md) at 2070 MHz: FP32 FMA 121 lanes/clock
# (FP32x2 FMA the same 120: packing halves the issue slots, not the pipe time), MUFU ex2 32
# lanes/clock, MUFU sqrt / rsqrt / rcp 16.  The rooflines use the nominal 128 for FP32.
FP32_LANES, MUFU_LANES = 128.0, 32.0
MUFU_CLOCKS = {"ex2": 1.0 / 32.0, "sqrt": 1.0 / 16.0, "rsqrt": 1.0 / 16.0, "rcp": 1.0 / 16.0, "lg2": 1.0 / 16.0}


def nterms(d: int, p: int) -> int:
    n = 1
    for i in range(1, d + 1):
        n = n * (p + i) // i
    return n


def near_kernel_name(kname: str, nw: int, near_precision: str = "fp32") -> str:
    if nw == 32 and near_precision == "f16x3" and kname != "laplace":
        return f"near_tc2_kernel<3,{kname}>"
    if nw == 32 and near_precision in ("tf32x3", "f16x3"):
        return f"near_tc_kernel<3,{kname}>"
    base = "near_kernel" if nw == 1 else "near_wide_kernel" if nw in (4, 8) else "near_tile_kernel"
    return f"{base}<3,{kname},{nw}>"


def far_kernel_name(p: int, far_precision: str, nrhs: int, far_kernel: str = "single", d: int = 3) -> str:
    if far_precision == "fp32":
        return f"far_kernel<{d},{p},1>" if nrhs == 1 else f"far_mr_kernel<{d},{p}>"
    if far_precision == "tf32":
        return f"far_tc_kernel<3,{p},tf32>"
    pairs_ok = p <= (6 if far_precision == "bf16x3" else 9)  # two A buffers fit 256 tensor-memory columns
    if far_kernel == "pairs" and pairs_ok:
        return f"far_tc3_kernel<{p},{far_precision}>"
    return f"far_tc2_kernel<{p},{far_precision}>"


def near_pair_cost(kernel: str, nw: int, tensor: bool = False, d: int = 3):
    """Lower bound on SM work per near-field pair for a pass of nw right-hand sides:
    (FP32-pipe lane-ops, MUFU SM-clocks per lane).

    Per pair the method needs d subtractions and |x|^2 (1 MUL + d - 1 FMA), the kernel value and one
    FMA per right-hand side.  Kernel value: Gaussian 2^-q (ex2); Matern-3/2 sqrt, 1 + u ln2 (FMA),
    2^-u (ex2), product (MUL); Cauchy / rational quadratic 1 + q (ADD), reciprocal (rcp); Laplace
    rsqrt and the r = 0 test.  MUFU rates per operation as measured (MUFU_CLOCKS).  With the
    contraction on the tensor cores (tensor=True) the per-right-hand-side FMAs leave the FP32 pipe."""
    fma = 0 if tensor else nw
    extra, mufu = {"gaussian": (0, ["ex2"]), "matern32": (2, ["sqrt", "ex2"]), "cauchy": (1, ["rcp"]),
                   "ratquad": (1, ["rcp"]), "laplace": (1, ["rsqrt"]), "exponential": (0, ["sqrt", "ex2"]),
                   "matern52": (4, ["sqrt", "ex2"])}.get(kernel, (2, ["sqrt", "ex2"]))
    return 2 * d + extra + fma, sum(MUFU_CLOCKS[m] for m in mufu)


def far_pair_ops(p: int, diag: bool = False, d: int = 3) -> int:
    """FP32 lane-ops the method needs per (target, far node) pair in d = 3 before the contraction:
    distance and direction (~10), kernel derivatives J_m, m <= p (~3 per order), the radial sums
    R_kj = sum_m That_kjm J_m (j + 1 FMAs per (k, j)), the powers (s/r)^j and G = (s/r)^j R (p + pairs),
    the (p+1)^2 harmonics by recurrence (~3 each) and the products Y_kh G_kj (one per term).
    diag: the radially compressed expansion of 1/r (only j = k), (p+1)^2 terms.  d = 2: distance and
    direction ~7, the 2p circular harmonics by the complex recurrence (~2 each)."""
    pairs = [(k, j) for k in range(p + 1) for j in range(k, p + 1, 2) if not diag or j == k]
    nt = (p + 1) ** 2 if diag else nterms(d, p)
    if d == 2:
        return 7 + 3 * (p + 1) + sum(j + 1 for _, j in pairs) + p + len(pairs) + 4 * p + nt
    return 10 + 3 * (p + 1) + sum(j + 1 for _, j in pairs) + p + len(pairs) + 3 * (p + 1) ** 2 + nt


def launches_per_step(nrhs: int, far_precision: str) -> int:
    """Kernels the library launches per fkt_mvm.  Per pass of up to 32 right-hand sides: permute
    and near field once; s2m + s2m_reduce per group of 8 (1 for a single right-hand side on the
    float32 path); the float32 far field once per group, the tensor-core far field (pack + far)
    once per pass; unpermute once."""
    total = 0
    for r0 in range(0, nrhs, PASS):
        npass = min(PASS, nrhs - r0)
        group = 1 if (nrhs == 1 and far_precision == "fp32") else 8
        groups = (npass + group - 1) // group
        total += 3 + 2 * groups + (groups if far_precision == "fp32" else 2)
    return total


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="matern1m", choices=list(WORKLOADS))
    ap.add_argument("--kernel", default=None, choices=list(KERNELS),
                    help="kernel of the matern1m workload (default matern32)")
    ap.add_argument("--p", type=int, default=None)
    ap.add_argument("--theta", type=float, default=None)
    ap.add_argument("--leaf", type=int, default=None)
    ap.add_argument("--nrhs", type=int, default=None)
    ap.add_argument("--far-precision", default=None, choices=["bf16x3", "tf32", "bf16", "fp32"])
    ap.add_argument("--near-precision", default=None, choices=["tf32x3", "f16x3", "fp32"],
                    help="near-field contraction of 32-wide passes: tensor cores (TF32 hi/lo) or CUDA cores")
    ap.add_argument("--far-kernel", default="single", choices=["pairs", "single", "held"],
                    help="tensor-core far field (d = 3, BF16 forms): two far entries per thread, one, or one "
                         "with the row held in registers until the previous entry's MMAs complete")
    ap.add_argument("--radial-compression", default="auto", choices=["auto", "off"],
                    help="drop the radial terms that vanish for the kernel (1/r in d = 3: j > k)")
    ap.add_argument("--compare", default="fp32", choices=["fp32", "none"],
                    help="plain float32 form (near and far on the CUDA cores) timed beside the headline one")
    ap.add_argument("--second-kernel", default="cauchy", choices=list(KERNELS) + ["none"],
                    help="second kernel of the matern1m workload")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--err-targets", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--coarse-rank", type=int, default=256, help="gpsolve: coarse space of the timed solves")
    ap.add_argument("--tol", type=float, default=1e-5, help="gpsolve: CG tolerance")
    ap.add_argument("--compare-iters", type=int, default=3000,
                    help="gpsolve: iteration cap of the comparison solves (no preconditioner, block-Jacobi)")
    a = ap.parse_args()
    w = WORKLOADS[a.workload]
    for key, wkey in [("p", "p"), ("theta", "theta"), ("leaf", "leaf"), ("nrhs", "nrhs"), ("far_precision", "far"),
                      ("near_precision", "near"), ("n", "n"), ("err_targets", "err_targets")]:
        if getattr(a, key) is None:
            setattr(a, key, w[wkey])
    a.kern = w["kernel"]
    a.d = w.get("d", 3)
    if a.workload == "matern1m" and a.kernel:
        a.kern = KERNELS[a.kernel]
    if a.workload != "matern1m":
        a.second_kernel = "none"
    return a


def workload_name(a, kern=None):
    if a.workload == "batch256":
        return (f"{WORKLOADS['batch256']['desc']}, p={a.p} leaf={a.leaf or 'autotuned'} theta={a.theta} nrhs={a.nrhs} "
                f"near={a.near_precision} far={a.far_precision}")
    k = kern or a.kern
    desc = WORKLOADS[a.workload]["desc"].replace(f"N={WORKLOADS[a.workload]['n']}", f"N={a.n}")
    return (f"{k[0]} l={k[1]}{' scale=1/(4pi)' if k[0] == 'laplace' and k[3] != 1.0 else ''} {desc} p={a.p} "
            f"leaf={a.leaf} theta={a.theta} nrhs={a.nrhs} near={a.near_precision} far={a.far_precision}")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The largest x over all ranks (the slowest replica's time); x itself on one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(steps: int, units_per_step: int, world: int, total_ms: float) -> float:
    """Whole-job throughput of independent replicas: the units all ranks processed over the
    slowest rank's time."""
    return steps * units_per_step * world / (total_ms / 1e3)


def time_form(obj, Wd, Yd, steps, warmup, flush, stream, stats=True):
    """Per-step CUDA-event times of obj.mvm on the launching stream, with the library's own
    per-stage events (near, far + wait, s2m) read after each step when stats is set."""
    import torch

    for _ in range(warmup):
        obj.mvm(Wd, out=Yd)
    torch.cuda.synchronize()
    step_ms, near_ms, far_ms, s2m_ms = [], [], [], []
    for _ in range(steps):
        flush.fill_(1.0)  # evict L2 between steps (outside the timed events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        obj.mvm(Wd, out=Yd)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        if stats:
            s = obj.stats()
            near_ms.append(s["last_near_ms"])
            far_ms.append(s["last_far_ms"])
            s2m_ms.append(s["last_s2m_ms"])
    torch.cuda.synchronize()
    mean = lambda v: float(np.mean(v)) if v else None  # noqa: E731
    return {"step_ms": step_ms, "near_ms": mean(near_ms), "far_ms": mean(far_ms), "s2m_ms": mean(s2m_ms)}


def rel_errs(y, z, idx):
    """Per right-hand side relative 2-norm error of y (all targets) on the sampled targets idx."""
    return [float(np.linalg.norm(y[r, idx] - z[r]) / np.linalg.norm(z[r])) for r in range(z.shape[0])]


def make_weights(a, n):
    if WORKLOADS[a.workload]["weights"] == "uniform":
        return inputs.uniform_weights(n, a.nrhs)
    return inputs.normal_weights(n, a.nrhs)


def rooflines(a, stats, head, nsm, peaks, src, kname, passes):
    """Roofline of the near and far kernels of the headline form, dominant first."""
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    nw = (1 if (a.nrhs == 1 and a.far_precision == "fp32")
          else 4 if a.nrhs <= 4 else 8 if a.nrhs <= 8 else 16 if a.nrhs <= 16 else 32)
    near_tc = nw == 32 and a.near_precision in ("tf32x3", "f16x3")
    fp32_ops, mufu_clk = near_pair_cost(kname, nw, near_tc, getattr(a, "d", 3))
    slots = max(fp32_ops / FP32_LANES, mufu_clk)  # SM clocks per pair
    peak_pairs = nsm * sm_max * 1e6 / slots
    near_pairs = stats["near_pairs"] * passes  # one launch per pass; its kernel value serves the pass
    near_ach = near_pairs / (head["near_ms"] / 1e3)
    near_name = near_kernel_name(kname, nw, a.near_precision)
    key = (a.kern[0], a.p, a.theta, a.leaf, a.nrhs, a.n)
    near_roof = {"kernel": near_name, "bound": "alu", "achieved": near_ach / 1e9, "peak": peak_pairs / 1e9,
                 "unit": "Gpair/s", "frac": near_ach / peak_pairs,
                 "traffic": PROFILED_TRAFFIC.get((near_name,) + key),
                 "traffic_unit": "bytes per launch (ncu dram__bytes_read + write)", "ms_per_step": head["near_ms"],
                 "work_per_unit": f"{fp32_ops} FP32 lane-ops + {mufu_clk:.4f} MUFU SM-clocks per (target, source) near pair"
                                  f"{'; contraction on the tensor cores' if near_tc else ''}",
                 "peak_source": f"{nsm} SMs x {sm_max:.0f} MHz / max({fp32_ops}/{FP32_LANES:.0f} FP32, "
                                f"{mufu_clk:.4f} MUFU: measured ex2 32, sqrt/rsqrt/rcp 16 lanes per SM-clock) "
                                f"SM-clocks per pair ({src} clock)"}
    roofs = [near_roof]
    if stats["far_pairs"] > 0 and head["far_ms"]:
        diag = stats.get("nterms") == (a.p + 1) ** 2 and a.p > 0 and a.kern[0] == "laplace"
        nt_used = stats.get("nterms") or nterms(getattr(a, "d", 3), a.p)
        ops = far_pair_ops(a.p, diag, getattr(a, "d", 3))
        far_peak = nsm * sm_max * 1e6 * FP32_LANES / ops
        far_ach = stats["far_pairs"] / (head["far_ms"] / 1e3)
        far_name = far_kernel_name(a.p, a.far_precision, a.nrhs, a.far_kernel, getattr(a, "d", 3))
        roof = {"kernel": far_name, "bound": "alu", "achieved": far_ach / 1e9, "peak": far_peak / 1e9,
                "unit": "Gpair/s", "frac": far_ach / far_peak, "traffic": PROFILED_TRAFFIC.get((far_name,) + key),
                "traffic_unit": "bytes per launch (ncu dram__bytes_read + write)", "ms_per_step": head["far_ms"],
                "work_per_unit": f"{ops} FP32 lane-ops per (target, far node) pair (basis), "
                                 f"+ 2 x {nt_used} x nrhs contraction flops"
                                 f"{' (radially compressed expansion: j = k terms only)' if diag else ''}",
                "peak_source": f"{nsm} SMs x {sm_max:.0f} MHz x {FP32_LANES:.0f} lanes / {ops} ({src} clock); "
                               f"far stage time on its stream"}
        if a.far_precision != "fp32":
            copies = 3 if a.far_precision == "bf16x3" else 1
            flops = 2.0 * stats["far_pairs"] * nt_used * a.nrhs * copies
            peak_tf = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0))
            if a.far_precision == "tf32":
                peak_tf *= 0.5  # nominal TF32 : BF16 dense ratio
            ach_tf = flops / (head["far_ms"] / 1e3) / 1e12
            roof["tensor"] = {"achieved_tflops": ach_tf, "peak_tflops": peak_tf, "frac": ach_tf / peak_tf,
                              "method_frac": ach_tf / copies / peak_tf,
                              "note": f"{copies} MMA products per term (hi/lo split); method_frac counts the "
                                      f"method's own contraction once; {src} sustained bf16 peak"}
        roofs.append(roof)
    roofs.sort(key=lambda r: -(r["ms_per_step"] or 0.0))
    return roofs


def run_ours(a):
    import torch

    from paper_2106_04487_gb300 import fkt

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    batch = a.workload == "batch256"
    if batch:
        sizes = inputs.batch_sizes(256, 2000, 200000)
        probs = [(inputs.unit_ball(int(n), 3, seed=100 + i), *BATCH_KERNELS[i % 3]) for i, n in enumerate(sizes)]
        obj = fkt.Batch(probs, p=a.p, leaf_size=a.leaf, theta=a.theta)
        N = obj.N
        X = None
        stats = dict(obj.totals)
    else:
        N = a.n
        X = WORKLOADS[a.workload]["points"](N)
        kname, ell, alpha, scale = a.kern
        obj = fkt.Plan(torch.from_numpy(X).cuda(), kname, lengthscale=ell, alpha=alpha, scale=scale, p=a.p,
                       leaf_size=a.leaf, theta=a.theta)
        obj.set_option("timing", "1")
        stats = obj.stats()
    W = make_weights(a, N)
    Wd = torch.from_numpy(W).cuda()
    Yd = torch.empty_like(Wd)
    obj.set_option("far_precision", a.far_precision)
    obj.set_option("near_precision", a.near_precision)
    tuned = obj.autotune(a.nrhs) if batch else None  # kernel variants of the batch (leaf sizes: leaf_size 0)
    if not batch:
        obj.set_option("far_kernel", a.far_kernel)
        obj.set_option("radial_compression", a.radial_compression)
        stats = obj.stats()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    # headline form: warm-up, then exactly K timed steps between barriers
    for _ in range(a.warmup):
        obj.mvm(Wd, out=Yd)
    barrier()
    with ClockSampler(local) as clk:
        head = time_form(obj, Wd, Yd, a.steps, 0, flush, stream, stats=not batch)
    barrier()
    obj.check()  # raises if a bounded device-side wait ran out during the timed steps
    total_ms = max_over_ranks(float(sum(head["step_ms"])), world)
    mvms_per_step = a.nrhs * (256 if batch else 1)
    value = replica_value(a.steps, mvms_per_step, world, total_ms)
    y_head = Yd.cpu().numpy().astype(np.float64)

    # the plain float32 form on the same plan
    comp = None
    if a.compare != "none" and (a.far_precision, a.near_precision) != ("fp32", "fp32"):
        obj.set_option("far_precision", "fp32")
        obj.set_option("near_precision", "fp32")
        comp = time_form(obj, Wd, Yd, max(3, a.steps // 2), 3, flush, stream, stats=not batch)
        obj.check()
        y_comp = Yd.cpu().numpy().astype(np.float64)
        obj.set_option("far_precision", a.far_precision)
        obj.set_option("near_precision", a.near_precision)

    # end to end through the host-buffer entry point (copies inside the timed region)
    Wh = torch.from_numpy(W).pin_memory()
    Yh = torch.empty_like(Wh).pin_memory()
    e2e_steps = max(3, a.steps // 2)
    if batch:  # the batched entry point takes device buffers: the copies are timed around it
        def host_call():
            Wd.copy_(Wh, non_blocking=True)
            obj.mvm(Wd, out=Yd)
            Yh.copy_(Yd, non_blocking=True)
            torch.cuda.synchronize()
    else:
        obj.set_option("timing", "0")

        def host_call():
            fkt.fkt_mvm_host(obj.h, Wh, Yh, a.nrhs)  # H2D copy, MVM, D2H copy, stream sync
    for _ in range(2):
        host_call()
    torch.cuda.synchronize()
    e2e_total = 0.0
    for _ in range(e2e_steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        host_call()
        e2e_total += time.perf_counter() - t1
    e2e_value = e2e_steps * mvms_per_step / e2e_total
    if not batch:
        obj.close()

    # second kernel of the workload (both forms, fewer steps)
    second = None
    if a.second_kernel != "none" and KERNELS[a.second_kernel] != a.kern:
        k2 = KERNELS[a.second_kernel]
        p2 = fkt.Plan(torch.from_numpy(X).cuda(), k2[0], lengthscale=k2[1], alpha=k2[2], scale=k2[3], p=a.p,
                      leaf_size=a.leaf, theta=a.theta)
        p2.set_option("timing", "1")
        second = {"kernel": f"{k2[0]} l={k2[1]}"}
        ys = {}
        forms = {f"near {a.near_precision}, far {a.far_precision}": (a.near_precision, a.far_precision)}
        if comp is not None:
            forms["near fp32, far fp32"] = ("fp32", "fp32")
        for form, (npr, fpr) in forms.items():
            p2.set_option("near_precision", npr)
            p2.set_option("far_precision", fpr)
            r = time_form(p2, Wd, Yd, max(3, a.steps // 4), 3, flush, stream)
            p2.check()
            second[form] = {"value": a.nrhs / (np.mean(r["step_ms"]) / 1e3), "ms_per_step": float(np.mean(r["step_ms"]))}
            ys[form] = Yd.cpu().numpy().astype(np.float64)
        p2.close()

    # accuracy of every form against the float64 dense product on sampled targets
    from oracle import oracle as O

    if batch:
        err_head, err_comp = [], []
        order = np.argsort(sizes)
        for i in sorted({int(order[0]), int(order[-1]), 1, 2, 100}):
            Xi, kn, ell, alpha, scale = probs[i]
            lo, hi = obj.offsets[i], obj.offsets[i + 1]
            idx = inputs.subsample(hi - lo, a.err_targets, seed=7 + i)
            zd = O.dense(Xi, O.kparams(kn, ell, alpha=alpha, scale=scale), W[:, lo:hi], idx)
            err_head += rel_errs(y_head[:, lo:hi], zd, idx)
            if comp is not None:
                err_comp += rel_errs(y_comp[:, lo:hi], zd, idx)
        err_note = f"5 problems (smallest, largest, 3 others) x {a.err_targets} targets"
    else:
        idx = inputs.subsample(N, a.err_targets)
        zd = O.dense(X, O.kparams(a.kern[0], a.kern[1], alpha=a.kern[2], scale=a.kern[3]), W, idx)
        err_head = rel_errs(y_head, zd, idx)
        if comp is not None:
            err_comp = rel_errs(y_comp, zd, idx)
        err_note = f"{len(idx)} sampled targets"
    if second is not None:
        n2 = min(2000, a.err_targets)
        idx2 = inputs.subsample(N, n2, seed=7)
        k2 = KERNELS[a.second_kernel]
        z2 = O.dense(X, O.kparams(k2[0], k2[1], alpha=k2[2], scale=k2[3]), W, idx2)
        for form, y in ys.items():
            e = rel_errs(y, z2, idx2)
            second[form]["rel_err_max"] = max(e)
            second[form]["rel_err_median"] = float(np.median(e))
        second["err_targets"] = n2

    peaks, src = load_peaks()
    clocks = clk.summary()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    passes = (a.nrhs + PASS - 1) // PASS
    roofs = [] if batch else rooflines(a, stats, head, nsm, peaks, src, a.kern[0], passes)
    if batch:
        unit_desc = "problem-MVMs/s: one MVM = one right-hand side of one of the 256 problems"
    else:
        unit_desc = "one MVM = one right-hand side"
    out = {
        "metric": metric_name(a.workload),
        "value": value,
        "unit": "MVM/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": total_ms / a.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": (f"f32 kernel values, {'tf32x3 tensor-core' if a.near_precision == 'tf32x3' and a.nrhs > 16 else 'f32'} "
                  f"near contraction, {a.far_precision} far contraction, f32 accumulate"),
        "data": "synthetic",
        "config": {"workload": workload_name(a), "unit_note": unit_desc, "l2": "flushed between steps (256 MiB write)",
                   "rel_err_max": max(err_head), "rel_err_median": float(np.median(err_head)),
                   "err_targets": err_note, "err_reference": "float64 dense oracle",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "plan_ms": stats.get("plan_ms"), "points": int(N), "near_pairs": stats["near_pairs"],
                   "far_pairs": stats["far_pairs"], "s2m_pairs": stats["s2m_pairs"],
                   "stage_ms": {"near": head["near_ms"], "far+wait": head["far_ms"], "s2m": head["s2m_ms"]}},
        "roofline": roofs[0] if roofs else None,
        "roofline_other": roofs[1:],
        "e2e": {"value": e2e_value, "unit": "MVM/s", "h2d_bytes_per_step": int(W.nbytes),
                "d2h_bytes_per_step": int(W.nbytes)},
        "gpu_launches": (None if batch else launches_per_step(a.nrhs, a.far_precision) * a.steps),
        "clocks": clocks,
    }
    if batch:
        out["gpu_launches_note"] = "one CUDA graph replay per step (near field per kernel kind, far field, s2m, permutes)"
        out["config"]["autotuned"] = {"kernel_variants": tuned,
                                      "leaf_sizes": {int(s): int((obj.leaf_sizes == s).sum()) for s in set(obj.leaf_sizes.tolist())}}
    if comp is not None:
        cv = mvms_per_step * len(comp["step_ms"]) / (sum(comp["step_ms"]) / 1e3)
        out["compare_form"] = {"form": "plain float32 (near and far on the CUDA cores)", "value": cv, "unit": "MVM/s",
                               "ms_per_step": float(np.mean(comp["step_ms"])), "rel_err_max": max(err_comp),
                               "rel_err_median": float(np.median(err_comp)),
                               "stage_ms": {"near": comp["near_ms"], "far+wait": comp["far_ms"], "s2m": comp["s2m_ms"]},
                               "speedup_of_headline": value / world / cv}
    if second is not None:
        out["second_kernel"] = second
    if rank == 0 and world == 1 and not a.no_cpu_baseline:  # the CPU baseline is a single-GPU figure
        out["cpu_baseline"] = cpu_baseline(a, X, W, probs if batch else None, obj if batch else None)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return out if rank == 0 else None


def solve_record(plan, b, pc: str, rank: int, tol: float, max_iter: int) -> dict:
    """One fkt_solve with the given first-level preconditioner and coarse rank (fkt_solve
    synchronises, so the host clock brackets the device work)."""
    plan.set_option("preconditioner", pc)
    plan.set_option("coarse_rank", str(rank))
    t0 = time.perf_counter()
    _, info = plan.solve(GP_SIGMA2, b, tol=tol, max_iter=max_iter, raise_on_not_converged=False)
    dt = time.perf_counter() - t0
    st = plan.stats()
    return {"preconditioner": pc, "coarse_rank": rank, "coarse_columns": st["coarse_columns"],
            "iterations": info["iterations"], "converged": bool(info["converged"]),
            "rel_residual": info["rel_residual"], "true_rel_residual": info["true_rel_residual"], "seconds": dt}


def run_gpsolve(a, fkt=None, torch=None):
    """GP solves per second through fkt_solve with the coarse space (timed steps), beside one solve
    without a preconditioner and one with block-Jacobi (iteration cap --compare-iters)."""
    if torch is None:
        import torch
    if fkt is None:
        from paper_2106_04487_gb300 import fkt
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    X = WORKLOADS["gpsolve"]["points"](a.n)
    kname, ell, alpha, scale = a.kern
    plan = fkt.Plan(torch.from_numpy(X).cuda(), kname, lengthscale=ell, alpha=alpha, scale=scale, p=a.p,
                    leaf_size=a.leaf, theta=a.theta)
    plan.set_option("far_precision", a.far_precision)
    plan.set_option("near_precision", a.near_precision)
    B = inputs.normal_weights(a.n, a.nrhs)
    b = torch.from_numpy(B).cuda()
    # one-time set-up of the coarse space (features, Gram, W = A Q, E): a solve of one iteration
    setup = solve_record(plan, b, "none", a.coarse_rank, a.tol, 1)
    for _ in range(a.warmup):
        solve_record(plan, b, "none", a.coarse_rank, a.tol, 5)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    steps = []
    with ClockSampler(local) as clk:
        for _ in range(a.steps):
            steps.append(solve_record(plan, b, "none", a.coarse_rank, a.tol, a.compare_iters))
    total_ms = max_over_ranks(1e3 * sum(r["seconds"] for r in steps), world)
    value = replica_value(a.steps, a.nrhs, world, total_ms)
    # end to end: b from pinned host memory in, x back to host, inside the timed region
    Bh = torch.from_numpy(B).pin_memory()
    Xh = torch.empty_like(Bh).pin_memory()
    t0 = time.perf_counter()
    bd = Bh.to("cuda", non_blocking=True)
    plan.set_option("preconditioner", "none")
    x, _ = plan.solve(GP_SIGMA2, bd, tol=a.tol, max_iter=a.compare_iters, raise_on_not_converged=False)
    Xh.copy_(x)
    e2e_s = time.perf_counter() - t0
    compare = [solve_record(plan, b, pc, 0, a.tol, a.compare_iters) for pc in ("none", "block_jacobi")]
    plan.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    if rank != 0:
        return None
    last = steps[-1]
    return {
        "metric": f"GP solves (RHS/s) to rel. residual {a.tol:g}, fkt_solve with a {a.coarse_rank}-feature coarse space",
        "value": value, "unit": "RHS/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 products, f64 CG iterates and dots", "data": "synthetic",
        "config": {"workload": workload_name(a) + f" sigma2={GP_SIGMA2} tol={a.tol}", "points": int(a.n),
                   "timed_solve": last, "coarse_setup_s": setup["seconds"],
                   "l2": "not flushed: each step is thousands of products over a working set far above L2",
                   "compare": compare},
        "roofline": None,
        "roofline_note": "the products inside the solve are the kernels the MVM workloads report rooflines for",
        "e2e": {"value": a.nrhs / e2e_s, "unit": "RHS/s", "h2d_bytes_per_step": int(B.nbytes),
                "d2h_bytes_per_step": int(B.nbytes)},
        "gpu_launches": None,
        "gpu_launches_note": "per CG iteration one fkt_mvm (launches_per_step) plus the CG and coarse-space kernels",
        "clocks": clk.summary(),
    }


# Targets per oracle step.  One oracle step = s2m over every node for all right-hand sides plus the
# per-target traversal (m2t + near field) of this many sampled targets; its work is the fraction
# targets / N of a full product.  The reference arm and the cpu_baseline leg both use this rule.
ORACLE_TARGETS = 40_000


def metric_name(workload: str) -> str:
    """The metric string, identical in both arms (the headline one is the benchmark's own)."""
    if workload == "matern1m":
        return "FKT MVMs/s at N=1M,d=3 (rel.err\u22641e-4) vs plain FP32 form; % of roofline"
    return f"FKT MVMs/s ({workload})"


class OracleRunner:
    """The float64 oracle, as it stands, on the host cores.  Its tree (its plan) is built once and
    not counted; step() runs one oracle step (see ORACLE_TARGETS) and returns its two times."""

    def __init__(self, X, kern, p, leaf, theta, nrhs):
        from oracle import oracle as O

        self.O = O
        t0 = time.perf_counter()
        self.F = O.FKT(X, O.kparams(kern[0], kern[1], alpha=kern[2], scale=kern[3]), p, leaf, theta)
        self.plan_s = time.perf_counter() - t0
        self.n, self.nrhs = len(X), nrhs

    def step(self, W, targets: int, seed: int = 5):
        import ctypes

        O = self.O
        idx = inputs.subsample(self.n, targets, seed=seed)
        Wd = np.ascontiguousarray(W, dtype=np.float64)
        t1 = time.perf_counter()
        O.lib().orc_fkt_s2m(self.F.h, Wd.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self.nrhs)
        t2 = time.perf_counter()
        out = np.zeros((self.nrhs, len(idx)))
        T = np.ascontiguousarray(idx, dtype=np.int64)
        O.lib().orc_fkt_eval(self.F.h, T.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(T),
                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        t3 = time.perf_counter()
        return t2 - t1, t3 - t2


def oracle_steps(runners, steps: int, warmup: int, units_full: float, n_total: int) -> dict:
    """Time `steps` oracle steps over the given (runner, weights, targets) triples (one triple per
    sampled problem) after `warmup` untimed ones of 200 targets.  value = the MVM-equivalents the
    timed steps produced (units_full x sampled targets / n_total, units_full = MVMs of one full
    product of n_total points) over their elapsed time, so steps x ms_per_step is the time actually
    spent; extrapolated_value = the same oracle's full product (s2m once + every target, sampled
    problems extrapolated by points) estimated from the measured times."""
    for _ in range(warmup):
        for R, W, T in runners:
            R.step(W, min(200, T))
    s2m = [0.0] * len(runners)
    trav = [0.0] * len(runners)
    t0 = time.perf_counter()
    for k in range(steps):
        for i, (R, W, T) in enumerate(runners):
            a, b = R.step(W, T, seed=5 + k)
            s2m[i] += a
            trav[i] += b
    elapsed = time.perf_counter() - t0
    sampled = sum(T for _, _, T in runners)
    done = steps * units_full * sampled / n_total
    full_s = sum((s2m[i] + trav[i] * R.n / T) / steps for i, (R, _, T) in enumerate(runners))
    full_s *= n_total / sum(R.n for R, _, _ in runners)
    return {"value": done / elapsed, "ms_per_step": 1e3 * elapsed / steps, "elapsed_s": elapsed,
            "extrapolated_value": units_full / full_s, "s2m_s": sum(s2m) / steps,
            "traversal_s": sum(trav) / steps, "targets_per_step": sampled}


def oracle_setup(a, X=None, W=None, probs=None, offsets=None, leafs=None):
    """(runners, units of a full product, points of a full product, description) for the workload:
    the problem itself, or problems 0, 1, 2 of the batch (at the batch's leaf sizes when given;
    512 when the batch autotunes them and no tuned sizes are known)."""
    if probs is not None:
        runners, n_total = [], int(offsets[-1])
        for i in (0, 1, 2):
            Xi, *kern = probs[i]
            lo, hi = offsets[i], offsets[i + 1]
            leaf = int(leafs[i]) if leafs is not None else (a.leaf or 512)
            runners.append((OracleRunner(Xi, kern, a.p, leaf, a.theta, a.nrhs), W[:, lo:hi],
                            min(hi - lo, ORACLE_TARGETS // 3)))
        return runners, 256 * a.nrhs, n_total, "problems 0, 1, 2 of the batch"
    R = OracleRunner(X, a.kern, a.p, a.leaf, a.theta, a.nrhs)
    return [(R, W, min(len(X), ORACLE_TARGETS))], a.nrhs, len(X), "the whole problem"


def oracle_sample_note(rec, runners, what) -> str:
    return (f"per step: s2m of {runners[0][0].nrhs} right-hand sides over all nodes ({rec['s2m_s']:.1f} s) + "
            f"traversal of {rec['targets_per_step']} sampled targets ({rec['traversal_s']:.1f} s) of {what}; "
            f"value = outputs produced / elapsed time; extrapolated full product "
            f"{rec['extrapolated_value']:.3g} MVM/s; oracle tree not counted")


def cpu_baseline(a, X, W, probs=None, batch=None):
    """The oracle on the host cores: two oracle steps, the reference arm's rule."""
    from oracle import oracle as O

    runners, units, n_total, what = oracle_setup(a, X, W, probs, batch.offsets if batch is not None else None,
                                                 batch.leaf_sizes if batch is not None else None)
    rec = oracle_steps(runners, 2, 0, units, n_total)
    return {"value": rec["value"], "unit": "MVM/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": oracle_sample_note(rec, runners, what), "extrapolated_value": rec["extrapolated_value"]}


def run_reference(a):
    """The oracle (the deliberately slow reference program) on the host cores, on the same
    workload; each step is one oracle step (ORACLE_TARGETS sampled targets)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    if a.workload == "gpsolve":
        return {"impl": "reference", "unavailable": "the float64 oracle has no solver: the GP-solve workload has "
                                                    "no CPU reference program"}
    if a.workload == "batch256":
        sizes = inputs.batch_sizes(256, 2000, 200000)
        probs = [(inputs.unit_ball(int(n), 3, seed=100 + i), *BATCH_KERNELS[i % 3]) for i in range(3)
                 for n in [sizes[i]]]
        offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        W = make_weights(a, int(offsets[-1]))
        runners, units, n_total, what = oracle_setup(a, W=W, probs=probs, offsets=offsets)
    else:
        X = WORKLOADS[a.workload]["points"](a.n)
        W = make_weights(a, len(X))
        runners, units, n_total, what = oracle_setup(a, X, W)
    rec = oracle_steps(runners, a.steps, a.warmup, units, n_total)
    from oracle import oracle as O

    cb = {"value": rec["value"], "unit": "MVM/s", "cores": O.num_threads(), "kind": "oracle",
          "sample": oracle_sample_note(rec, runners, what), "extrapolated_value": rec["extrapolated_value"]}
    return {"impl": "reference", "metric": metric_name(a.workload),
            "value": rec["value"], "unit": "MVM/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "sample": cb["sample"], "timed_s": rec["elapsed_s"],
                       "extrapolated_value": rec["extrapolated_value"],
                       "extrapolated_note": "full product (s2m once + all targets) estimated from the timed steps"},
            "cpu_baseline": cb,
            "e2e": {"value": rec["value"], "unit": "MVM/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_pipes(a):
    """Lane-operation throughput of the FP32, FP32x2 and MUFU pipes (fkt_probe_pipe_rate) with the SM
    clock sampled during the runs: the per-SM, per-clock rates the ALU rooflines divide by."""
    import torch

    from paper_2106_04487_gb300 import fkt

    torch.cuda.set_device(0)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    fkt.fkt_probe_pipe_rate("ffma", 1 << 12)  # load the module, wake the clocks
    rates = {}
    with ClockSampler(0) as clk:
        for op in fkt.PIPE_OPS:
            fkt.fkt_probe_pipe_rate(op, 1 << 14)
            rates[op] = max(fkt.fkt_probe_pipe_rate(op, 1 << 16) for _ in range(3))
    c = clk.summary()
    mhz = c["sm_mhz"] or load_peaks()[0].get("sm_max_mhz", 2070.0)
    per_clk = {op: r / (nsm * mhz * 1e6) for op, r in rates.items()}
    return {"metric": "pipe lane-ops per SM per clock", "value": per_clk["ex2"], "unit": "lanes/SM/clock (ex2)",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "pipes: 8 CTAs x 256 threads per SM, 8 independent chains, 2^16 iterations",
                       "lane_ops_per_second": rates, "lanes_per_sm_per_clock": per_clk, "sms": nsm,
                       "sm_mhz_used": mhz},
            "clocks": c}


def main():
    a = parse()
    if a.workload == "pipes":
        print(json.dumps(run_pipes(a)))
        return
    if a.impl == "reference":
        out = run_reference(a)
    elif a.workload == "gpsolve":
        out = run_gpsolve(a)
    else:
        out = run_ours(a)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
