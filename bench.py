"""Benchmark: FKT MVMs/s on one GB300 for the N = 1M, d = 3 Gaussian-mixture workload.

Headline: the precision form (far field on the tensor cores, BF16 hi/lo split with float32
accumulation; near field float32) for 32 right-hand sides of the Matern-3/2 kernel, with the
plain float32 form timed on the same plan beside it, the Cauchy kernel as a second line, and the
error of every form against the float64 dense product on a 10,000-target subsample.

One step = one fkt_mvm call over all right-hand sides (all stages of Algorithm 1: permute, s2m,
near field, m2t + combine) on resident device buffers; one MVM = one right-hand side.  L2 is
flushed between timed steps (a 256 MiB write outside the timed events).  Prints ONE JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--kernel matern32|cauchy] [--p P] [--theta T] [--leaf M] [--nrhs R]
                    [--far-precision bf16x3|tf32|bf16|fp32] [--near-precision tf32x3|fp32]
                    [--compare fp32|none]

--impl reference times the CPU float64 oracle (the slow reference program) on a bounded sample
of the same workload.  Multi-GPU runs are independent replicas (one plan per rank, no
collective): the value is the sum over ranks.
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

KERNELS = {"matern32": ("matern32", 0.2), "cauchy": ("cauchy", 0.05)}
PASS = 32  # right-hand sides per pass of the library

# DRAM bytes (read + write) per launch of a kernel from one ncu capture, keyed by kernel and
# workload (kernel, p, theta, leaf, nrhs, N); see profiles/near_tc_matern1m_p6_theta0375_nrhs32.md.
# Any other workload reports null.
PROFILED_TRAFFIC = {("near_tile_kernel<3,matern32,32>", "matern32", 6, 0.375, 256, 32, 1_000_000): 1.339e9 + 0.136e9,
                    ("near_tc_kernel<3,matern32>", "matern32", 6, 0.375, 256, 32, 1_000_000): 0.899e9 + 0.130e9}


def near_kernel_name(kname: str, nw: int, near_precision: str = "fp32") -> str:
    if nw == 32 and near_precision == "tf32x3":
        return f"near_tc_kernel<3,{kname}>"
    base = "near_kernel" if nw == 1 else "near_wide_kernel" if nw == 8 else "near_tile_kernel"
    return f"{base}<3,{kname},{nw}>"


def launches_per_step(nrhs: int, far_precision: str) -> int:
    """Kernels the library launches per fkt_mvm.  Per pass of up to 32 right-hand sides: permute
    and near field once; s2m + s2m_reduce per group of 8 (1 for a single right-hand side on the
    float32 path); the float32 far field once per group, the tensor-core far field (pack + far)
    once per pass."""
    total = 0
    for r0 in range(0, nrhs, PASS):
        npass = min(PASS, nrhs - r0)
        group = 1 if (nrhs == 1 and far_precision == "fp32") else 8
        groups = (npass + group - 1) // group
        total += 2 + 2 * groups + (groups if far_precision == "fp32" else 2)
    return total


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel", default="matern32", choices=list(KERNELS))
    ap.add_argument("--p", type=int, default=6)
    ap.add_argument("--theta", type=float, default=0.375)
    ap.add_argument("--leaf", type=int, default=256)
    ap.add_argument("--nrhs", type=int, default=32)
    ap.add_argument("--near-tpt", type=int, default=2, choices=[2, 4])
    ap.add_argument("--far-precision", default="bf16x3", choices=["bf16x3", "tf32", "bf16", "fp32"])
    ap.add_argument("--near-precision", default="tf32x3", choices=["tf32x3", "fp32"],
                    help="near-field contraction of 32-wide passes: tensor cores (TF32 hi/lo) or CUDA cores")
    ap.add_argument("--compare", default="fp32", choices=["fp32", "none"],
                    help="plain float32 form (near and far on the CUDA cores) timed beside the headline one")
    ap.add_argument("--second-kernel", default="cauchy", choices=list(KERNELS) + ["none"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--err-targets", type=int, default=10000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload_name(a, kernel=None):
    k, ell = KERNELS[kernel or a.kernel]
    return (f"{k} l={ell} d=3 N={a.n} gaussian-mixture(10 comps, std 0.05) p={a.p} leaf={a.leaf} "
            f"theta={a.theta} nrhs={a.nrhs} near={a.near_precision} far={a.far_precision}")


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


def near_pair_cost(kernel: str, nw: int, tensor: bool = False):
    """Lower bound on SM issue slots per near-field pair for a pass of nw right-hand sides:
    (FP32-pipe lane-ops, MUFU lane-ops).

    Per pair the method needs d = 3 subtractions, |x|^2 (1 MUL + 2 FMA), the kernel value and
    one FMA per right-hand side.  Matern-3/2: sqrt (MUFU), (1 + u ln2) (FMA), 2^-u (MUFU ex2),
    product (MUL).  Cauchy: 1 + q (ADD), reciprocal (MUFU).  With the contraction on the tensor
    cores (tensor=True) the per-right-hand-side FMAs leave the FP32 pipe."""
    fma = 0 if tensor else nw
    if kernel == "matern32":
        return 3 + 3 + 2 + fma, 2
    return 3 + 3 + 1 + fma, 1


def nterms(d: int, p: int) -> int:
    n = 1
    for i in range(1, d + 1):
        n = n * (p + i) // i
    return n


def time_form(plan, Wd, Yd, steps, warmup, flush, stream):
    """Per-step CUDA-event times of plan.mvm on the plan's launching stream, with the library's
    own per-stage events (near, far + wait, s2m) read after each step."""
    import torch

    for _ in range(warmup):
        plan.mvm(Wd, out=Yd)
    torch.cuda.synchronize()
    step_ms, near_ms, far_ms, s2m_ms = [], [], [], []
    for _ in range(steps):
        flush.fill_(1.0)  # evict L2 between steps (outside the timed events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.mvm(Wd, out=Yd)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        s = plan.stats()
        near_ms.append(s["last_near_ms"])
        far_ms.append(s["last_far_ms"])
        s2m_ms.append(s["last_s2m_ms"])
    torch.cuda.synchronize()
    return {"step_ms": step_ms, "near_ms": float(np.mean(near_ms)), "far_ms": float(np.mean(far_ms)),
            "s2m_ms": float(np.mean(s2m_ms))}


def rel_errs(y, z, idx):
    """Per right-hand side relative 2-norm error of y (all targets) on the sampled targets idx."""
    return [float(np.linalg.norm(y[r, idx] - z[r]) / np.linalg.norm(z[r])) for r in range(z.shape[0])]


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
    kname, ell = KERNELS[a.kernel]
    X = inputs.gaussian_mixture(a.n, 3, 10, 0.05)
    W = inputs.normal_weights(a.n, a.nrhs)
    Xd = torch.from_numpy(X).cuda()
    Wd = torch.from_numpy(W).cuda()
    Yd = torch.empty_like(Wd)
    plan = fkt.Plan(Xd, kname, lengthscale=ell, p=a.p, leaf_size=a.leaf, theta=a.theta)
    plan.set_option("timing", "1")
    plan.set_option("near_targets_per_thread", str(a.near_tpt))
    plan.set_option("far_precision", a.far_precision)
    plan.set_option("near_precision", a.near_precision)
    stats = plan.stats()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    # headline form: warm-up, then exactly K timed steps between barriers
    for _ in range(a.warmup):
        plan.mvm(Wd, out=Yd)
    barrier()
    with ClockSampler(local) as clk:
        head = time_form(plan, Wd, Yd, a.steps, 0, flush, stream)
    barrier()
    plan.check()  # raises if a bounded device-side wait ran out during the timed steps
    total_ms = float(sum(head["step_ms"]))
    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = a.steps * a.nrhs * world / (total_ms / 1e3)
    y_head = Yd.cpu().numpy().astype(np.float64)

    # the plain float32 form on the same plan
    comp = None
    if a.compare != "none" and (a.far_precision, a.near_precision) != ("fp32", "fp32"):
        plan.set_option("far_precision", "fp32")
        plan.set_option("near_precision", "fp32")
        comp = time_form(plan, Wd, Yd, max(3, a.steps // 2), 3, flush, stream)
        plan.check()
        y_comp = Yd.cpu().numpy().astype(np.float64)
        plan.set_option("far_precision", a.far_precision)
        plan.set_option("near_precision", a.near_precision)

    # end to end through the host-buffer entry point (copies inside the timed region)
    Wh = torch.from_numpy(W).pin_memory()
    Yh = torch.empty_like(Wh).pin_memory()
    plan.set_option("timing", "0")
    for _ in range(2):
        fkt.fkt_mvm_host(plan.h, Wh, Yh, a.nrhs)
    torch.cuda.synchronize()
    e2e_steps = max(3, a.steps // 2)
    e2e_total = 0.0
    for _ in range(e2e_steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        fkt.fkt_mvm_host(plan.h, Wh, Yh, a.nrhs)  # H2D copy, MVM, D2H copy, stream sync
        e2e_total += time.perf_counter() - t1
    e2e_value = e2e_steps * a.nrhs / e2e_total
    plan.close()

    # second kernel of the workload (both forms, fewer steps)
    second = None
    if a.second_kernel != "none" and a.second_kernel != a.kernel:
        k2, ell2 = KERNELS[a.second_kernel]
        p2 = fkt.Plan(Xd, k2, lengthscale=ell2, p=a.p, leaf_size=a.leaf, theta=a.theta)
        p2.set_option("timing", "1")
        p2.set_option("near_targets_per_thread", str(a.near_tpt))
        second = {"kernel": f"{k2} l={ell2}"}
        ys = {}
        head_form = f"near {a.near_precision}, far {a.far_precision}"
        forms = {head_form: (a.near_precision, a.far_precision)}
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

    idx = inputs.subsample(a.n, a.err_targets)
    zd = O.dense(X, O.kparams(kname, ell), W, idx)
    err_head = rel_errs(y_head, zd, idx)
    if comp is not None:
        err_comp = rel_errs(y_comp, zd, idx)
    if second is not None:
        n2 = min(2000, a.err_targets)
        idx2 = inputs.subsample(a.n, n2, seed=7)
        z2 = O.dense(X, O.kparams(*KERNELS[a.second_kernel]), W, idx2)
        for form, y in ys.items():
            e = rel_errs(y, z2, idx2)
            second[form]["rel_err_max"] = max(e)
            second[form]["rel_err_median"] = float(np.median(e))
        second["err_targets"] = n2

    # roofline of the dominant kernel: the near field (FP32 + MUFU pipes, ALU bound) or the
    # tensor-core far field (its contraction on the tensor pipe)
    peaks, src = load_peaks()
    clocks = clk.summary()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    nw = 1 if (a.nrhs == 1 and a.far_precision == "fp32") else (8 if a.nrhs <= 8 else 16 if a.nrhs <= 16 else 32)
    passes = (a.nrhs + PASS - 1) // PASS
    near_tc = nw == 32 and a.near_precision == "tf32x3"
    fp32_ops, mufu_ops = near_pair_cost(kname, nw, near_tc)
    slots_per_pair = max(fp32_ops / 128.0, mufu_ops / 16.0)  # SM clocks per pair (128 FP32, 16 MUFU lanes/SM)
    peak_pairs = nsm * sm_max * 1e6 / slots_per_pair
    near_pairs = stats["near_pairs"] * passes  # one launch per pass; its kernel value serves the pass
    near_ach = near_pairs / (head["near_ms"] / 1e3)
    near_name = near_kernel_name(kname, nw, a.near_precision)
    traffic = PROFILED_TRAFFIC.get((near_name, kname, a.p, a.theta, a.leaf, a.nrhs, a.n))
    near_roof = {"kernel": near_name, "bound": "alu", "achieved": near_ach / 1e9,
                 "peak": peak_pairs / 1e9, "unit": "Gpair/s", "frac": near_ach / peak_pairs, "traffic": traffic,
                 "traffic_unit": "bytes per launch (ncu dram__bytes_read + write)",
                 "ms_per_step": head["near_ms"],
                 "peak_source": f"{nsm} SMs x {sm_max:.0f} MHz / max({fp32_ops}/128 FP32, {mufu_ops}/16 MUFU) "
                                f"SM-clocks per pair ({src} clock)"}
    roofs = [near_roof]
    if a.far_precision != "fp32":
        nt = nterms(3, a.p)
        flops = 2.0 * stats["far_pairs"] * nt * a.nrhs  # the m2t contraction, once (not the hi/lo copies)
        far_ms = head["far_ms"]
        peak_tf = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0))
        if a.far_precision == "tf32":
            peak_tf *= 0.5  # nominal TF32 : BF16 dense ratio
        ach_tf = flops / (far_ms / 1e3) / 1e12
        roofs.append({"kernel": f"far_tc_kernel<3,{a.p},{a.far_precision}>", "bound": "tensor", "achieved": ach_tf,
                      "peak": peak_tf, "unit": "TFLOP/s", "frac": ach_tf / peak_tf, "traffic": None,
                      "ms_per_step": far_ms,
                      "peak_source": f"{src} bf16 dense (sustained){' x 0.5 for tf32' if a.far_precision == 'tf32' else ''};"
                                     f" far stage time (far_tc launch + wait for pack)"})
    roofs.sort(key=lambda r: -r["ms_per_step"])
    out = {
        "metric": f"FKT MVMs/s at N=1M, d=3 ({kname}, near {a.near_precision}, far {a.far_precision}, "
                  f"rel.err vs FP64 dense {max(err_head):.1e})",
        "value": value,
        "unit": "MVM/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": total_ms / a.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": (f"f32 kernel values, {'tf32x3 tensor-core' if near_tc else 'f32'} near contraction, "
                  f"{a.far_precision} far contraction, f32 accumulate"),
        "data": "synthetic",
        "config": {"workload": workload_name(a), "l2": "flushed between steps (256 MiB write)",
                   "rel_err_max": max(err_head), "rel_err_median": float(np.median(err_head)),
                   "err_targets": a.err_targets, "err_reference": "float64 dense oracle",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "plan_ms": stats["plan_ms"], "near_pairs": stats["near_pairs"], "far_pairs": stats["far_pairs"],
                   "s2m_pairs": stats["s2m_pairs"],
                   "stage_ms": {"near": head["near_ms"], "far+wait": head["far_ms"], "s2m": head["s2m_ms"]}},
        "roofline": roofs[0],
        "roofline_other": roofs[1:],
        "e2e": {"value": e2e_value, "unit": "MVM/s", "h2d_bytes_per_step": int(W.nbytes),
                "d2h_bytes_per_step": int(W.nbytes)},
        "gpu_launches": launches_per_step(a.nrhs, a.far_precision) * a.steps,
        "clocks": clocks,
    }
    if comp is not None:
        cv = a.nrhs * len(comp["step_ms"]) / (sum(comp["step_ms"]) / 1e3)
        out["compare_form"] = {"form": "plain float32 (near and far on the CUDA cores)", "value": cv, "unit": "MVM/s",
                               "ms_per_step": float(np.mean(comp["step_ms"])), "rel_err_max": max(err_comp),
                               "rel_err_median": float(np.median(err_comp)),
                               "stage_ms": {"near": comp["near_ms"], "far+wait": comp["far_ms"], "s2m": comp["s2m_ms"]},
                               "speedup_of_headline": value / world / cv}
    if second is not None:
        out["second_kernel"] = second
    if rank == 0 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(a, X, W)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return out if rank == 0 else None


class OracleRunner:
    """The float64 oracle, as it stands, on the host cores.  One sample = s2m over all nodes
    (needed by any target) + the per-target traversal for a sample of targets, extrapolated to
    one full MVM of all right-hand sides; the oracle's tree (its plan) is built once and not
    counted."""

    def __init__(self, a, X):
        from oracle import oracle as O

        self.O = O
        kname, ell = KERNELS[a.kernel]
        t0 = time.perf_counter()
        self.F = O.FKT(X, O.kparams(kname, ell), a.p, a.leaf, a.theta)
        self.plan_s = time.perf_counter() - t0
        self.a = a

    def mvm_seconds(self, W, target_sample):
        import ctypes

        O, a = self.O, self.a
        idx = inputs.subsample(a.n, target_sample, seed=5)
        Wd = np.ascontiguousarray(W, dtype=np.float64)
        t1 = time.perf_counter()
        O.lib().orc_fkt_s2m(self.F.h, Wd.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a.nrhs)
        t2 = time.perf_counter()
        out = np.zeros((a.nrhs, len(idx)))
        T = np.ascontiguousarray(idx, dtype=np.int64)
        O.lib().orc_fkt_eval(self.F.h, T.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(T),
                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        t3 = time.perf_counter()
        return (t2 - t1) + (t3 - t2) * a.n / len(idx), t2 - t1, t3 - t2

    def describe(self, s2m_s, trav_s, target_sample):
        return (f"s2m of {self.a.nrhs} right-hand sides over all nodes ({s2m_s:.1f} s) + traversal of "
                f"{target_sample} of {self.a.n} targets ({trav_s:.1f} s), extrapolated to all targets; "
                f"oracle tree ({self.plan_s:.1f} s) not counted")


def cpu_baseline(a, X, W, target_sample: int = 2000, budget_s: float = 10.0):
    R = OracleRunner(a, X)
    per_mvm, s2m_s, trav_s = R.mvm_seconds(W, target_sample)
    if trav_s < budget_s / 2:  # grow the target sample to about budget_s of traversal
        target_sample = int(min(a.n, target_sample * budget_s / max(trav_s, 1e-3)))
        per_mvm, s2m_s, trav_s = R.mvm_seconds(W, target_sample)
    return {"value": a.nrhs / per_mvm, "unit": "MVM/s", "cores": R.O.num_threads(), "kind": "oracle",
            "sample": R.describe(s2m_s, trav_s, target_sample)}


def run_reference(a):
    """The oracle (the deliberately slow reference program) on the host cores, on the same
    workload; each step is one bounded sample scaled to MVM/s."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    X = inputs.gaussian_mixture(a.n, 3, 10, 0.05)
    W = inputs.normal_weights(a.n, a.nrhs)
    R = OracleRunner(a, X)
    sample = 200
    for _ in range(a.warmup):
        R.mvm_seconds(W, 20)
    total, s2m_tot, trav_tot = 0.0, 0.0, 0.0
    for _ in range(a.steps):
        per_mvm, s2m_s, trav_s = R.mvm_seconds(W, sample)
        total += per_mvm
        s2m_tot += s2m_s
        trav_tot += trav_s
    value = a.steps * a.nrhs / total
    cb = {"value": value, "unit": "MVM/s", "cores": R.O.num_threads(), "kind": "oracle",
          "sample": R.describe(s2m_tot / a.steps, trav_tot / a.steps, sample) + " (per step)"}
    return {"impl": "reference", "metric": f"FKT MVMs/s at N=1M, d=3 ({KERNELS[a.kernel][0]}, float64 oracle)",
            "value": value, "unit": "MVM/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * total / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": {"workload": workload_name(a)}, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "MVM/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    a = parse()
    if a.impl == "reference":
        out = run_reference(a)
    else:
        out = run_ours(a)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
