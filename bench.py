"""Benchmark: FKT MVMs/s on one GB300 for the N = 1M, d = 3 Gaussian-mixture workload.

One step = one fkt_mvm call (all stages of Algorithm 1: permute, s2m, near field,
m2t + combine) on resident device buffers.  L2 is flushed between timed steps
(a 256 MiB write outside the timed events).  Prints ONE JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--kernel matern32|cauchy] [--p P] [--theta T] [--leaf M] [--nrhs R]

--impl reference times the CPU float64 oracle (the slow reference program) on a
bounded sample of the same workload.  Multi-GPU runs are independent replicas
(one plan per rank, no collective): the value is the sum over ranks.
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
def launches_per_step(nrhs: int, far_precision: str) -> int:
    """Kernels the library launches per fkt_mvm: per group of right-hand sides (1 or 8) permute, s2m,
    s2m_reduce and near field; the float32 far field once per group, the tensor-core far field
    (pack + far) once per pass of 32."""
    if far_precision == "fp32":
        groups = 1 if nrhs == 1 else (nrhs + 7) // 8
        return 5 * groups
    groups = (nrhs + 7) // 8
    passes = (nrhs + 31) // 32
    return 4 * groups + 2 * passes


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel", default="matern32", choices=list(KERNELS))
    ap.add_argument("--p", type=int, default=6)
    ap.add_argument("--theta", type=float, default=0.4)
    ap.add_argument("--leaf", type=int, default=256)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--near-tpt", type=int, default=2, choices=[2, 4])
    ap.add_argument("--far-precision", default="fp32", choices=["fp32", "bf16x3", "tf32", "bf16"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--err-targets", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload_name(a):
    k, ell = KERNELS[a.kernel]
    return (f"{k} l={ell} d=3 N={a.n} gaussian-mixture(10 comps, std 0.05) p={a.p} leaf={a.leaf} "
            f"theta={a.theta} nrhs={a.nrhs} near_tpt={a.near_tpt} far={a.far_precision}")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


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


def near_pair_cost(kernel: str, nrhs: int):
    """Lower bound on SM issue slots per near-field pair: (FP32-pipe ops, MUFU ops).

    Per pair the method needs d = 3 subtractions, |x|^2 (1 MUL + 2 FMA), the kernel value
    and one FMA per right-hand side.  Matern-3/2: sqrt (MUFU), u = c r (MUL), exp(-u) (MUFU ex2),
    (1 + c r) e (FMA + MUL).  Cauchy: 1 + c r^2 (FMA), reciprocal (MUFU)."""
    if kernel == "matern32":
        return 3 + 3 + 1 + 2 + nrhs, 2
    return 3 + 3 + 1 + nrhs, 1


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
    stats = plan.stats()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(a.warmup):
        plan.mvm(Wd, out=Yd)
    barrier()
    step_ms, near_ms, far_ms, s2m_ms = [], [], [], []
    with ClockSampler(local) as clk:
        for _ in range(a.steps):
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
    barrier()
    plan.check()  # raises if a bounded device-side wait ran out during the timed steps
    total_ms = float(sum(step_ms))
    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    mvms = a.steps * a.nrhs * world
    value = mvms / (total_ms / 1e3)

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

    # accuracy of this launch against the float64 dense product on sampled targets
    from oracle import oracle as O

    idx = inputs.subsample(a.n, a.err_targets)
    y = Yd.cpu().numpy().astype(np.float64)
    zd = O.dense(X, O.kparams(kname, ell), W, idx)
    rel_err = float(max(np.linalg.norm(y[r, idx] - zd[r]) / np.linalg.norm(zd[r]) for r in range(a.nrhs)))

    # roofline of the dominant kernel (near field): ALU bound, FP32 + MUFU pipes
    peaks, src = load_peaks()
    clocks = clk.summary()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_ops, mufu_ops = near_pair_cost(kname, a.nrhs)
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    slots_per_pair = max(fp32_ops / 128.0, mufu_ops / 16.0)  # SM clocks per pair (128 FP32, 16 MUFU lanes/SM)
    peak_pairs = nsm * sm_max * 1e6 / slots_per_pair
    near_pairs = stats["near_pairs"]  # the kernel value of a pair serves every right-hand side
    near_avg_ms = float(np.mean(near_ms))
    achieved = near_pairs / (near_avg_ms / 1e3)
    out = {
        "metric": f"FKT MVMs/s at N=1M, d=3 ({kname}, rel.err vs FP64 dense {rel_err:.1e})",
        "value": value,
        "unit": "MVM/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": total_ms / a.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_name(a), "l2": "flushed between steps (256 MiB write)",
                   "rel_err_vs_fp64_dense": rel_err, "err_targets": a.err_targets,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "plan_ms": stats["plan_ms"], "near_pairs": stats["near_pairs"], "far_pairs": stats["far_pairs"],
                   "s2m_pairs": stats["s2m_pairs"], "stage_ms": {"near": near_avg_ms, "far+wait": float(np.mean(far_ms)),
                                                                 "s2m": float(np.mean(s2m_ms))}},
        "roofline": {"kernel": "near_kernel", "bound": "alu", "achieved": achieved / 1e9, "peak": peak_pairs / 1e9,
                     "unit": "Gpair/s", "frac": achieved / peak_pairs, "traffic": None,
                     "peak_source": f"{nsm} SMs x {sm_max:.0f} MHz / max({fp32_ops}/128 FP32, {mufu_ops}/16 MUFU) "
                                    f"SM-clocks per pair ({src} clock)"},
        "e2e": {"value": e2e_value, "unit": "MVM/s", "h2d_bytes_per_step": int(W.nbytes),
                "d2h_bytes_per_step": int(W.nbytes)},
        "gpu_launches": launches_per_step(a.nrhs, a.far_precision) * a.steps,
        "clocks": clocks,
    }
    if rank == 0 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(a, X, W)
    plan.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return out if rank == 0 else None


class OracleRunner:
    """The float64 oracle, as it stands, on the host cores.  One sample = s2m over all nodes
    (needed by any target) + the per-target traversal for a sample of targets, extrapolated to
    one full MVM; the oracle's tree (its plan) is built once and not counted."""

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
        return (f"s2m over all nodes ({s2m_s:.1f} s) + traversal of {target_sample} of {self.a.n} targets "
                f"({trav_s:.1f} s), extrapolated to all targets; oracle tree ({self.plan_s:.1f} s) not counted")


def cpu_baseline(a, X, W, target_sample: int = 2000):
    R = OracleRunner(a, X)
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
    sample = 500
    for _ in range(a.warmup):
        R.mvm_seconds(W, 50)
    total, s2m_tot, trav_tot = 0.0, 0.0, 0.0
    for _ in range(a.steps):
        per_mvm, s2m_s, trav_s = R.mvm_seconds(W, sample)
        total += per_mvm
        s2m_tot += s2m_s
        trav_tot += trav_s
    value = a.steps * a.nrhs / total
    cb = {"value": value, "unit": "MVM/s", "cores": R.O.num_threads(), "kind": "oracle",
          "sample": R.describe(s2m_tot / a.steps, trav_tot / a.steps, sample) + " (per step)"}
    return {"impl": "reference", "metric": f"FKT MVMs/s at N=1M, d=3 ({KERNELS[a.kernel][0]})", "value": value,
            "unit": "MVM/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
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
