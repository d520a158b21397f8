"""Host arithmetic of bench.py that its JSON line rests on: expansion sizes, the per-pair work
counts behind the rooflines, and the launch count per step.  No GPU."""
import pytest

import bench


def test_expansion_sizes():
    # binom(p + d, d): 35 / 84 / 165 terms at p = 4 / 6 / 8 in d = 3, 210 at p = 6 in d = 4
    assert [bench.nterms(3, p) for p in (4, 6, 8)] == [35, 84, 165]
    assert bench.nterms(4, 6) == 210


def test_far_pair_ops_counts_each_stage():
    p = 6
    pairs = [(k, j) for k in range(p + 1) for j in range(k, p + 1, 2)]
    assert len(pairs) == 16
    radial = sum(j + 1 for _, j in pairs)           # R_kj = sum_m That_kjm J_m
    assert radial == 78
    assert bench.far_pair_ops(p) == 10 + 3 * (p + 1) + radial + p + len(pairs) + 3 * (p + 1) ** 2 + 84 == 362
    # the compressed 1/r expansion: radial pairs (k, k) only, (p+1)^2 terms
    assert bench.far_pair_ops(p, diag=True) == 10 + 3 * 7 + sum(k + 1 for k in range(7)) + p + 7 + 3 * 49 + 49


@pytest.mark.parametrize("kernel,nw,tensor,want", [("matern32", 32, True, (8, 1 / 16 + 1 / 32)),
                                                   ("matern32", 32, False, (40, 1 / 16 + 1 / 32)),
                                                   ("gaussian", 1, False, (7, 1 / 32)), ("cauchy", 8, False, (15, 1 / 16))])
def test_near_pair_cost(kernel, nw, tensor, want):
    assert bench.near_pair_cost(kernel, nw, tensor) == pytest.approx(want)


def test_launches_per_step():
    # one pass of 32: permute, near, 4 x (s2m + reduce), pack + tensor-core far, unpermute
    assert bench.launches_per_step(32, "bf16x3") == 13
    # float32 far field: one far launch per group of 8
    assert bench.launches_per_step(32, "fp32") == 3 + 8 + 4
    # one right-hand side on the float32 path: s2m, reduce and far once
    assert bench.launches_per_step(1, "fp32") == 6
    # two passes (33 right-hand sides)
    assert bench.launches_per_step(33, "bf16x3") == 13 + (3 + 2 + 2)


def test_gpsolve_orchestration_with_a_fake_plan(monkeypatch):
    """bench.py --workload gpsolve on stand-ins for torch and the binding: the timed solves use the
    coarse space, the comparison solves do not, and the JSON line adds up."""
    import numpy as np

    class T:
        def __init__(self, a):
            self.a = a

        def cuda(self):
            return self

        def pin_memory(self):
            return self

        def to(self, *args, **kw):
            return self

        def copy_(self, o):
            self.a[...] = o.a
            return self

    class FakeTorch:
        class cuda:
            set_device = staticmethod(lambda i: None)
            synchronize = staticmethod(lambda: None)

        from_numpy = staticmethod(T)
        empty_like = staticmethod(lambda t: T(np.empty_like(t.a)))

    calls = []

    class Plan:
        def __init__(self, X, kname, **kw):
            assert kname == "matern52" and X.a.shape == (1000, 4)
            self.opt = {}

        def set_option(self, k, v):
            self.opt[k] = v

        def solve(self, sigma2, b, tol, max_iter, raise_on_not_converged):
            calls.append((self.opt["preconditioner"], self.opt.get("coarse_rank"), max_iter))
            its = 100 if self.opt.get("coarse_rank") != "0" else max_iter
            return T(np.zeros_like(b.a)), {"iterations": min(its, max_iter), "converged": its <= max_iter,
                                           "rel_residual": 1e-6, "true_rel_residual": 1e-3}

        def stats(self):
            return {"coarse_columns": 173 if self.opt.get("coarse_rank") != "0" else 0}

        def close(self):
            pass

    class FakeFkt:
        pass

    FakeFkt.Plan = Plan
    monkeypatch.setattr("sys.argv", ["bench.py", "--workload", "gpsolve", "--n", "1000", "--steps", "2",
                                     "--warmup", "3", "--compare-iters", "50"])
    out = bench.run_gpsolve(bench.parse(), fkt=FakeFkt, torch=FakeTorch)
    timed = [c for c in calls if c[1] == "256" and c[2] == 50]
    assert len(timed) >= 2 + 1                       # the timed steps and the end-to-end solve
    assert ("none", "0", 50) in calls and ("block_jacobi", "0", 50) in calls
    assert out["unit"] == "RHS/s" and out["steps"] == 2 and out["value"] > 0
    assert out["config"]["timed_solve"]["coarse_columns"] == 173
    assert [c["preconditioner"] for c in out["config"]["compare"]] == ["none", "block_jacobi"]
    assert out["e2e"]["h2d_bytes_per_step"] == 8 * 1000 * 4


def test_reference_arm_line(monkeypatch):
    """bench.py --impl reference (the float64 oracle on the host cores) on a small case: the keys
    of the line the reference arm must print."""
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--workload", "gauss20k", "--n", "3000",
                                     "--steps", "1", "--warmup", "1"])
    out = bench.run_reference(bench.parse())
    assert out["impl"] == "reference" and out["unit"] == "MVM/s" and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] >= 1
    assert out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"] == {"value": out["value"], "unit": "MVM/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert out["config"]["workload"].startswith("gaussian l=0.1 d=3 N=3000")
    # what was timed: steps x ms_per_step is the elapsed time of the timed steps
    assert abs(out["steps"] * out["ms_per_step"] / 1e3 - out["config"]["timed_s"]) < 1e-6
    # N = 3000 <= the per-step target sample: every step is a whole product, so the measured
    # rate and the full-product extrapolation agree up to timing noise
    assert 0.5 < out["config"]["extrapolated_value"] / out["value"] < 2.0
    assert out["metric"] == bench.metric_name("gauss20k")


def test_metric_names_match_the_benchmark():
    """Both arms print the same metric string; the headline one is the benchmark's own."""
    import json
    import os

    with open(os.path.join(os.path.dirname(bench.__file__), "BASELINE.json")) as fh:
        assert bench.metric_name("matern1m") == json.load(fh)["metric"]
    assert len({bench.metric_name(w) for w in bench.WORKLOADS}) == len(bench.WORKLOADS)


def test_oracle_step_accounting():
    """oracle_steps on stand-in runners with known times: value counts only the outputs produced."""
    import time

    class R:
        n, nrhs = 1000, 4

        def step(self, W, T, seed=5):
            time.sleep(0.01)
            return 0.004, 0.006

    rec = bench.oracle_steps([(R(), None, 100)], steps=3, warmup=0, units_full=4, n_total=1000)
    assert rec["targets_per_step"] == 100
    # 3 steps x 4 MVMs x 100/1000 of the outputs = 1.2 MVM-equivalents in about 0.03 s
    assert 1.2 / (3 * 0.02) < rec["value"] < 1.2 / (3 * 0.0099)
    # full product: s2m 0.004 s + traversal 0.006 s x 10
    assert abs(rec["extrapolated_value"] - 4 / 0.064) < 1e-9


def test_two_dimensional_counts():
    # d = 2: binom(p + 2, 2) terms = 1 + 2 per degree k >= 1, times the radial terms of degree k
    assert bench.nterms(2, 4) == 15 == sum((1 if k == 0 else 2) * ((4 - k) // 2 + 1) for k in range(5))
    p = 4
    pairs = [(k, j) for k in range(p + 1) for j in range(k, p + 1, 2)]
    assert bench.far_pair_ops(p, d=2) == 7 + 3 * (p + 1) + sum(j + 1 for _, j in pairs) + p + len(pairs) + 4 * p + 15
    # two coordinate differences and |x|^2 with one MUL + one FMA
    assert bench.near_pair_cost("cauchy", 1, False, d=2) == pytest.approx((4 + 1 + 1, 1 / 16))
    assert bench.far_kernel_name(4, "fp32", 1, d=2) == "far_kernel<2,4,1>"
