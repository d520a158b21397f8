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


@pytest.mark.parametrize("kernel,nw,tensor,want", [("matern32", 32, True, (8, 2)), ("matern32", 32, False, (40, 2)),
                                                   ("gaussian", 1, False, (7, 1)), ("cauchy", 8, False, (15, 1))])
def test_near_pair_cost(kernel, nw, tensor, want):
    assert bench.near_pair_cost(kernel, nw, tensor) == want


def test_launches_per_step():
    # one pass of 32: permute, near, 4 x (s2m + reduce), pack + tensor-core far, unpermute
    assert bench.launches_per_step(32, "bf16x3") == 13
    # float32 far field: one far launch per group of 8
    assert bench.launches_per_step(32, "fp32") == 3 + 8 + 4
    # one right-hand side on the float32 path: s2m, reduce and far once
    assert bench.launches_per_step(1, "fp32") == 6
    # two passes (33 right-hand sides)
    assert bench.launches_per_step(33, "bf16x3") == 13 + (3 + 2 + 2)
