"""fkt_mvm_noalloc: the FKT product for callers that cannot allocate device memory.

Callers recording a CUDA graph, latency-critical loops, and hosts whose device memory
belongs to another allocator cannot let fkt_mvm grow its work buffers with cudaMalloc.
fkt_mvm_noalloc takes those buffers from a fixed array the library declares statically.
This file is collected last on purpose, so a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2106_04487_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the relative 2-norm bar the other GPU tests use


@pytest.fixture(scope="module")
def fkt():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_04487_gb300 import build, fkt as F

    build.build()
    F.lib()
    return F


def _rel(a, b):
    return max(np.linalg.norm(a[i] - b[i]) / np.linalg.norm(b[i]) for i in range(len(b)))


@pytest.mark.parametrize("far_precision,nrhs,near_precision", [("fp32", 1, "fp32"), ("fp32", 11, "fp32"),
                                                                ("bf16x3", 11, "fp32"), ("bf16x3", 3, "fp32"),
                                                                ("bf16x3", 20, "tf32x3"), ("fp32", 32, "tf32x3")])
def test_noalloc_matches_fkt_mvm_on_two_calls(fkt, far_precision, nrhs, near_precision):
    """Both far-field paths: float32 on the CUDA cores, and the tensor-core path whose packed
    multipole image is also carved out of the scratch; nrhs 3 and 11 leave partial groups of 8.
    With 20 or 32 right-hand sides on the TF32 near kernel the pass's near-field image is carved
    out of the scratch too (at N = 20k, where everything fits the 48 MiB)."""
    import torch

    n = 60000 if near_precision == "fp32" else 20000
    X = torch.from_numpy(inputs.gaussian_mixture(n, 3, 10, 0.05, seed=21)).cuda()
    plan = fkt.Plan(X, "matern32", lengthscale=0.2, p=6, leaf_size=256, theta=0.5)
    plan.set_option("far_precision", far_precision)
    plan.set_option("near_precision", near_precision)
    for call, seed in enumerate((22, 23)):          # two calls in a row share the scratch
        w = torch.from_numpy(inputs.normal_weights(n, nrhs, seed=seed)).cuda()
        want = plan.mvm(w).cpu().numpy()             # the existing entry point
        got = torch.full_like(w, float("nan"))
        fkt.fkt_mvm_noalloc(plan.h, w, got, nrhs)
        torch.cuda.synchronize()
        got = got.cpu().numpy()
        assert np.isfinite(got).all(), call
        assert _rel(got, want) < TOL, call
    plan.close()


@pytest.mark.parametrize("far_precision", ["fp32", "bf16x3"])
def test_noalloc_call_allocates_no_device_memory(fkt, far_precision):
    """The defining property: on a fresh plan (none of fkt_mvm's work buffers exist yet) a call
    leaves the device's free memory unchanged.  A warm-up call on another plan first loads the
    kernels and the scratch array itself (module loading, not the call's own allocation)."""
    import torch

    X = torch.from_numpy(inputs.gaussian_mixture(60000, 3, 10, 0.05, seed=31)).cuda()
    w = torch.from_numpy(inputs.normal_weights(60000, 11, seed=32)).cuda()
    y = torch.empty_like(w)
    warm = fkt.Plan(X, "matern32", lengthscale=0.2, p=6, leaf_size=256, theta=0.5)
    warm.set_option("far_precision", far_precision)
    fkt.fkt_mvm_noalloc(warm.h, w, y, 11)
    torch.cuda.synchronize()
    want = y.cpu().numpy()
    warm.close()
    plan = fkt.Plan(X, "matern32", lengthscale=0.2, p=6, leaf_size=256, theta=0.5)
    plan.set_option("far_precision", far_precision)
    y.fill_(float("nan"))
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    fkt.fkt_mvm_noalloc(plan.h, w, y, 11)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before, (free_before, free_after)
    assert _rel(y.cpu().numpy(), want) < TOL
    plan.close()


def test_noalloc_rejects_requests_beyond_its_scratch(fkt):
    import torch

    n = 300000                                        # 64 right-hand sides need > 48 MiB
    X = torch.from_numpy(inputs.uniform_cube(n, 3, seed=24)).cuda()
    plan = fkt.Plan(X, "gaussian", lengthscale=0.1, p=2, leaf_size=512, theta=0.5)
    w = torch.zeros((64, n), device="cuda")
    y = torch.zeros_like(w)
    with pytest.raises(fkt.FktError) as e:
        fkt.fkt_mvm_noalloc(plan.h, w, y, 64)
    assert e.value.status == fkt.FKT_ERR_SCRATCH_LIMIT
    plan.close()
