"""Failure detection on the GPU without a GPU fault.

Every wait of the tensor-core kernels is bounded: one that runs out records FKT_ERR_TIMEOUT in
the plan's error word, drains the copies and MMAs its CTA issued, frees its tensor memory and
returns, so the context stays usable.  Here the pipeline waits (a copy landing, the hand-off of
a chunk or entry to the MMA issuer) get a limit of a single poll (option wait_limit_cycles = 0),
so they run out on valid work; nothing hangs and no kernel faults.  The test checks that
fkt_check reports the timeout and clears it, and that the next product with the normal limit
matches the float64 oracle FKT.
"""
import numpy as np
import pytest

from bars import assert_bars
from paper_2106_04487_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fkt():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_04487_gb300 import build, fkt as F

    build.build()
    F.lib()
    return F


@pytest.mark.parametrize("near,far", [("tf32x3", "fp32"), ("fp32", "bf16x3")])
def test_wait_timeout_is_reported_cleared_and_recovered(fkt, orc, near, far):
    import torch

    X = inputs.gaussian_mixture(5000, 3, 5, 0.08, seed=41)
    W = inputs.normal_weights(5000, 32, seed=42)
    plan = fkt.Plan(torch.from_numpy(X).cuda(), "matern32", lengthscale=0.2, p=6, leaf_size=128, theta=0.5)
    s = plan.stats()
    assert s["far_pairs"] > 0 and s["near_pairs"] > 0
    plan.set_option("near_precision", near)
    plan.set_option("far_precision", far)
    Wd = torch.from_numpy(W).cuda()
    plan.set_option("wait_limit_cycles", "0")
    plan.mvm(Wd)
    assert fkt.lib().fkt_check(plan.h) == fkt.FKT_ERR_TIMEOUT
    assert fkt.lib().fkt_check(plan.h) == fkt.FKT_OK          # the record was cleared
    plan.set_option("wait_limit_cycles", "default")
    y = plan.mvm(Wd).cpu().numpy().astype(np.float64)
    assert fkt.lib().fkt_check(plan.h) == fkt.FKT_OK
    plan.close()
    z = orc.FKT(X, orc.kparams("matern32", 0.2), p=6, leaf_size=128, theta=0.5).mvm(W)
    assert_bars(y, z, 3e-5, f"near {near}, far {far} after a timeout")


def test_wait_limit_option_rejects_bad_values(fkt):
    import torch

    plan = fkt.Plan(torch.from_numpy(inputs.uniform_cube(500, 3)).cuda(), "gaussian", lengthscale=0.1, p=2,
                    leaf_size=64, theta=0.5)
    for bad in ("-1", "x", "", "3000000000"):
        with pytest.raises(fkt.FktError):
            plan.set_option("wait_limit_cycles", bad)
    plan.set_option("wait_limit_cycles", "1000")
    plan.set_option("wait_limit_cycles", "default")
    plan.close()
