"""The target-sharded product (fkt_shard_set, fkt_mvm_shard_begin / _end) on one GPU, with the
ranks run one after the other and the exchange (the allreduce of the partial multipoles) done as
a sum of the ranks' arrays on the device.  The assembled product must match the single-process
fkt_mvm (same kernels; only the order of the multipole sums differs) and the float64 oracle."""
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


@pytest.mark.parametrize("nranks,nrhs,far,near", [(2, 11, "fp32", "fp32"), (3, 32, "bf16x3", "tf32x3"),
                                                  (4, 1, "fp32", "fp32")])
def test_sharded_product_matches_single_process(fkt, orc, nranks, nrhs, far, near):
    import torch

    n = 60000
    X = inputs.gaussian_mixture(n, 3, 10, 0.05, seed=71)
    W = inputs.normal_weights(n, nrhs, seed=72)
    Xd, Wd = torch.from_numpy(X).cuda(), torch.from_numpy(W).cuda()

    def plan():
        p = fkt.Plan(Xd, "matern32", lengthscale=0.2, p=6, leaf_size=256, theta=0.5)
        p.set_option("far_precision", far)
        p.set_option("near_precision", near)
        return p

    ranks = [plan() for _ in range(nranks)]
    infos = [ranks[r].shard_set(nranks, r) for r in range(nranks)]
    # the ranks' block and target ranges tile the whole problem in order
    assert infos[0]["block_lo"] == 0 and infos[0]["target_lo"] == 0
    assert infos[-1]["target_hi"] == n and infos[-1]["block_hi"] == ranks[0].stats()["target_blocks"]
    for a, b in zip(infos, infos[1:]):
        assert a["block_hi"] == b["block_lo"] and a["target_hi"] == b["target_lo"]
    work = ranks[0].block_work()
    bounds = fkt.fkt_shard_partition(work, nranks)
    assert [i["block_lo"] for i in infos] == bounds[:-1].tolist()
    mult = [ranks[r].shard_begin(Wd) for r in range(nranks)]
    total = torch.stack(mult).sum(0)                    # the allreduce
    y = torch.full_like(Wd, float("nan"))
    for r in range(nranks):
        ranks[r].shard_end(total, y)
    torch.cuda.synchronize()
    for r in ranks:
        r.check()
    y = y.cpu().numpy().astype(np.float64)
    assert np.isfinite(y).all()                         # every target written by its rank
    single = plan()
    want = single.mvm(Wd).cpu().numpy().astype(np.float64)
    # same arithmetic up to the order of the multipole sums and, for one right-hand side, the
    # kernel widths (the single-process product runs its 1-wide kernels, the sharded one 8-wide):
    # float32 rounding, within the float32 parity bar
    e2, einf = assert_bars(y, want, 1e-5, f"{nranks} ranks vs fkt_mvm")
    idx = inputs.subsample(n, 300, seed=73)
    z = orc.FKT(X, orc.kparams("matern32", 0.2), p=6, leaf_size=256, theta=0.5).mvm(W, idx)
    assert_bars(y[:, idx], z, 3e-5 if far == "bf16x3" else 1e-5, f"{nranks} ranks vs oracle")
    print(f"{nranks} ranks ({far}/{near}, nrhs {nrhs}): vs fkt_mvm {e2:.1e} / {einf:.1e}; rank work "
          f"{[float(work[i['block_lo']:i['block_hi']].sum() / work.sum()) for i in infos]}")
