"""The target-sharded product (multi-GPU form of Algorithm 1) on CPU ranks, with the float64
oracle as each rank's arithmetic and gloo as the exchange (world sizes 2 and 3).  No GPU.

Each rank takes a contiguous range of target blocks (128 consecutive targets of one leaf, in
tree order) from the library's own partition (fkt_shard_partition, host only), computes the
partial multipoles of the sources in its range (the oracle's s2m with the weights outside the
range set to zero), sums them over the ranks with one allreduce, and evaluates its own targets
with the summed multipoles and the full weights.  The assembled product must equal the
single-process oracle product: every target is evaluated exactly once, and the partial
multipoles add up to the full ones (s2m is linear in the weights)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2106_04487_gb300 import inputs

N, P, LEAF, THETA = 4000, 4, 64, 0.5
KERNEL = ("matern32", 0.2)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _blocks(tree):
    """Target blocks as the library forms them: each leaf (in tree order) cut into 128s."""
    out = []
    for b in np.nonzero(tree["leaf"])[0]:
        for lo in range(int(tree["begin"][b]), int(tree["end"][b]), 128):
            out.append((lo, min(lo + 128, int(tree["end"][b]))))
    return sorted(out)


def _work(F, tree, blocks):
    """Near pairs + 50 x far pairs of each block (the weights of fkt_shard_block_work)."""
    size = tree["end"] - tree["begin"]
    w = []
    for lo, hi in blocks:
        tot = 0.0
        for t in range(lo, hi):
            far, near = F.target_lists(int(tree["perm"][t]))
            tot += 50.0 * len(far) + float(size[near].sum())
        w.append(tot)
    return np.array(w)


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_2106_04487_gb300 import fkt

        X = inputs.gaussian_mixture(N, 3, 5, 0.08, seed=61)
        W = inputs.normal_weights(N, 3, seed=62).astype(np.float64)
        F = O.FKT(X, O.kparams(*KERNEL), P, LEAF, THETA)
        tree = F.tree()
        blocks = _blocks(tree)
        work = _work(F, tree, blocks)
        bounds = fkt.fkt_shard_partition(work, world)
        b0, b1 = int(bounds[rank]), int(bounds[rank + 1])
        lo, hi = (blocks[b0][0], blocks[b1 - 1][1]) if b1 > b0 else (0, 0)
        own = tree["perm"][lo:hi]
        Wr = np.zeros_like(W)
        Wr[:, own] = W[:, own]                 # this rank's sources
        F.s2m(Wr)
        M = torch.from_numpy(F.multipoles())
        dist.all_reduce(M)                     # the one exchange: sum of the partial multipoles
        F.s2m(W)                               # every rank reads all weights in its near field
        F.set_multipoles(M.numpy())
        q.put((rank, lo, hi, F.eval(own), bounds.tolist(), float(work[b0:b1].sum()), float(work.sum())))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_product_equals_single_process(orc, world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, qu)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((qu.get(timeout=280) for _ in range(world)), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    X = inputs.gaussian_mixture(N, 3, 5, 0.08, seed=61)
    W = inputs.normal_weights(N, 3, seed=62)
    F = orc.FKT(X, orc.kparams(*KERNEL), P, LEAF, THETA)
    perm = F.tree()["perm"]
    want = F.mvm(W, perm)                      # the single-process product in tree order
    # the ranks' target ranges tile [0, N) in order, so every target is evaluated exactly once
    assert [o[1] for o in out][0] == 0 and out[-1][2] == N
    assert all(out[i][2] == out[i + 1][1] for i in range(world - 1))
    got = np.concatenate([o[3] for o in out], axis=1)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12 * np.abs(want).max())
    # the partition balances the work to within one block's share
    total = out[0][6]
    assert max(o[5] for o in out) <= total / world * 1.25


def test_partition_is_contiguous_and_balanced():
    from paper_2106_04487_gb300 import fkt

    rng = np.random.default_rng(0)
    w = rng.exponential(1.0, 5000)
    for n in (1, 2, 3, 8, 152):
        b = fkt.fkt_shard_partition(w, n)
        assert b[0] == 0 and b[-1] == len(w) and np.all(np.diff(b) >= 0)
        loads = np.array([w[b[i]:b[i + 1]].sum() for i in range(n)])
        assert loads.max() <= w.sum() / n + w.max()


def test_partition_edge_cases():
    from paper_2106_04487_gb300 import fkt

    assert fkt.fkt_shard_partition(np.ones(3), 5).tolist() in ([0, 0, 1, 2, 3, 3], [0, 1, 1, 2, 3, 3],
                                                               [0, 1, 2, 2, 3, 3], [0, 1, 2, 3, 3, 3],
                                                               [0, 0, 1, 1, 2, 3], [0, 1, 1, 2, 2, 3])
    assert fkt.fkt_shard_partition(np.zeros(4), 2).tolist()[-1] == 4
    assert fkt.fkt_shard_partition(np.zeros(0), 3).tolist() == [0, 0, 0, 0]
    for bad in (np.array([1.0, -1.0]), np.array([np.nan])):
        with pytest.raises(fkt.FktError):
            fkt.fkt_shard_partition(bad, 2)
    with pytest.raises(fkt.FktError):
        fkt.fkt_shard_partition(np.ones(3), 0)
