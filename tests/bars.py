"""Parity bars shared by the GPU tests (not a test module).

Two bars per comparison of the GPU product y with the float64 oracle z on sampled targets:
  * per right-hand side, the relative 2-norm  |y_r - z_r|_2 / |z_r|_2;
  * per target, the element-wise bound  max_t |y_rt - z_rt| / |z_r|_inf,
    so that a wrong result confined to a few targets (one 32-target warp of one mask word,
    one 128-target block) cannot hide under a 2-norm over hundreds of samples.
Both are maxima over right-hand sides.
"""
from __future__ import annotations

import numpy as np


def rel_2norm(y, z) -> float:
    y, z = np.atleast_2d(y), np.atleast_2d(z)
    return max(float(np.linalg.norm(y[r] - z[r]) / np.linalg.norm(z[r])) for r in range(len(z)))


def rel_elementwise(y, z) -> float:
    y, z = np.atleast_2d(y), np.atleast_2d(z)
    return max(float(np.max(np.abs(y[r] - z[r])) / np.max(np.abs(z[r]))) for r in range(len(z)))


def assert_bars(y, z, tol, what=""):
    """Both bars at the same tolerance; returns (2-norm, element-wise) for printing."""
    e2, einf = rel_2norm(y, z), rel_elementwise(y, z)
    assert e2 < tol, f"{what}: per-RHS relative 2-norm {e2:.3e} >= {tol:g}"
    assert einf < tol, f"{what}: per-target max |y - z| / |z|_inf {einf:.3e} >= {tol:g}"
    return e2, einf


def partly_masked_targets(lists: dict, count: int, seed: int = 0) -> np.ndarray:
    """Sorted target positions that sit in partly-active warps: 32-target groups of a block in
    which an interaction-list entry (far node or near leaf) is taken by some, but not all, of the
    group's targets.  These are the targets whose results depend on the per-lane masking of the
    kernels (disabled MMA rows, masked kernel values).  Returns up to `count` distinct positions,
    half of them inside the entry's mask and half outside."""
    rng = np.random.default_rng(seed)
    br = lists["block_range"]
    sizes = (br[:, 1] - br[:, 0]).astype(np.int64)
    masks = lists["masks"]
    picks = []
    for off_key, msk_key in (("far_off", "far_mask"), ("near_off", "near_mask")):
        off, msk = lists[off_key], lists[msk_key]
        blk = np.repeat(np.arange(len(br)), np.diff(off))
        sel = np.nonzero(msk >= 0)[0]
        if len(sel) == 0:
            continue
        words = masks[msk[sel]].astype(np.uint64)                      # [entries][4]
        n = sizes[blk[sel]]
        lanes = np.clip(n[:, None] - 32 * np.arange(4)[None, :], 0, 32)  # valid lanes per word
        full = np.where(lanes >= 32, np.uint64(0xFFFFFFFF), (np.uint64(1) << lanes.astype(np.uint64)) - np.uint64(1))
        part = (words != 0) & (words != full)
        ent, wd = np.nonzero(part)
        if len(ent) == 0:
            continue
        take = rng.choice(len(ent), size=min(len(ent), count), replace=False)
        for j, i in enumerate(take):
            e, w = ent[i], wd[i]
            word = int(words[e, w])
            nl = int(lanes[e, w])
            inside = [l for l in range(nl) if (word >> l) & 1]
            outside = [l for l in range(nl) if not (word >> l) & 1]
            pool = inside if (j % 2 == 0 and inside) or not outside else outside
            lane = int(rng.choice(pool))
            picks.append(int(br[blk[sel[e]], 0]) + 32 * int(w) + lane)
    picks = np.unique(np.asarray(picks, dtype=np.int64))
    if len(picks) > count:
        picks = np.sort(rng.choice(picks, size=count, replace=False))
    return picks
