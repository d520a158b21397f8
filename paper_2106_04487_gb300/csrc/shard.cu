// Target-sharded product over several processes (one GPU each): the host side.
//
// Every rank builds the same plan (the tree and lists are deterministic) from all the points.
// The targets are partitioned into contiguous ranges of target blocks in target (tree, Morton) order,
// balanced by the block's work: its near pairs plus kFarPairCost times its far pairs (the
// per-target decisions of Sec. 3.1 are unchanged, so every (target, source) pair is still
// evaluated exactly once, by the rank owning the target).  Rank r owns the sources in its target
// range too: its s2m items are the plan's items cut to that range, so the ranks' partial
// multipoles sum to the full ones (s2m is linear in the weights, Algorithm 1).  The one exchange
// is that sum (an allreduce by the caller between fkt_mvm_shard_begin and fkt_mvm_shard_end);
// w is needed in full on every rank (the near field reads any source).
#include <algorithm>
#include <vector>

#include "fkt_internal.h"

namespace fkt {

// Relative cost of one (target, far node) pair against one near pair: the far basis row of
// order p costs a few hundred lane operations against about ten for a near pair (measured at the
// 1M-point Matern workload, p = 6: 20.8 ms for 2.5e8 far pairs, 18.5 ms for 1.3e10 near pairs).
constexpr double kFarPairCost = 50.0;

int shard_partition(int64_t nblocks, const double* work, int nranks, int64_t* bounds) {
    if (nblocks < 0 || nranks < 1 || !bounds || (nblocks > 0 && !work)) return FKT_ERR_INVALID_ARG;
    double total = 0.0;
    for (int64_t b = 0; b < nblocks; ++b) {
        if (!(work[b] >= 0.0)) return FKT_ERR_INVALID_ARG;
        total += work[b];
    }
    // rank r takes the blocks whose cumulative work midpoint falls in [r, r+1) * total / nranks
    bounds[0] = 0;
    double acc = 0.0;
    int r = 1;
    for (int64_t b = 0; b < nblocks && r < nranks; ++b) {
        const double mid = acc + 0.5 * work[b];
        while (r < nranks && mid >= total * r / nranks) bounds[r++] = b;
        acc += work[b];
    }
    while (r < nranks) bounds[r++] = nblocks;
    bounds[nranks] = nblocks;
    for (int i = 0; i < nranks; ++i)
        if (bounds[i + 1] < bounds[i]) bounds[i + 1] = bounds[i];
    return FKT_OK;
}

static int popc4(const uint32_t* m) {
    return __builtin_popcount(m[0]) + __builtin_popcount(m[1]) + __builtin_popcount(m[2]) + __builtin_popcount(m[3]);
}

// The work of every target block, in target order (blocks sorted by their first target: the
// plan enumerates them leaf by leaf, which is not the targets' tree order); order[i] = the
// block index of the i-th block in that order.
int shard_block_work(fkt_plan_s* P, std::vector<double>& work, std::vector<int32_t>* order_out) {
    const int64_t nb = P->nblocks, nn = P->nnodes;
    std::vector<int2> blk(nb), far_ent(P->nfar), near_ent(P->nnear);
    std::vector<int64_t> far_off(nb + 1), near_off(nb + 1);
    std::vector<uint32_t> masks((size_t)std::max<int64_t>(P->nmasks, 1) * kMaskWords);
    std::vector<int32_t> beg(nn), end(nn);
    FKT_CUDA_TRY(cudaStreamSynchronize(P->stream));
    FKT_CUDA_TRY(cudaMemcpy(blk.data(), P->blk_range, sizeof(int2) * nb, cudaMemcpyDeviceToHost));
    FKT_CUDA_TRY(cudaMemcpy(far_off.data(), P->far_off, 8 * (nb + 1), cudaMemcpyDeviceToHost));
    FKT_CUDA_TRY(cudaMemcpy(near_off.data(), P->near_off, 8 * (nb + 1), cudaMemcpyDeviceToHost));
    if (P->nfar) FKT_CUDA_TRY(cudaMemcpy(far_ent.data(), P->far_ent, sizeof(int2) * P->nfar, cudaMemcpyDeviceToHost));
    if (P->nnear) FKT_CUDA_TRY(cudaMemcpy(near_ent.data(), P->near_ent, sizeof(int2) * P->nnear, cudaMemcpyDeviceToHost));
    if (P->nmasks)
        FKT_CUDA_TRY(cudaMemcpy(masks.data(), P->masks, 4 * kMaskWords * P->nmasks, cudaMemcpyDeviceToHost));
    FKT_CUDA_TRY(cudaMemcpy(beg.data(), P->nd_begin, 4 * nn, cudaMemcpyDeviceToHost));
    FKT_CUDA_TRY(cudaMemcpy(end.data(), P->nd_end, 4 * nn, cudaMemcpyDeviceToHost));
    std::vector<int32_t> order(nb);
    for (int64_t b = 0; b < nb; ++b) order[b] = (int32_t)b;
    std::sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return blk[x].x < blk[y].x; });
    work.assign(nb, 0.0);
    for (int64_t ib = 0; ib < nb; ++ib) {
        const int64_t b = order[ib];
        const int64_t nt = blk[b].y - blk[b].x;
        double w = 0.0;
        for (int64_t e = far_off[b]; e < far_off[b + 1]; ++e)
            w += kFarPairCost * (far_ent[e].y < 0 ? nt : popc4(&masks[(size_t)far_ent[e].y * kMaskWords]));
        for (int64_t e = near_off[b]; e < near_off[b + 1]; ++e) {
            const int leaf = near_ent[e].x;
            const int64_t nt_on = near_ent[e].y < 0 ? nt : popc4(&masks[(size_t)near_ent[e].y * kMaskWords]);
            w += (double)nt_on * (end[leaf] - beg[leaf]);
        }
        work[ib] = w;
    }
    if (order_out) *order_out = std::move(order);
    return FKT_OK;
}

void free_shard(fkt_plan_s* P) {
    cudaFree(P->sh_items);
    cudaFree(P->sh_item_off);
    cudaFree(P->sh_blocks);
    P->sh_items = nullptr;
    P->sh_item_off = nullptr;
    P->sh_blocks = nullptr;
    P->sh_nranks = 0;
}

int shard_set(fkt_plan_s* P, int nranks, int rank) {
    if (P->nprob) return FKT_ERR_UNSUPPORTED;
    std::vector<double> work;
    std::vector<int32_t> order;
    int rc = shard_block_work(P, work, &order);
    if (rc) return rc;
    std::vector<int64_t> bounds(nranks + 1);
    if ((rc = shard_partition(P->nblocks, work.data(), nranks, bounds.data()))) return rc;
    const int64_t b0 = bounds[rank], b1 = bounds[rank + 1];
    int64_t t0 = 0, t1 = 0;
    if (b1 > b0) {  // the rank's blocks, consecutive in target order, tile [t0, t1)
        int2 lo, hi;
        FKT_CUDA_TRY(cudaMemcpy(&lo, P->blk_range + order[b0], sizeof(int2), cudaMemcpyDeviceToHost));
        FKT_CUDA_TRY(cudaMemcpy(&hi, P->blk_range + order[b1 - 1], sizeof(int2), cudaMemcpyDeviceToHost));
        t0 = lo.x;
        t1 = hi.y;
    }
    // the plan's s2m items cut to the rank's sources [t0, t1)
    const int64_t nn = P->nnodes, ni = P->n_s2m_items;
    std::vector<int4> items(ni);
    std::vector<int64_t> off(nn + 1);
    if (ni) FKT_CUDA_TRY(cudaMemcpy(items.data(), P->s2m_items, sizeof(int4) * ni, cudaMemcpyDeviceToHost));
    FKT_CUDA_TRY(cudaMemcpy(off.data(), P->s2m_item_off, 8 * (nn + 1), cudaMemcpyDeviceToHost));
    std::vector<int4> mine;
    std::vector<int64_t> moff(nn + 1, 0);
    for (int64_t n = 0; n < nn; ++n) {
        moff[n] = (int64_t)mine.size();
        for (int64_t i = off[n]; i < off[n + 1]; ++i) {
            const int lo = (int)std::max<int64_t>(items[i].y, t0), hi = (int)std::min<int64_t>(items[i].z, t1);
            if (lo < hi) mine.push_back(make_int4(items[i].x, lo, hi, 0));
        }
    }
    moff[nn] = (int64_t)mine.size();
    free_shard(P);
    FKT_CUDA_TRY(cudaMalloc(&P->sh_items, sizeof(int4) * (mine.size() + 1)));
    FKT_CUDA_TRY(cudaMalloc(&P->sh_item_off, 8 * (nn + 1)));
    if (!mine.empty())
        FKT_CUDA_TRY(cudaMemcpy(P->sh_items, mine.data(), sizeof(int4) * mine.size(), cudaMemcpyHostToDevice));
    FKT_CUDA_TRY(cudaMemcpy(P->sh_item_off, moff.data(), 8 * (nn + 1), cudaMemcpyHostToDevice));
    FKT_CUDA_TRY(cudaMalloc(&P->sh_blocks, sizeof(int32_t) * std::max<int64_t>(b1 - b0, 1)));
    if (b1 > b0)
        FKT_CUDA_TRY(cudaMemcpy(P->sh_blocks, order.data() + b0, sizeof(int32_t) * (b1 - b0), cudaMemcpyHostToDevice));
    P->sh_nranks = nranks;
    P->sh_rank = rank;
    P->sh_b0 = b0;
    P->sh_b1 = b1;
    P->sh_t0 = t0;
    P->sh_t1 = t1;
    P->sh_nitems = (int64_t)mine.size();
    return FKT_OK;
}

}  // namespace fkt
