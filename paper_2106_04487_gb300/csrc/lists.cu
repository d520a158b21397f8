// Interaction lists (Sec. 3.1-3.2): for every target point t the far set is the set of
// nodes b reached from the root with rho_b / |x_t - c_b| < theta (eq. accparam), not
// descending below an accepted node (F_i disjoint along ancestor chains), and the near
// set is the leaves reached without acceptance (N_l of Sec. 3.2).
//
// Targets are grouped in blocks of <= 128 consecutive sorted points of one leaf.  One
// warp walks the tree for a block with a 128-bit "active" mask (targets that have not
// accepted an ancestor).  Per node the warp first classifies with the block's bounding
// sphere (all far / none far, with a 1e-12 relative safety margin); only nodes in the
// uncertain shell evaluate the exact per-target predicate
//     rho2_b < theta^2 * |x_t - c_b|^2       (float64, explicit round-to-nearest)
// so every decision is the one the per-point rule makes.  Entries carry a mask index
// (-1 when the entry applies to the whole block).  A count pass sizes the arrays, an
// exclusive scan places each block, and a fill pass writes them.
#include <cub/cub.cuh>

#include <vector>

#include "fkt_internal.h"

namespace fkt {
namespace {

constexpr int kStack = 160;       // DFS stack per warp (>= 2 * max depth + 2)
constexpr int kWarpsPerCta = 4;

struct ListCounts {
    int32_t nfar, nnear, nmask;
    int32_t pad;
};

__device__ __forceinline__ double d2_exact(const double* x, const double* c, int d) {
    double dx = __dsub_rn(x[0], c[0]);
    double acc = __dmul_rn(dx, dx);
    dx = __dsub_rn(x[1], c[1]);
    acc = __dadd_rn(acc, __dmul_rn(dx, dx));
    dx = __dsub_rn(x[2], c[2]);
    acc = __dadd_rn(acc, __dmul_rn(dx, dx));
    if (d == 4) {
        dx = __dsub_rn(x[3], c[3]);
        acc = __dadd_rn(acc, __dmul_rn(dx, dx));
    }
    return acc;
}

// FILL = false: count entries per block.  FILL = true: write them at the scanned offsets.
template <bool FILL>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
lists_kernel(int64_t nblocks, const int2* __restrict__ blk, const int32_t* __restrict__ blk_leaf,
             const float4* __restrict__ xs, int d, double theta, double theta2, const double* __restrict__ centre,
             const double* __restrict__ rho2, const int32_t* __restrict__ leaf, const int32_t* __restrict__ child,
             const int32_t* __restrict__ nd_begin, const int32_t* __restrict__ nd_end, ListCounts* counts,
             const int64_t* __restrict__ far_off, const int64_t* __restrict__ near_off,
             const int64_t* __restrict__ mask_off, int2* far_ent, int2* near_ent, uint32_t* masks, int32_t* used,
             unsigned long long* pair_stats, int* err) {
    __shared__ int32_t s_node[kWarpsPerCta][kStack];
    __shared__ uint32_t s_act[kWarpsPerCta][kStack][kMaskWords];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t bi = (int64_t)blockIdx.x * kWarpsPerCta + warp;
    if (bi >= nblocks) return;
    const int2 r = blk[bi];
    const int nt = r.y - r.x;
    // this lane's targets: t = lane + 32 w
    double tx[kMaskWords][4];
    uint32_t valid[kMaskWords];
    const int lf = blk_leaf[bi];
    double cT[4];
    for (int a = 0; a < 4; ++a) cT[a] = centre[lf * 4 + a];
    double rT = 0.0;
    for (int w = 0; w < kMaskWords; ++w) {
        int t = lane + 32 * w;
        bool ok = t < nt;
        valid[w] = __ballot_sync(0xffffffffu, ok);
        float4 x = ok ? xs[r.x + t] : make_float4(0.f, 0.f, 0.f, 0.f);
        tx[w][0] = x.x; tx[w][1] = x.y; tx[w][2] = x.z; tx[w][3] = x.w;
        if (ok) rT = fmax(rT, sqrt(d2_exact(tx[w], cT, d)));
    }
    for (int off = 16; off; off >>= 1) rT = fmax(rT, __shfl_xor_sync(0xffffffffu, rT, off));
    int32_t nfar = 0, nnear = 0, nmask = 0;
    int64_t fo = 0, no = 0, mo = 0;
    if (FILL) { fo = far_off[bi]; no = near_off[bi]; mo = mask_off[bi]; }
    unsigned long long far_pairs = 0, near_pairs = 0;
    int sp = 0;
    if (lane == 0) {
        s_node[warp][0] = 0;
        for (int w = 0; w < kMaskWords; ++w) s_act[warp][0][w] = valid[w];
    }
    sp = 1;
    __syncwarp();
    const double margin_lo = 1.0 - 1e-12, margin_hi = 1.0 + 1e-12;
    while (sp > 0) {
        --sp;
        const int b = s_node[warp][sp];
        uint32_t act[kMaskWords];
        for (int w = 0; w < kMaskWords; ++w) act[w] = s_act[warp][sp][w];
        __syncwarp();
        double c[4];
        for (int a = 0; a < 4; ++a) c[a] = centre[b * 4 + a];
        const double rb2 = rho2[b];
        double dist = sqrt(d2_exact(cT, c, d));
        double rb = sqrt(rb2);
        uint32_t F[kMaskWords], R[kMaskWords];
        if (rb * margin_hi < theta * (dist - rT) * margin_lo) {          // every target far
            for (int w = 0; w < kMaskWords; ++w) { F[w] = act[w]; R[w] = 0; }
        } else if (rb * margin_lo > theta * (dist + rT) * margin_hi) {   // no target far
            for (int w = 0; w < kMaskWords; ++w) { F[w] = 0; R[w] = act[w]; }
        } else {
            for (int w = 0; w < kMaskWords; ++w) {
                bool on = (act[w] >> lane) & 1u;
                bool far = on && (rb2 < __dmul_rn(theta2, d2_exact(tx[w], c, d)));
                F[w] = __ballot_sync(0xffffffffu, far);
                R[w] = act[w] & ~F[w];
            }
        }
        bool anyF = false, anyR = false, fullF = true, fullR = true;
        int popF = 0, popR = 0;
        for (int w = 0; w < kMaskWords; ++w) {
            anyF |= F[w] != 0;
            anyR |= R[w] != 0;
            fullF &= F[w] == valid[w];
            fullR &= R[w] == valid[w];
            popF += __popc(F[w]);
            popR += __popc(R[w]);
        }
        const bool isleaf = leaf[b] != 0;
        if (anyF) {
            if (lane == 0) {
                int mi = -1;
                if (!fullF) {
                    mi = (int)(mo + nmask);
                    if (FILL)
                        for (int w = 0; w < kMaskWords; ++w) masks[(int64_t)mi * kMaskWords + w] = F[w];
                    ++nmask;
                }
                if (FILL) {
                    far_ent[fo + nfar] = make_int2(b, mi);
                    used[b] = 1;
                }
                ++nfar;
                far_pairs += popF;
            }
        }
        if (anyR) {
            if (isleaf) {
                if (lane == 0) {
                    int mi = -1;
                    if (!fullR) {
                        mi = (int)(mo + nmask);
                        if (FILL)
                            for (int w = 0; w < kMaskWords; ++w) masks[(int64_t)mi * kMaskWords + w] = R[w];
                        ++nmask;
                    }
                    if (FILL) near_ent[no + nnear] = make_int2(b, mi);
                    ++nnear;
                    near_pairs += (unsigned long long)popR * (unsigned long long)(nd_end[b] - nd_begin[b]);
                }
            } else {
                const int c0 = child[2 * b], c1 = child[2 * b + 1];
                if (sp + 2 > kStack) {  // cannot happen for depth <= 64; report instead of overflowing
                    if (lane == 0) atomicExch(err, 1);
                    break;
                }
                if (lane == 0) {
                    if (c1 >= 0) {
                        s_node[warp][sp] = c1;
                        for (int w = 0; w < kMaskWords; ++w) s_act[warp][sp][w] = R[w];
                    }
                    int sp2 = sp + (c1 >= 0);
                    if (c0 >= 0) {
                        s_node[warp][sp2] = c0;
                        for (int w = 0; w < kMaskWords; ++w) s_act[warp][sp2][w] = R[w];
                    }
                }
                sp += (c1 >= 0) + (c0 >= 0);
                __syncwarp();
            }
        }
    }
    if (lane == 0) {
        if (!FILL) counts[bi] = ListCounts{nfar, nnear, nmask, 0};
        else {
            atomicAdd(&pair_stats[0], far_pairs);
            atomicAdd(&pair_stats[1], near_pairs);
        }
    }
}

__global__ void blocks_per_leaf_kernel(const int32_t* __restrict__ leaf, const int32_t* __restrict__ b,
                                       const int32_t* __restrict__ e, int64_t nn, int32_t* nb) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    nb[i] = leaf[i] ? (e[i] - b[i] + kTB - 1) / kTB : 0;
}

__global__ void emit_blocks_kernel(const int32_t* __restrict__ leaf, const int32_t* __restrict__ b,
                                   const int32_t* __restrict__ e, int64_t nn, const int32_t* __restrict__ nb,
                                   const int32_t* __restrict__ off, int2* blk, int32_t* blk_leaf) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nn || !leaf[i]) return;
    for (int k = 0; k < nb[i]; ++k) {
        int lo = b[i] + k * kTB;
        blk[off[i] + k] = make_int2(lo, min(lo + kTB, e[i]));
        blk_leaf[off[i] + k] = (int32_t)i;
    }
}

__global__ void unpack_counts_kernel(const ListCounts* c, int64_t n, int64_t* f, int64_t* nr, int64_t* m) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    f[i] = c[i].nfar;
    nr[i] = c[i].nnear;
    m[i] = c[i].nmask;
}

// s2m work: each used node is split into chunks of <= kS2MChunk points.
constexpr int kS2MChunk = 1024;

__global__ void s2m_items_count_kernel(const int32_t* __restrict__ used, const int32_t* __restrict__ b,
                                       const int32_t* __restrict__ e, int64_t nn, int64_t* cnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    cnt[i] = used[i] ? (e[i] - b[i] + kS2MChunk - 1) / kS2MChunk : 0;
}

__global__ void s2m_items_emit_kernel(const int32_t* __restrict__ used, const int32_t* __restrict__ b,
                                      const int32_t* __restrict__ e, int64_t nn, const int64_t* __restrict__ off,
                                      int4* items) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nn || !used[i]) return;
    int64_t o = off[i];
    for (int lo = b[i], k = 0; lo < e[i]; lo += kS2MChunk, ++k)
        items[o + k] = make_int4((int)i, lo, min(lo + kS2MChunk, e[i]), 0);
}

template <typename T>
int scan_exclusive(const T* in, T* out, int64_t n, cudaStream_t st) {
    size_t sb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, sb, in, out, (int)n, st);
    void* tmp = nullptr;
    FKT_CUDA_TRY(cudaMalloc(&tmp, sb ? sb : 1));
    FKT_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, sb, in, out, (int)n, st));
    FKT_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(tmp);
    return FKT_OK;
}

}  // namespace

int build_lists(fkt_plan_s* P) {
    cudaStream_t st = P->stream;
    const int64_t nn = P->nnodes;
    int rc;
    // ---- target blocks
    int32_t *nb = nullptr, *nboff = nullptr, *blk_leaf = nullptr;
    FKT_CUDA_TRY(cudaMalloc(&nb, 4 * (nn + 1)));
    FKT_CUDA_TRY(cudaMalloc(&nboff, 4 * (nn + 1)));
    FKT_CUDA_TRY(cudaMemsetAsync(nb, 0, 4 * (nn + 1), st));
    unsigned g = (unsigned)((nn + 255) / 256);
    blocks_per_leaf_kernel<<<g, 256, 0, st>>>(P->nd_leaf, P->nd_begin, P->nd_end, nn, nb);
    if ((rc = scan_exclusive(nb, nboff, nn + 1, st))) return rc;
    int32_t nblk = 0;
    FKT_CUDA_TRY(cudaMemcpy(&nblk, nboff + nn, 4, cudaMemcpyDeviceToHost));
    P->nblocks = nblk;
    FKT_CUDA_TRY(cudaMalloc(&P->blk_range, sizeof(int2) * nblk));
    FKT_CUDA_TRY(cudaMalloc(&blk_leaf, 4 * nblk));
    emit_blocks_kernel<<<g, 256, 0, st>>>(P->nd_leaf, P->nd_begin, P->nd_end, nn, nb, nboff, P->blk_range, blk_leaf);
    FKT_CUDA_TRY(cudaGetLastError());
    // ---- count pass
    ListCounts* counts = nullptr;
    int64_t *cf = nullptr, *cn = nullptr, *cm = nullptr, *mask_off = nullptr;
    int* err = nullptr;
    unsigned long long* pstats = nullptr;
    FKT_CUDA_TRY(cudaMalloc(&counts, sizeof(ListCounts) * nblk));
    FKT_CUDA_TRY(cudaMalloc(&cf, 8 * (nblk + 1)));
    FKT_CUDA_TRY(cudaMalloc(&cn, 8 * (nblk + 1)));
    FKT_CUDA_TRY(cudaMalloc(&cm, 8 * (nblk + 1)));
    FKT_CUDA_TRY(cudaMalloc(&P->far_off, 8 * (nblk + 1)));
    FKT_CUDA_TRY(cudaMalloc(&P->near_off, 8 * (nblk + 1)));
    FKT_CUDA_TRY(cudaMalloc(&mask_off, 8 * (nblk + 1)));
    FKT_CUDA_TRY(cudaMalloc(&err, sizeof(int)));
    FKT_CUDA_TRY(cudaMalloc(&pstats, 2 * sizeof(unsigned long long)));
    FKT_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    FKT_CUDA_TRY(cudaMemsetAsync(pstats, 0, 2 * sizeof(unsigned long long), st));
    FKT_CUDA_TRY(cudaMemsetAsync(cf, 0, 8 * (nblk + 1), st));
    FKT_CUDA_TRY(cudaMemsetAsync(cn, 0, 8 * (nblk + 1), st));
    FKT_CUDA_TRY(cudaMemsetAsync(cm, 0, 8 * (nblk + 1), st));
    const double theta = P->theta, theta2 = P->theta * P->theta;
    unsigned lg = (unsigned)((nblk + kWarpsPerCta - 1) / kWarpsPerCta);
    lists_kernel<false><<<lg, kWarpsPerCta * 32, 0, st>>>(
        nblk, P->blk_range, blk_leaf, P->xs, P->d, theta, theta2, P->nd_centre, P->nd_rho2, P->nd_leaf, P->nd_child,
        P->nd_begin, P->nd_end, counts, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, err);
    FKT_CUDA_TRY(cudaGetLastError());
    unpack_counts_kernel<<<(unsigned)((nblk + 255) / 256), 256, 0, st>>>(counts, nblk, cf, cn, cm);
    if ((rc = scan_exclusive(cf, P->far_off, nblk + 1, st)) || (rc = scan_exclusive(cn, P->near_off, nblk + 1, st)) ||
        (rc = scan_exclusive(cm, mask_off, nblk + 1, st)))
        return rc;
    int64_t tot[3];
    FKT_CUDA_TRY(cudaMemcpy(&tot[0], P->far_off + nblk, 8, cudaMemcpyDeviceToHost));
    FKT_CUDA_TRY(cudaMemcpy(&tot[1], P->near_off + nblk, 8, cudaMemcpyDeviceToHost));
    FKT_CUDA_TRY(cudaMemcpy(&tot[2], mask_off + nblk, 8, cudaMemcpyDeviceToHost));
    P->nfar = tot[0];
    P->nnear = tot[1];
    P->nmasks = tot[2];
    FKT_CUDA_TRY(cudaMalloc(&P->far_ent, sizeof(int2) * (tot[0] + 1)));
    FKT_CUDA_TRY(cudaMalloc(&P->near_ent, sizeof(int2) * (tot[1] + 1)));
    FKT_CUDA_TRY(cudaMalloc(&P->masks, sizeof(uint32_t) * kMaskWords * (tot[2] + 1)));
    // ---- fill pass
    lists_kernel<true><<<lg, kWarpsPerCta * 32, 0, st>>>(
        nblk, P->blk_range, blk_leaf, P->xs, P->d, theta, theta2, P->nd_centre, P->nd_rho2, P->nd_leaf, P->nd_child,
        P->nd_begin, P->nd_end, counts, P->far_off, P->near_off, mask_off, P->far_ent, P->near_ent, P->masks,
        P->nd_used, pstats, err);
    FKT_CUDA_TRY(cudaGetLastError());
    int herr = 0;
    unsigned long long hp[2];
    FKT_CUDA_TRY(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    FKT_CUDA_TRY(cudaMemcpy(hp, pstats, sizeof(hp), cudaMemcpyDeviceToHost));
    if (herr) return FKT_ERR_INTERNAL;
    P->stats.far_pairs = (int64_t)hp[0];
    P->stats.near_pairs = (int64_t)hp[1];
    // ---- s2m work items over the nodes some target uses
    int64_t *icnt = nullptr;
    FKT_CUDA_TRY(cudaMalloc(&icnt, 8 * (nn + 1)));
    FKT_CUDA_TRY(cudaMalloc(&P->s2m_item_off, 8 * (nn + 1)));
    FKT_CUDA_TRY(cudaMemsetAsync(icnt, 0, 8 * (nn + 1), st));
    s2m_items_count_kernel<<<g, 256, 0, st>>>(P->nd_used, P->nd_begin, P->nd_end, nn, icnt);
    if ((rc = scan_exclusive(icnt, P->s2m_item_off, nn + 1, st))) return rc;
    int64_t nitems = 0;
    FKT_CUDA_TRY(cudaMemcpy(&nitems, P->s2m_item_off + nn, 8, cudaMemcpyDeviceToHost));
    P->n_s2m_items = nitems;
    FKT_CUDA_TRY(cudaMalloc(&P->s2m_items, sizeof(int4) * (nitems + 1)));
    s2m_items_emit_kernel<<<g, 256, 0, st>>>(P->nd_used, P->nd_begin, P->nd_end, nn, P->s2m_item_off, P->s2m_items);
    FKT_CUDA_TRY(cudaGetLastError());
    // stats: used nodes and (source, node) pairs
    std::vector<int32_t> hu(nn), hb(nn), he(nn);
    FKT_CUDA_TRY(cudaMemcpy(hu.data(), P->nd_used, 4 * nn, cudaMemcpyDeviceToHost));
    FKT_CUDA_TRY(cudaMemcpy(hb.data(), P->nd_begin, 4 * nn, cudaMemcpyDeviceToHost));
    FKT_CUDA_TRY(cudaMemcpy(he.data(), P->nd_end, 4 * nn, cudaMemcpyDeviceToHost));
    int64_t un = 0, sp = 0;
    for (int64_t i = 0; i < nn; ++i)
        if (hu[i]) { ++un; sp += he[i] - hb[i]; }
    P->stats.s2m_nodes = un;
    P->stats.s2m_pairs = sp;
    cudaFree(icnt);
    cudaFree(nb);
    cudaFree(nboff);
    cudaFree(blk_leaf);
    cudaFree(counts);
    cudaFree(cf);
    cudaFree(cn);
    cudaFree(cm);
    cudaFree(mask_off);
    cudaFree(err);
    cudaFree(pstats);
    return FKT_OK;
}

}  // namespace fkt
