// __global__ kernels of the FKT matrix-vector product (Algorithm 1).
//   permute_kernel   w (caller order) -> sorted weights of one group of NR right-hand sides
//   s2m_kernel       per (node, <=1024-point chunk): partial multipoles (source2mult)
//   s2m_reduce       per node: sum of its chunks' partials (deterministic order)
//   near_kernel      per target block: dense K(near, leaf) * w[leaf] over the near leaves
//                    (also the exact all-pairs product, with the root as the only "near leaf")
//   far_kernel       per target block: m2t * multipole over the far nodes (far_mr_kernel: 8 RHS),
//                    written in tree order; unpermute adds the near field and scatters the sum
//                    back to the caller's order
#pragma once

#include <type_traits>

#include "fkt_kernels.cuh"
#include "ptx.cuh"

namespace fkt {

// Source records for one pass: point (tree order) followed by this pass's weights.
// Coordinates are stored multiplied by sigma = KernelParams::sig so that the near field works
// with distances already in the kernel's own units (see kval).
template <int D, int NR>
__global__ void permute_kernel(int64_t N, const int32_t* __restrict__ perm, const float4* __restrict__ xs,
                               const float* __restrict__ w, int nr, float sig_all, const float* __restrict__ pt_sig,
                               float4* __restrict__ rec) {
    using R = Rec<D, NR>;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t j = perm[i];
    const float sig = pt_sig ? pt_sig[i] : sig_all;
    float v[R::F4 * 4];
    const float4 x = xs[i];
    v[0] = x.x * sig; v[1] = x.y * sig; v[2] = x.z * sig; v[3] = x.w * sig;
#pragma unroll
    for (int q = 4; q < R::F4 * 4; ++q) v[q] = 0.f;
#pragma unroll
    for (int r = 0; r < NR; ++r) v[R::WOFF + r] = r < nr ? __ldg(&w[r * N + j]) : 0.0f;
#pragma unroll
    for (int q = 0; q < R::F4; ++q) rec[i * R::F4 + q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// y[perm[i]] = sum_{s < parts} (ys[s][i] + yadd[s][i]): one right-hand side whose near and far
// fields were split over several CTAs per target block (partial rows summed in a fixed order).
template <int Unused = 0>
__global__ void unpermute_parts_kernel(int64_t N, int parts, const int32_t* __restrict__ perm,
                                       const float* __restrict__ ys, const float* __restrict__ yadd,
                                       float* __restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float v = ys[i], f = yadd[i];
    for (int s = 1; s < parts; ++s) {
        v += ys[s * N + i];
        f += yadd[s * N + i];
    }
    y[perm[i]] = v + f;
}

// y[r][perm[i]] = ys[r][i] (+ yadd[r][i]): back to the caller's order, adding the far field
// to the near field when yadd is given.
template <int Unused = 0>
__global__ void unpermute_kernel(int64_t N, int nr, const int32_t* __restrict__ perm, const float* __restrict__ ys,
                                 const float* __restrict__ yadd, float* __restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t o = perm[i];
    if (yadd)
        for (int r = 0; r < nr; ++r) y[r * N + o] = ys[r * N + i] + yadd[r * N + i];
    else
        for (int r = 0; r < nr; ++r) y[r * N + o] = ys[r * N + i];
}

// ------------------------------------------------------------------- s2m
template <int D, int P, int NR>
struct S2MShape {
    static constexpr int NT = Layout<D, P>::nterms;
    static constexpr int ROW = NT | 1;                  // odd row stride: conflict-free column reads
    static constexpr int WARPS = NT <= 120 ? 4 : 2;
    static constexpr int TPL = (NT + 31) / 32;          // terms per lane
    static constexpr size_t smem_bytes() {
        size_t tile = (size_t)WARPS * 32 * ROW + (size_t)WARPS * 32 * NR;
        size_t red = (size_t)WARPS * NT * NR;
        return sizeof(float) * (tile > red ? tile : red);
    }
};

template <int D, int P, int NR>
__global__ void __launch_bounds__(S2MShape<D, P, NR>::WARPS * 32)
s2m_kernel(MvmArgs a, const __grid_constant__ FarTables T) {
    using Sh = S2MShape<D, P, NR>;
    using Lay = Layout<D, P>;
    constexpr int NT = Sh::NT, ROW = Sh::ROW, WARPS = Sh::WARPS, TPL = Sh::TPL;
    extern __shared__ float smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* tile = smem + warp * 32 * ROW;
    float* wt = smem + WARPS * 32 * ROW + warp * 32 * NR;
    const int4 it = a.s2m_items[blockIdx.x];
    const int node = it.x;
    const float4 c = a.nd_cf[node];
    const float inv_s = 1.0f / a.nd_scale[node];
    // accumulators as pairs of right-hand sides (packed FMA) when NR is even
    constexpr int NP = NR % 2 == 0 ? NR / 2 : NR;
    using Acc = typename std::conditional<NR % 2 == 0, float2, float>::type;
    Acc acc[TPL][NP];
#pragma unroll
    for (int i = 0; i < TPL; ++i)
#pragma unroll
        for (int r = 0; r < NP; ++r) {
            if constexpr (NR % 2 == 0) acc[i][r] = make_float2(0.f, 0.f);
            else acc[i][r] = 0.f;
        }
    for (int base = it.y + warp * 32; base < it.z; base += WARPS * 32) {
        const int s = base + lane;
        const bool ok = s < it.z;
        float4 x = ok ? a.xs[s] : c;
        float x0 = (x.x - c.x) * inv_s, x1 = (x.y - c.y) * inv_s, x2 = (x.z - c.z) * inv_s;
        float x3 = dim_of(D) == 4 ? (x.w - c.w) * inv_s : 0.f;
        float r2_3 = x0 * x0 + x1 * x1 + x2 * x2;
        float r2 = r2_3 + x3 * x3;
        float rp[P / 2 + 1];  // (r'^2)^i
        rp[0] = ok ? 1.f : 0.f;
#pragma unroll
        for (int i = 1; i <= P / 2; ++i) rp[i] = rp[i - 1] * r2;
        solid_harmonics<D, P>(x0, x1, x2, x3, r2_3, r2, T, [&](int k, int h, float Y) {
            const int o = Lay::off(k) + h * Lay::nj(k);
#pragma unroll
            for (int jj = 0; jj < Lay::nj(k); ++jj) tile[lane * ROW + o + jj] = Y * rp[jj];
        });
#pragma unroll
        for (int r = 0; r < NR; ++r)
            wt[lane * NR + r] = (ok && r < a.nr) ? reinterpret_cast<const float*>(a.rec + (int64_t)s * a.rec_f4)[a.woff + r]
                                                 : 0.f;  // records of a narrow pass hold only its nr weights
        __syncwarp();
#pragma unroll 4
        for (int row = 0; row < 32; ++row) {
            Acc wr[NP];
#pragma unroll
            for (int r = 0; r < NP; ++r) {
                if constexpr (NR % 2 == 0) wr[r] = *reinterpret_cast<const float2*>(&wt[row * NR + 2 * r]);
                else wr[r] = wt[row * NR + r];
            }
#pragma unroll
            for (int i = 0; i < TPL; ++i) {
                const int t = lane + 32 * i;
                if (t < NT) {
                    const float b = tile[row * ROW + t];
#pragma unroll
                    for (int r = 0; r < NP; ++r) {
                        if constexpr (NR % 2 == 0) acc[i][r] = __ffma2_rn(make_float2(b, b), wr[r], acc[i][r]);
                        else acc[i][r] = fmaf(b, wr[r], acc[i][r]);
                    }
                }
            }
        }
        __syncwarp();
    }
    __syncthreads();
    float* red = smem;  // [WARPS][NT][NR], reuses the tiles
#pragma unroll
    for (int i = 0; i < TPL; ++i) {
        const int t = lane + 32 * i;
        if (t < NT)
#pragma unroll
            for (int r = 0; r < NP; ++r) {
                if constexpr (NR % 2 == 0) {
                    red[(warp * NT + t) * NR + 2 * r] = acc[i][r].x;
                    red[(warp * NT + t) * NR + 2 * r + 1] = acc[i][r].y;
                } else {
                    red[(warp * NT + t) * NR + r] = acc[i][r];
                }
            }
    }
    __syncthreads();
    float* out = a.part + (int64_t)blockIdx.x * NT * NR;
    for (int q = threadIdx.x; q < NT * NR; q += WARPS * 32) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) v += red[w * NT * NR + q];
        out[q] = v;
    }
}

template <int Unused = 0>
__global__ void s2m_reduce_kernel(int64_t nnodes, const int64_t* __restrict__ item_off, int ntr,
                                  const float* __restrict__ part, float* __restrict__ mult) {
    const int64_t node = blockIdx.x;
    const int64_t i0 = item_off[node], i1 = item_off[node + 1];
    if (i0 == i1) return;
    for (int q = threadIdx.x; q < ntr; q += blockDim.x) {
        float v = 0.f;
        for (int64_t i = i0; i < i1; ++i) v += part[i * ntr + q];
        mult[node * ntr + q] = v;
    }
}

// ----------------------------------------------------------------- near
// Kernel value without the scale factor (applied once per target at the end), with the
// MUFU approximations ex2 / sqrt / rcp / rsqrt.approx.  q is the squared distance in the
// kernel's own units, the coordinates having been multiplied by sigma (KernelParams::sig):
//   Gaussian            sigma^2 = log2(e) / (2 l^2):  K = 2^(-q)
//   exponential/Matern  sigma   = c log2(e):         u = sqrt(q) = c r log2(e), K = poly(u ln2) 2^(-u)
//   Cauchy / RQ         sigma^2 = c1:                K = (1 + q)^(-alpha)
//   Laplace             sigma   = 1:                 K = q^(-1/2), 0 at q = 0
template <int KIND>
__device__ __forceinline__ float kval(float q, const KernelParams& kp) {
    constexpr float kLn2 = 0.69314718055994531f;
    if (KIND == FKT_GAUSSIAN) {
        return ptx::ex2(-q);
    } else if (KIND == FKT_EXPONENTIAL) {
        return ptx::ex2(-ptx::sqrt_approx(q));
    } else if (KIND == FKT_MATERN32) {
        const float u = ptx::sqrt_approx(q);
        return fmaf(u, kLn2, 1.0f) * ptx::ex2(-u);
    } else if (KIND == FKT_MATERN52) {
        const float u = ptx::sqrt_approx(q);
        const float t = u * kLn2;
        return fmaf(t, fmaf(t, 1.0f / 3.0f, 1.0f), 1.0f) * ptx::ex2(-u);
    } else if (KIND == FKT_CAUCHY) {
        return ptx::rcp_approx(1.0f + q);
    } else if (KIND == FKT_RATQUAD) {
        const float b = 1.0f + q;
        return kp.alpha == 1.0f ? ptx::rcp_approx(b) : ptx::ex2(-kp.alpha * ptx::lg2(b));
    } else {
        return q > 0.0f ? ptx::rsqrt_approx(q) : 0.0f;
    }
}


// T targets per thread (128 / T threads per 128-target block); ST-stage ring of CH-point chunks.
// Thread tl owns targets tl + (128 / T) j, so the targets of slot j of one warp form one
// 32-target group -- one word of an entry's mask.  Accumulators hold pairs of right-hand sides
// (float2, packed FMA) when NR >= 4.  Passes of 16 or 32 right-hand sides (SEL) zero the
// kernel value of a target outside an entry's mask instead of keeping a second set of
// per-entry accumulators.
template <int D, int NR, int T>
struct NearShape {
    static constexpr int F4 = Rec<D, NR>::F4;
    static constexpr int THREADS = kTB / T;
    static constexpr int CH = F4 == 1 ? 256 : (F4 >= 9 ? 64 : 128);
    static constexpr int ST = T >= 4 ? 2 : 3;
    static constexpr bool SEL = NR >= 16;
    static constexpr bool PAIRS = NR >= 4;
    static constexpr int NA = PAIRS ? NR / 2 : NR;  // accumulators per target
    using Acc = typename std::conditional<PAIRS, float2, float>::type;
    static constexpr int MINB = 1;
};

__device__ __forceinline__ float2 ffma2(float a, float2 w, float2 c) { return __ffma2_rn(make_float2(a, a), w, c); }

// One staged chunk of n source records against this thread's targets.  Slot j takes part only
// when bit j of JM is set (its warp's 32-target group has an active target for this entry);
// within a slot, act[j] gates the target itself.
template <int D, int KIND, int NR, int T, unsigned JM>
__device__ __forceinline__ void near_chunk(const float4* __restrict__ sb, int n, const float (&tx)[T][4],
                                           const bool (&act)[T], typename NearShape<D, NR, T>::Acc (&acc)[T][NearShape<D, NR, T>::NA],
                                           const KernelParams& kp) {
    using R = Rec<D, NR>;
    using Sh = NearShape<D, NR, T>;
    constexpr int F4 = R::F4;
    auto kvalue = [&](const float4& sx, int j) {
        const float dx = tx[j][0] - sx.x, dy = tx[j][1] - sx.y, dz = tx[j][2] - sx.z;
        float q = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (D == 4) { const float dw = tx[j][3] - sx.w; q = fmaf(dw, dw, q); }
        return kval<KIND>(q, kp);
    };
    if constexpr (Sh::SEL) {
        // One kernel value per (target, source) serves all NR right-hand sides.  Sources go in
        // batches of KB: the KB kernel values (independent dependency chains through the MUFU)
        // first, then the packed FMAs, so that neither waits on the other's latency.
        constexpr int KB = 8;
        auto fmas = [&](int i, const float (&kv)[T]) {
            const float4* wv = sb + i * F4 + 1;
#pragma unroll
            for (int r4 = 0; r4 < NR / 4; ++r4) {
                const float4 w4 = wv[r4];
                const float2 wa = make_float2(w4.x, w4.y), wb = make_float2(w4.z, w4.w);
#pragma unroll
                for (int j = 0; j < T; ++j)
                    if ((JM >> j) & 1u) {
                        acc[j][2 * r4] = ffma2(kv[j], wa, acc[j][2 * r4]);
                        acc[j][2 * r4 + 1] = ffma2(kv[j], wb, acc[j][2 * r4 + 1]);
                    }
            }
        };
        const int nfull = n & ~(KB - 1);
#pragma unroll 1
        for (int i0 = 0; i0 < nfull; i0 += KB) {
            float kb[KB][T];
#pragma unroll
            for (int b = 0; b < KB; ++b) {
                const float4 sx = sb[(i0 + b) * F4];
#pragma unroll
                for (int j = 0; j < T; ++j)
                    if ((JM >> j) & 1u) kb[b][j] = act[j] ? kvalue(sx, j) : 0.0f;
            }
#pragma unroll
            for (int b = 0; b < KB; ++b) fmas(i0 + b, kb[b]);
        }
#pragma unroll 1
        for (int i = nfull; i < n; ++i) {
            const float4 sx = sb[i * F4];
            float kv[T];
#pragma unroll
            for (int j = 0; j < T; ++j)
                if ((JM >> j) & 1u) kv[j] = act[j] ? kvalue(sx, j) : 0.0f;
            fmas(i, kv);
        }
    } else if constexpr (Sh::PAIRS) {
        float2 ea[T][Sh::NA];
#pragma unroll
        for (int j = 0; j < T; ++j)
#pragma unroll
            for (int r = 0; r < Sh::NA; ++r) ea[j][r] = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int i = 0; i < n; ++i) {
            const float4 sx = sb[i * F4];
            float kv[T];
#pragma unroll
            for (int j = 0; j < T; ++j)
                if ((JM >> j) & 1u) kv[j] = kvalue(sx, j);
            const float4* wv = sb + i * F4 + 1;
#pragma unroll
            for (int r4 = 0; r4 < NR / 4; ++r4) {
                const float4 w4 = wv[r4];
                const float2 wa = make_float2(w4.x, w4.y), wb = make_float2(w4.z, w4.w);
#pragma unroll
                for (int j = 0; j < T; ++j)
                    if ((JM >> j) & 1u) {
                        ea[j][2 * r4] = ffma2(kv[j], wa, ea[j][2 * r4]);
                        ea[j][2 * r4 + 1] = ffma2(kv[j], wb, ea[j][2 * r4 + 1]);
                    }
            }
        }
#pragma unroll
        for (int j = 0; j < T; ++j)
            if (((JM >> j) & 1u) && act[j])
#pragma unroll
                for (int r = 0; r < Sh::NA; ++r) {
                    acc[j][r].x += ea[j][r].x;
                    acc[j][r].y += ea[j][r].y;
                }
    } else {
        float ea[T][NR];
#pragma unroll
        for (int j = 0; j < T; ++j)
#pragma unroll
            for (int r = 0; r < NR; ++r) ea[j][r] = 0.f;
#pragma unroll 4
        for (int i = 0; i < n; ++i) {
            const float4 sx = sb[i * F4];
            float kv[T];
#pragma unroll
            for (int j = 0; j < T; ++j)
                if ((JM >> j) & 1u) kv[j] = kvalue(sx, j);
            if (D == 3 && NR == 1) {
#pragma unroll
                for (int j = 0; j < T; ++j)
                    if ((JM >> j) & 1u) ea[j][0] = fmaf(kv[j], sx.w, ea[j][0]);
            } else {
                const float* wv = reinterpret_cast<const float*>(sb + i * F4) + R::WOFF;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const float wr = wv[r];
#pragma unroll
                    for (int j = 0; j < T; ++j)
                        if ((JM >> j) & 1u) ea[j][r] = fmaf(kv[j], wr, ea[j][r]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < T; ++j)
            if (((JM >> j) & 1u) && act[j])
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[j][r] += ea[j][r];
    }
}

// Near field of one target block: for each near entry (leaf, mask), every point of the leaf is
// streamed through shared memory by the bulk-copy engine (ST-stage mbarrier ring, issued by
// thread 0) and each thread accumulates K(|x_t - x_s|) w_s for its T targets.  With
// a.near_split = S > 1 (one right-hand side, small problems) S CTAs share a block: CTA part s
// takes entries s, s + S, ... and writes its partial sums to row s of ynear.
template <int D, int KIND, int NR, int T>
__global__ void __launch_bounds__(NearShape<D, NR, T>::THREADS, NearShape<D, NR, T>::MINB) near_kernel(MvmArgs a, KernelParams kp_all) {
    using R = Rec<D, NR>;
    using Sh = NearShape<D, NR, T>;
    constexpr int F4 = R::F4, CH = Sh::CH, ST = Sh::ST, NTH = Sh::THREADS, NA = Sh::NA;
    static_assert(!Sh::PAIRS || (R::WOFF == 4 && NR % 4 == 0), "multi-RHS passes read whole float4s of weights");
    using Acc = typename Sh::Acc;
    __shared__ __align__(128) float4 buf[ST][CH * F4];
    __shared__ __align__(8) uint64_t full[ST];
    const int tl = threadIdx.x;
    const int S = NR == 1 ? a.near_split : 1, part = (int)(blockIdx.x % S);
    const int64_t gi = blockIdx.x / S;
    const int64_t blk = a.blk_list ? (int64_t)a.blk_list[gi] : gi;
    const KernelParams kp = block_params(a, blk, kp_all);
    const int2 rg = a.blk[blk];
    float tx[T][4];
    bool valid[T];
#pragma unroll
    for (int j = 0; j < T; ++j) {
        const int t = rg.x + tl + NTH * j;
        valid[j] = t < rg.y;
        const float4 x = valid[j] ? a.xs[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        tx[j][0] = x.x * kp.sig; tx[j][1] = x.y * kp.sig; tx[j][2] = x.z * kp.sig; tx[j][3] = x.w * kp.sig;
    }
    Acc acc[T][NA];
#pragma unroll
    for (int j = 0; j < T; ++j)
#pragma unroll
        for (int r = 0; r < NA; ++r) {
            if constexpr (Sh::PAIRS) acc[j][r] = make_float2(0.f, 0.f);
            else acc[j][r] = 0.f;
        }
    const int64_t e0 = a.near_off[blk] + part, e1 = a.near_off[blk + 1];
    bool ok_all = true;
    if (e0 < e1) {
        if (tl == 0) {
#pragma unroll
            for (int s = 0; s < ST; ++s) ptx::mbar_init(&full[s], 1);
            ptx::fence_mbar_init();
        }
        __syncthreads();
        // producer cursor, used by thread 0 only
        int64_t pe = e0;
        int pcb = a.nd_begin[a.near_ent[e0].x];
        int issued = 0;
        auto issue = [&](int stage) {
            while (pe < e1) {
                const int s1 = a.nd_end[a.near_ent[pe].x];
                if (pcb < s1) {
                    const int n = min(CH, s1 - pcb);
                    const uint32_t bytes = (uint32_t)n * F4 * 16u;
                    ptx::mbar_arrive_expect_tx(&full[stage], bytes);
                    ptx::bulk_g2s(&buf[stage][0], a.rec + (int64_t)pcb * F4, bytes, &full[stage]);
                    pcb += n;
                    ++issued;
                    return;
                }
                pe += S;
                if (pe < e1) pcb = a.nd_begin[a.near_ent[pe].x];
            }
        };
        if (tl == 0)
            for (int s = 0; s < ST; ++s) issue(s);
        int k = 0;
        for (int64_t e = e0; e < e1 && ok_all; e += S) {
            const int2 ent = a.near_ent[e];
            bool act[T];
            unsigned jm = 0;  // slots whose 32-target group has an active target (warp-uniform)
#pragma unroll
            for (int j = 0; j < T; ++j) {
                act[j] = valid[j] && entry_active(ent.y, a.masks, tl + NTH * j);
                if (__any_sync(0xffffffffu, act[j])) jm |= 1u << j;
            }
            const int s0 = a.nd_begin[ent.x], s1 = a.nd_end[ent.x];
            for (int cb = s0; cb < s1; cb += CH, ++k) {
                const int n = min(CH, s1 - cb);
                const int stage = k % ST;
                const bool ok = ptx::mbar_wait_bounded(&full[stage], (uint32_t)((k / ST) & 1), kWaitCycles);
                if (ok) {
                    const float4* sb = &buf[stage][0];
                    if constexpr (T == 2) {
                        if (jm == 3u) near_chunk<D, KIND, NR, T, 3u>(sb, n, tx, act, acc, kp);
                        else if (jm == 1u) near_chunk<D, KIND, NR, T, 1u>(sb, n, tx, act, acc, kp);
                        else if (jm == 2u) near_chunk<D, KIND, NR, T, 2u>(sb, n, tx, act, acc, kp);
                    } else {
                        if (jm != 0u) near_chunk<D, KIND, NR, T, (1u << T) - 1u>(sb, n, tx, act, acc, kp);
                    }
                }
                ok_all = __syncthreads_and(ok) != 0;  // every thread is done with this stage
                if (!ok_all) break;
                if (tl == 0) {
                    ptx::fence_proxy_async_smem();
                    issue(stage);
                }
            }
        }
        if (!ok_all) {
            // A wait ran out: record it, let the copies still in flight land (bounded), stop.
            if (tl == 0) {
                atomicExch(a.err, 1);
                for (int q = k; q < issued; ++q)  // chunk k (the one that timed out) onwards
                    ptx::mbar_wait_bounded(&full[q % ST], (uint32_t)((q / ST) & 1), kWaitCycles);
            }
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < T; ++j) {
        const int t = rg.x + tl + NTH * j;
        if (valid[j]) {
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                float v;
                if constexpr (Sh::PAIRS) v = (r & 1) ? acc[j][r / 2].y : acc[j][r / 2].x;
                else v = acc[j][r];
                a.ynear[(int64_t)(r + part) * a.N + t] = v * kp.scale;  // part > 0 only when NR == 1
            }
        }
    }
}

// Multi-RHS near field (passes of 8, 16 or 32 right-hand sides).  One warp per CTA handles 32 T
// targets of a target block -- T 32-target groups, i.e. T words of every entry's mask -- with
// its own ST-stage bulk-copy ring.  An entry whose mask leaves all its groups empty is
// skipped outright (no copy, no wait), and no warp waits for another: the per-target near sets
// of a block differ, so a block-wide pipeline would make every warp wait through entries that
// only its neighbours need.
template <int D, int NR>
struct NearWideShape {
    static constexpr int T = NR >= 32 ? 1 : 2;     // targets per lane (32-target groups per CTA)
    static constexpr int F4 = Rec<D, NR>::F4;
    static constexpr int SPLIT = kTB / (32 * T);   // CTAs per 128-target block
    static constexpr int CH = F4 >= 9 ? 32 : 64;   // sources per stage
    static constexpr int ST = 3;
};

template <int D, int KIND, int NR>
__global__ void __launch_bounds__(32, 20) near_wide_kernel(MvmArgs a, KernelParams kp_all) {
    using R = Rec<D, NR>;
    using W = NearWideShape<D, NR>;
    using Sh = NearShape<D, NR, W::T>;
    constexpr int T = W::T, F4 = R::F4, CH = W::CH, ST = W::ST, NA = Sh::NA;
    static_assert(Sh::PAIRS, "multi-RHS passes only");
    __shared__ __align__(128) float4 buf[ST][CH * F4];
    __shared__ __align__(8) uint64_t full[ST];
    const int lane = threadIdx.x;
    const int64_t gi = blockIdx.x / W::SPLIT;
    const int w0 = (blockIdx.x % W::SPLIT) * T;  // first mask word (32-target group) of this CTA
    const int64_t blk = a.blk_list ? (int64_t)a.blk_list[gi] : gi;
    const KernelParams kp = block_params(a, blk, kp_all);
    const int2 rg = a.blk[blk];
    float tx[T][4];
    bool valid[T];
#pragma unroll
    for (int j = 0; j < T; ++j) {
        const int t = rg.x + 32 * (w0 + j) + lane;
        valid[j] = t < rg.y;
        const float4 x = valid[j] ? a.xs[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        tx[j][0] = x.x * kp.sig; tx[j][1] = x.y * kp.sig; tx[j][2] = x.z * kp.sig; tx[j][3] = x.w * kp.sig;
    }
    // bit j: group w0 + j has an active target for the entry with this mask (uniform over the warp)
    auto groups = [&](int mask) -> unsigned {
        unsigned m = 0;
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const bool any = mask < 0 ? (rg.x + 32 * (w0 + j) < rg.y)
                                      : (__ldg(&a.masks[(int64_t)mask * kMaskWords + w0 + j]) != 0u);
            if (any) m |= 1u << j;
        }
        return m;
    };
    typename Sh::Acc acc[T][NA];
#pragma unroll
    for (int j = 0; j < T; ++j)
#pragma unroll
        for (int r = 0; r < NA; ++r) acc[j][r] = make_float2(0.f, 0.f);
    const int64_t e0 = a.near_off[blk], e1 = a.near_off[blk + 1];
    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < ST; ++s) ptx::mbar_init(&full[s], 1);
        ptx::fence_mbar_init();
    }
    __syncwarp();
    // producer cursor (lane 0): entry pe, next source pcb; entries without an active group are passed over
    int64_t pe = e0;
    int pcb = 0;
    int issued = 0;
    auto settle = [&]() {
        while (pe < e1 && groups(a.near_ent[pe].y) == 0u) ++pe;
        if (pe < e1) pcb = a.nd_begin[a.near_ent[pe].x];
    };
    auto issue = [&](int stage) {
        while (pe < e1) {
            const int s1 = a.nd_end[a.near_ent[pe].x];
            if (pcb < s1) {
                const int n = min(CH, s1 - pcb);
                const uint32_t bytes = (uint32_t)n * F4 * 16u;
                ptx::mbar_arrive_expect_tx(&full[stage], bytes);
                ptx::bulk_g2s(&buf[stage][0], a.rec + (int64_t)pcb * F4, bytes, &full[stage]);
                pcb += n;
                ++issued;
                return;
            }
            ++pe;
            settle();
        }
    };
    if (lane == 0) {
        settle();
        for (int s = 0; s < ST; ++s) issue(s);
    }
    int k = 0;
    bool ok_all = true;
    for (int64_t e = e0; e < e1 && ok_all; ++e) {
        const int2 ent = a.near_ent[e];
        const unsigned jm = groups(ent.y);
        if (jm == 0u) continue;
        bool act[T];
#pragma unroll
        for (int j = 0; j < T; ++j) act[j] = valid[j] && entry_active(ent.y, a.masks, 32 * (w0 + j) + lane);
        const int s0 = a.nd_begin[ent.x], s1 = a.nd_end[ent.x];
        for (int cb = s0; cb < s1; cb += CH, ++k) {
            const int n = min(CH, s1 - cb);
            const int stage = k % ST;
            const bool ok = ptx::mbar_wait_bounded(&full[stage], (uint32_t)((k / ST) & 1), kWaitCycles);
            ok_all = __all_sync(0xffffffffu, ok);
            if (!ok_all) break;
            const float4* sb = &buf[stage][0];
            if constexpr (T == 1) {
                near_chunk<D, KIND, NR, T, 1u>(sb, n, tx, act, acc, kp);
            } else {
                if (jm == 3u) near_chunk<D, KIND, NR, T, 3u>(sb, n, tx, act, acc, kp);
                else if (jm == 1u) near_chunk<D, KIND, NR, T, 1u>(sb, n, tx, act, acc, kp);
                else near_chunk<D, KIND, NR, T, 2u>(sb, n, tx, act, acc, kp);
            }
            __syncwarp();  // every lane is done with this stage
            if (lane == 0) {
                ptx::fence_proxy_async_smem();
                issue(stage);
            }
        }
    }
    if (!ok_all) {
        // A wait ran out: record it, let the copies still in flight land (bounded), stop.
        if (lane == 0) {
            atomicExch(a.err, 1);
            for (int q = k; q < issued; ++q)
                ptx::mbar_wait_bounded(&full[q % ST], (uint32_t)((q / ST) & 1), kWaitCycles);
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < T; ++j) {
        const int t = rg.x + 32 * (w0 + j) + lane;
        if (valid[j])
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if (r < a.nr) a.ynear[(int64_t)r * a.N + t] = ((r & 1) ? acc[j][r / 2].y : acc[j][r / 2].x) * kp.scale;
    }
}

// Near field of 16- and 32-wide passes as a register-tiled product.  One warp per CTA handles one
// 32-target group (one word of every entry's mask) with its own ST-stage bulk-copy ring, so a
// warp passes over the entries its group does not need without waiting for anyone.  Per batch
// of KB staged sources:
//   A: lane = target: KB kernel values K[b][lane] (zero outside the entry's mask) -> shared tile;
//   B: lane = (i, j): targets 4i..4i+3 x right-hand sides (NR/4) j..: acc += K[b][4i..] w[b][..]
//      (packed FMAs, 4 x NR/4 independent accumulators per lane).
template <int D, int NR>
struct NearTileShape {
    static constexpr int F4 = Rec<D, NR>::F4;
    static constexpr int SPLIT = kTB / 32;          // CTAs per 128-target block
    static constexpr int CH = F4 >= 9 ? 16 : 32;    // sources per stage (small: ~8 KB of shared
    static constexpr int ST = 3;                    // memory per CTA keeps ~25 warps per SM)
    static constexpr int KB = 8;                    // sources per kernel-value batch
    static constexpr int RL = NR / 4;               // right-hand sides per lane
};

template <int D, int KIND, int NR>
__global__ void __launch_bounds__(32) near_tile_kernel(MvmArgs a, KernelParams kp_all) {
    using R = Rec<D, NR>;
    using S = NearTileShape<D, NR>;
    constexpr int F4 = R::F4, CH = S::CH, ST = S::ST, KB = S::KB, RL = S::RL;
    static_assert(R::WOFF == 4 && NR % 8 == 0, "whole float4s of weights, pairs per lane");
    __shared__ __align__(128) float4 buf[ST][CH * F4];
    __shared__ __align__(16) float Ks[KB][32];
    __shared__ __align__(8) uint64_t full[ST];
    const int lane = threadIdx.x;
    const int ti = lane >> 2, rj = lane & 3;        // phase-B tile coordinates
    const int64_t gi = blockIdx.x / S::SPLIT;
    const int grp = blockIdx.x % S::SPLIT;          // the 32-target group (mask word) of this CTA
    const int64_t blk = a.blk_list ? (int64_t)a.blk_list[gi] : gi;
    const KernelParams kp = block_params(a, blk, kp_all);
    const int2 rg = a.blk[blk];
    const int t0 = rg.x + 32 * grp;                 // first target of the group
    const bool valid = t0 + lane < rg.y;
    float tx[4];
    {
        const float4 x = valid ? a.xs[t0 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        tx[0] = x.x * kp.sig; tx[1] = x.y * kp.sig; tx[2] = x.z * kp.sig; tx[3] = x.w * kp.sig;
    }
    auto group_on = [&](int mask) -> bool {
        return mask < 0 ? (t0 < rg.y) : (__ldg(&a.masks[(int64_t)mask * kMaskWords + grp]) != 0u);
    };
    float2 acc[4][RL / 2];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < RL / 2; ++r) acc[q][r] = make_float2(0.f, 0.f);
    const int64_t e0 = a.near_off[blk], e1 = a.near_off[blk + 1];
    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < ST; ++s) ptx::mbar_init(&full[s], 1);
        ptx::fence_mbar_init();
    }
    __syncwarp();
    int64_t pe = e0;
    int pcb = 0;
    int issued = 0;
    auto settle = [&]() {
        while (pe < e1 && !group_on(a.near_ent[pe].y)) ++pe;
        if (pe < e1) pcb = a.nd_begin[a.near_ent[pe].x];
    };
    auto issue = [&](int stage) {
        while (pe < e1) {
            const int s1 = a.nd_end[a.near_ent[pe].x];
            if (pcb < s1) {
                const int n = min(CH, s1 - pcb);
                const uint32_t bytes = (uint32_t)n * F4 * 16u;
                ptx::mbar_arrive_expect_tx(&full[stage], bytes);
                ptx::bulk_g2s(&buf[stage][0], a.rec + (int64_t)pcb * F4, bytes, &full[stage]);
                pcb += n;
                ++issued;
                return;
            }
            ++pe;
            settle();
        }
    };
    if (lane == 0) {
        settle();
        for (int s = 0; s < ST; ++s) issue(s);
    }
    int k = 0;
    bool ok_all = true;
    for (int64_t e = e0; e < e1 && ok_all; ++e) {
        const int2 ent = a.near_ent[e];
        if (!group_on(ent.y)) continue;
        const bool act = valid && entry_active(ent.y, a.masks, 32 * grp + lane);
        const int s0 = a.nd_begin[ent.x], s1 = a.nd_end[ent.x];
        for (int cb = s0; cb < s1; cb += CH, ++k) {
            const int n = min(CH, s1 - cb);
            const int stage = k % ST;
            const bool ok = ptx::mbar_wait_bounded(&full[stage], (uint32_t)((k / ST) & 1), kWaitCycles);
            ok_all = __all_sync(0xffffffffu, ok);
            if (!ok_all) break;
            const float4* sb = &buf[stage][0];
            for (int i0 = 0; i0 < n; i0 += KB) {
                const int nb = min(KB, n - i0);
                // A: kernel values of this lane's target against the batch
#pragma unroll
                for (int b = 0; b < KB; ++b) {
                    float kv = 0.0f;
                    if (b < nb && act) {
                        const float4 sx = sb[(i0 + b) * F4];
                        const float dx = tx[0] - sx.x, dy = tx[1] - sx.y, dz = tx[2] - sx.z;
                        float q = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        if (D == 4) { const float dw = tx[3] - sx.w; q = fmaf(dw, dw, q); }
                        kv = kval<KIND>(q, kp);
                    }
                    Ks[b][lane] = kv;
                }
                __syncwarp();
                // B: 4 targets x RL right-hand sides per lane
#pragma unroll
                for (int b = 0; b < KB; ++b) {
                    if (b < nb) {
                        const float4 kk = *reinterpret_cast<const float4*>(&Ks[b][4 * ti]);
                        const float4* wv = sb + (i0 + b) * F4 + 1 + rj * (RL / 4);
#pragma unroll
                        for (int r4 = 0; r4 < RL / 4; ++r4) {
                            const float4 w4 = wv[r4];
                            const float2 wa = make_float2(w4.x, w4.y), wb = make_float2(w4.z, w4.w);
                            acc[0][2 * r4] = ffma2(kk.x, wa, acc[0][2 * r4]);
                            acc[0][2 * r4 + 1] = ffma2(kk.x, wb, acc[0][2 * r4 + 1]);
                            acc[1][2 * r4] = ffma2(kk.y, wa, acc[1][2 * r4]);
                            acc[1][2 * r4 + 1] = ffma2(kk.y, wb, acc[1][2 * r4 + 1]);
                            acc[2][2 * r4] = ffma2(kk.z, wa, acc[2][2 * r4]);
                            acc[2][2 * r4 + 1] = ffma2(kk.z, wb, acc[2][2 * r4 + 1]);
                            acc[3][2 * r4] = ffma2(kk.w, wa, acc[3][2 * r4]);
                            acc[3][2 * r4 + 1] = ffma2(kk.w, wb, acc[3][2 * r4 + 1]);
                        }
                    }
                }
                __syncwarp();  // Ks is rewritten by the next batch
            }
            if (lane == 0) {
                ptx::fence_proxy_async_smem();
                issue(stage);
            }
        }
    }
    if (!ok_all) {
        if (lane == 0) {
            atomicExch(a.err, 1);
            for (int q = k; q < issued; ++q)
                ptx::mbar_wait_bounded(&full[q % ST], (uint32_t)((q / ST) & 1), kWaitCycles);
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int t = t0 + 4 * ti + q;
        if (t < rg.y)
#pragma unroll
            for (int r = 0; r < RL; ++r) {
                const float v = (r & 1) ? acc[q][r / 2].y : acc[q][r / 2].x;
                if (rj * RL + r < a.nr) a.ynear[(int64_t)(rj * RL + r) * a.N + t] = v * kp.scale;
            }
    }
}

// ------------------------------------------------------------------ far
template <int D, int P, int NR>
struct FarShape {
    static constexpr int NT = Layout<D, P>::nterms;
    static constexpr int FB0 = 6144 / (NT * NR);
    static constexpr int FB = FB0 < 1 ? 1 : (FB0 > 8 ? 8 : FB0);   // entries staged per pass
    static constexpr size_t smem_bytes() { return sizeof(float) * (size_t)FB * NT * NR; }
};

template <int D, int P, int NR>
__global__ void __launch_bounds__(kTB) far_kernel(MvmArgs a, KernelParams kp_all, const __grid_constant__ FarTables T) {
    using Lay = Layout<D, P>;
    using Sh = FarShape<D, P, NR>;
    constexpr int NT = Sh::NT, FB = Sh::FB;
    extern __shared__ float sM[];
    __shared__ float4 s_c[FB];
    __shared__ float s_s[FB];
    __shared__ int s_m[FB];
    // a.far_split = S > 1 (one right-hand side, small problems): S CTAs share a target block, CTA
    // part s taking entries s, s + S, ... and writing its partial sums to row s of yfar
    const int S = NR == 1 ? a.far_split : 1, part = (int)(blockIdx.x % S);
    const int64_t gi = blockIdx.x / S;
    const int64_t blk = a.blk_list ? (int64_t)a.blk_list[gi] : gi;
    const KernelParams kp = block_params(a, blk, kp_all);
    const int2 rg = a.blk[blk];
    const int tl = threadIdx.x;
    const int t = rg.x + tl;
    const bool valid = t < rg.y;
    const float4 xt = valid ? a.xs[t] : make_float4(0.f, 0.f, 0.f, 0.f);
    float acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.f;
    const int64_t e0 = a.far_off[blk] + part, nall = a.far_off[blk + 1] - a.far_off[blk];
    const int64_t nmine = nall > part ? (nall - part + S - 1) / S : 0;  // entries e0 + S k, k < nmine
    for (int64_t kb = 0; kb < nmine; kb += FB) {
        const int nb = (int)min((int64_t)FB, nmine - kb);
        const int64_t eb = e0 + S * kb;
        __syncthreads();
        for (int i = tl; i < nb * NT * NR; i += kTB) {
            const int e = i / (NT * NR), q = i - e * NT * NR;
            const int node = a.far_ent[eb + (int64_t)S * e].x;
            sM[i] = a.mult[(int64_t)node * NT * NR + q];
        }
        if (tl < nb) {
            const int2 ent = a.far_ent[eb + (int64_t)S * tl];
            s_c[tl] = a.nd_cf[ent.x];
            s_s[tl] = a.nd_scale[ent.x];
            s_m[tl] = ent.y;
        }
        __syncthreads();
        for (int e = 0; e < nb; ++e) {
            if (!(valid && entry_active(s_m[e], a.masks, tl))) continue;
            const float4 c = s_c[e];
            const float dx = xt.x - c.x, dy = xt.y - c.y, dz = xt.z - c.z, dw = dim_of(D) == 4 ? xt.w - c.w : 0.f;
            const float r2 = dx * dx + dy * dy + dz * dz + dw * dw;
            const float rinv = rsqrtf(r2);
            const float r = r2 * rinv;
            const float u = s_s[e] * rinv;
            float J[P + 1];
            kernel_jets<P>(kp, r, rinv, J);
            float up[P + 1];
            up[0] = 1.f;
#pragma unroll
            for (int j = 1; j <= P; ++j) up[j] = up[j - 1] * u;
            float G[Lay::npairs];
#pragma unroll
            for (int k = 0; k <= P; ++k)
#pragma unroll
                for (int jj = 0; jj < Lay::nj(k); ++jj) {
                    const int j = k + 2 * jj, q = Lay::pair(k) + jj, tq = Lay::tpair(k, jj);
                    float R = 0.f;
#pragma unroll
                    for (int m = 0; m <= j; ++m) R = fmaf(T.That[tq][m], J[m], R);
                    G[q] = up[j] * R;
                }
            const float ux = dx * rinv, uy = dy * rinv, uz = dz * rinv, uw = dw * rinv;
            const float u2_3 = ux * ux + uy * uy + uz * uz;
            const float* Me = sM + e * NT * NR;
            solid_harmonics<D, P>(ux, uy, uz, uw, u2_3, u2_3 + uw * uw, T, [&](int k, int h, float Y) {
                const float* Mk = Me + (Lay::off(k) + h * Lay::nj(k)) * NR;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    float s = 0.f;
#pragma unroll
                    for (int jj = 0; jj < Lay::nj(k); ++jj) s = fmaf(G[Lay::pair(k) + jj], Mk[jj * NR + r], s);
                    acc[r] = fmaf(Y, s, acc[r]);
                }
            });
        }
    }
    if (valid) {
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (r < a.nr) a.yfar[(int64_t)(r + part) * a.N + t] = acc[r];  // part > 0 only when NR == 1
    }
}

// Multi-RHS far field (NR = 8 per pass): each thread writes its basis row
// U[t][q] = Yt_kh(x_t - c) (s/r)^j R_kj(r) for the current node into shared memory,
// then contracts it with the node's multipoles M[q][0..7] in a plain loop.
template <int D, int P>
struct FarMrShape {
    static constexpr int NT = Layout<D, P>::nterms;
    static constexpr int ROW = NT | 1;
    static constexpr size_t smem_bytes() { return sizeof(float) * ((size_t)kTB * ROW + (size_t)NT * 8); }
    static constexpr bool supported = smem_bytes() <= 200 * 1024;
};

template <int D, int P>
__global__ void __launch_bounds__(kTB) far_mr_kernel(MvmArgs a, KernelParams kp_all, const __grid_constant__ FarTables T) {
    using Lay = Layout<D, P>;
    constexpr int NT = Lay::nterms, ROW = FarMrShape<D, P>::ROW;
    extern __shared__ float sm[];
    float* U = sm;
    float4* Ms = reinterpret_cast<float4*>(sm + kTB * ROW);  // kTB * ROW is a multiple of 128 floats
    __shared__ float4 s_c;
    __shared__ float s_s;
    __shared__ int s_m;
    const int64_t blk = cta_block(a);
    const KernelParams kp = block_params(a, blk, kp_all);
    const int2 rg = a.blk[blk];
    const int tl = threadIdx.x;
    const int t = rg.x + tl;
    const bool valid = t < rg.y;
    const float4 xt = valid ? a.xs[t] : make_float4(0.f, 0.f, 0.f, 0.f);
    float acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = 0.f;
    float* Urow = U + tl * ROW;
    const int64_t e0 = a.far_off[blk], e1 = a.far_off[blk + 1];
    for (int64_t e = e0; e < e1; ++e) {
        __syncthreads();
        const int2 ent = a.far_ent[e];
        const float4* src = reinterpret_cast<const float4*>(a.mult + (int64_t)ent.x * NT * 8);
        for (int i = tl; i < NT * 2; i += kTB) Ms[i] = src[i];
        if (tl == 0) {
            s_c = a.nd_cf[ent.x];
            s_s = a.nd_scale[ent.x];
            s_m = ent.y;
        }
        __syncthreads();
        if (!(valid && entry_active(s_m, a.masks, tl))) continue;
        const float4 c = s_c;
        const float dx = xt.x - c.x, dy = xt.y - c.y, dz = xt.z - c.z, dw = dim_of(D) == 4 ? xt.w - c.w : 0.f;
        const float r2 = dx * dx + dy * dy + dz * dz + dw * dw;
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        const float u = s_s * rinv;
        float J[P + 1];
        kernel_jets<P>(kp, r, rinv, J);
        float up[P + 1];
        up[0] = 1.f;
#pragma unroll
        for (int j = 1; j <= P; ++j) up[j] = up[j - 1] * u;
        float G[Lay::npairs];
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int jj = 0; jj < Lay::nj(k); ++jj) {
                const int j = k + 2 * jj, q = Lay::pair(k) + jj, tq = Lay::tpair(k, jj);
                float R = 0.f;
#pragma unroll
                for (int m = 0; m <= j; ++m) R = fmaf(T.That[tq][m], J[m], R);
                G[q] = up[j] * R;
            }
        const float ux = dx * rinv, uy = dy * rinv, uz = dz * rinv, uw = dw * rinv;
        const float u2_3 = ux * ux + uy * uy + uz * uz;
        solid_harmonics<D, P>(ux, uy, uz, uw, u2_3, u2_3 + uw * uw, T, [&](int k, int h, float Y) {
            const int o = Lay::off(k) + h * Lay::nj(k);
#pragma unroll
            for (int jj = 0; jj < Lay::nj(k); ++jj) Urow[o + jj] = Y * G[Lay::pair(k) + jj];
        });
#pragma unroll 2
        for (int q = 0; q < NT; ++q) {
            const float uq = Urow[q];
            const float4 m0 = Ms[2 * q], m1 = Ms[2 * q + 1];
            acc[0] = fmaf(uq, m0.x, acc[0]);
            acc[1] = fmaf(uq, m0.y, acc[1]);
            acc[2] = fmaf(uq, m0.z, acc[2]);
            acc[3] = fmaf(uq, m0.w, acc[3]);
            acc[4] = fmaf(uq, m1.x, acc[4]);
            acc[5] = fmaf(uq, m1.y, acc[5]);
            acc[6] = fmaf(uq, m1.z, acc[6]);
            acc[7] = fmaf(uq, m1.w, acc[7]);
        }
    }
    if (valid) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
            if (r < a.nr) a.yfar[(int64_t)r * a.N + t] = acc[r];
    }
}

}  // namespace fkt
