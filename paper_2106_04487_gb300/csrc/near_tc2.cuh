// Near field of 32-wide passes on the tensor cores with FP16 hi/lo operands and double buffering.
//
// The same product as near_tc_kernel -- per 128-target block and chunk of up to 32 sources of a
// near leaf, z[t][r] += sum_s K(|x_t - x_s|) w[s][r] (Algorithm 1, the near-field sum of eq. nbody)
// -- with operands that let the MMAs of one chunk run while the next chunk is prepared:
//   * operands in FP16 (kind::f16, K = 16 per instruction, full rate): two MMA steps of three
//     products (hi*hi + hi*lo + lo*hi) per chunk instead of four TF32 steps; each factor v is split
//     into hi = v rounded to FP16 and lo = v - hi rounded to FP16 (about 22 significant bits; the
//     dropped lo*lo and the rounding of lo leave about 2^-21 of each product);
//   * range: kernel values K <= 1 (every kind except 1/r, which keeps the TF32 kernel) are computed
//     times 2^14, weights are multiplied by 2^-e_r per right-hand side r, with e_r the exponent that
//     puts the largest |w| of that right-hand side in [2^13, 2^14) (near_wscale_kernel); both are
//     exact powers of two, undone in the float32 sums at the end;
//   * tensor memory: two A buffers (hi, lo: 16 columns each for 32 sources) and two accumulators
//     (one per flush period of kFlush chunks): 128 columns, four CTAs per SM.  The consumers write
//     chunk c into A buffer c & 1 while the MMAs of chunk c - 1 run; they only wait for the MMAs of
//     chunk c - 2.  The accumulator of a period is added into float32 sums in shared memory one
//     chunk after the period ends (its last MMAs are then complete) and zeroed.
#pragma once

#include <cuda_fp16.h>

#include "near_tc.cuh"

namespace fkt {

struct NearTc2Shape {
    static constexpr int NR = 32;                     // right-hand sides (the MMA's N)
    static constexpr int CH = 32;                     // sources per chunk (2 MMA K-steps of 16)
    static constexpr int ST = 4;                      // record stages in flight
    static constexpr int F4 = (4 + NR + 3) / 4;       // float4s per source record
    static constexpr int CONSUMERS = 4;
    static constexpr int THREADS = 32 * (CONSUMERS + 1);
    static constexpr int TMEM_COLS = 128;             // D0 32 | D1 32 | A0 hi 16, lo 16 | A1 hi 16, lo 16
    static constexpr int COL_D = 0, COL_A = 64;       // D[i] at 32 i, A[b] hi at 64 + 32 b, lo at 80 + 32 b
    static constexpr int FLUSH = 4;                   // chunks (6 MMAs each) per accumulator period
    static constexpr float kKScale = 16384.0f;        // 2^14: kernel values into the FP16 range
};

// Largest |w| of each right-hand side of the pass, as float bits (non-negative floats order like
// their bits), from the source records: wmax[r] for r < nr.
template <int D>
__global__ void near_wscale_kernel(int64_t N, const float4* __restrict__ rec, int rec_f4, int woff, int nr,
                                   unsigned* __restrict__ wmax) {
    __shared__ unsigned s_max[32];
    if (threadIdx.x < 32) s_max[threadIdx.x] = 0u;
    __syncthreads();
    unsigned m[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) m[r] = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float* w = reinterpret_cast<const float*>(rec + i * rec_f4) + woff;
#pragma unroll
        for (int r = 0; r < 32; ++r)
            if (r < nr) m[r] = max(m[r], __float_as_uint(fabsf(w[r])));
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        unsigned v = m[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
        if ((threadIdx.x & 31) == 0 && r < nr) atomicMax(&s_max[r], v);
    }
    __syncthreads();
    if (threadIdx.x < nr) atomicMax(&wmax[threadIdx.x], s_max[threadIdx.x]);
}

// 2^-e with e chosen so that m * 2^-e lies in [2^13, 2^14) (m = the largest |w|, as float bits);
// 1 for m = 0 or non-finite m.
__device__ __forceinline__ float wscale_of(unsigned mbits) {
    const int ex = (int)((mbits >> 23) & 0xFFu);           // biased exponent of m
    if (mbits == 0u || ex == 0xFF) return 1.0f;
    const int e = (ex - 127) - 13;                          // m in [2^(ex-127), 2^(ex-126))
    const int be = 127 - e;                                 // biased exponent of 2^-e
    return be >= 1 && be <= 254 ? __uint_as_float((unsigned)be << 23) : 1.0f;
}

// Kernel values times 2^14 for two pairs (the formulas of kval2, with the factor folded into the
// ex2 argument or the reciprocal where possible).  KIND != FKT_LAPLACE.
template <int KIND>
__device__ __forceinline__ float2 kval2_k14(float2 q, const KernelParams& kp) {
    constexpr float kLn2 = 0.69314718055994531f;
    if (KIND == FKT_GAUSSIAN) {
        return make_float2(ptx::ex2(14.0f - q.x), ptx::ex2(14.0f - q.y));
    } else if (KIND == FKT_EXPONENTIAL) {
        return make_float2(ptx::ex2(14.0f - ptx::sqrt_approx(q.x)), ptx::ex2(14.0f - ptx::sqrt_approx(q.y)));
    } else if (KIND == FKT_MATERN32) {
        const float2 u = make_float2(ptx::sqrt_approx(q.x), ptx::sqrt_approx(q.y));
        const float2 e = make_float2(ptx::ex2(14.0f - u.x), ptx::ex2(14.0f - u.y));
        return __fmul2_rn(__ffma2_rn(u, make_float2(kLn2, kLn2), make_float2(1.f, 1.f)), e);
    } else if (KIND == FKT_MATERN52) {
        const float2 u = make_float2(ptx::sqrt_approx(q.x), ptx::sqrt_approx(q.y));
        const float2 e = make_float2(ptx::ex2(14.0f - u.x), ptx::ex2(14.0f - u.y));
        const float2 t = __fmul2_rn(u, make_float2(kLn2, kLn2));
        const float2 poly = __ffma2_rn(t, __ffma2_rn(t, make_float2(1.f / 3.f, 1.f / 3.f), make_float2(1.f, 1.f)),
                                       make_float2(1.f, 1.f));
        return __fmul2_rn(poly, e);
    } else if (KIND == FKT_CAUCHY) {  // 2^14 / (1 + q) = 1 / (2^-14 + 2^-14 q)
        const float2 b = __ffma2_rn(q, make_float2(1.f / 16384.f, 1.f / 16384.f), make_float2(1.f / 16384.f, 1.f / 16384.f));
        return make_float2(ptx::rcp_approx(b.x), ptx::rcp_approx(b.y));
    } else {  // rational quadratic
        const float2 b = __fadd2_rn(q, make_float2(1.f, 1.f));
        if (kp.alpha == 1.0f) {
            const float2 bs = __fmul2_rn(b, make_float2(1.f / 16384.f, 1.f / 16384.f));
            return make_float2(ptx::rcp_approx(bs.x), ptx::rcp_approx(bs.y));
        }
        return make_float2(ptx::ex2(14.0f - kp.alpha * ptx::lg2(b.x)), ptx::ex2(14.0f - kp.alpha * ptx::lg2(b.y)));
    }
}

__device__ __forceinline__ uint32_t h2_bits(__half2 v) {
    uint32_t u;
    memcpy(&u, &v, sizeof(u));
    return u;
}

// (a, b) -> FP16 hi pair and FP16 lo pair (lo = the FP16 rounding of v - hi), a in the low half.
__device__ __forceinline__ void split_f16x2(float2 v, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(v.x, v.y);
    hi = h2_bits(h);
    const float2 hf = __half22float2(h);
    const float2 r = __ffma2_rn(hf, make_float2(-1.f, -1.f), v);
    lo = h2_bits(__floats2half2_rn(r.x, r.y));
}

// One CTA per 128-target block; warps 0-3 = targets (thread = target = tensor-memory lane),
// warp 4 = producer (chunk metadata, bulk copies of the source records ST chunks ahead) and MMA
// issuer.  Per chunk c the targets wait for its records, evaluate their kernel values (FP16
// hi/lo), wait until the MMAs of chunk c - 2 are complete (named barrier), write A buffer c & 1
// and their share of B buffer c & 1 (weights times the right-hand side's 2^-e_r, FP16 hi/lo) and
// arrive; the issuer runs the chunk's 6 MMAs (rows outside the chunk's mask disabled) into the
// period's accumulator, then polls the completion of chunk c - 1 and releases the targets.  Both
// roles run the block's chunk count of rounds whatever happens; a bounded wait that runs out
// sets s_fail, which only skips work.
template <int D, int KIND>
__global__ void __launch_bounds__(NearTc2Shape::THREADS, 4) near_tc2_kernel(MvmArgs a, KernelParams kp_all,
                                                                            const unsigned* __restrict__ wmax) {
    using S = NearTc2Shape;
    constexpr int CH = S::CH, ST = S::ST, F4 = S::F4, NR = S::NR, NC = S::CONSUMERS, FLUSH = S::FLUSH;
    constexpr uint32_t IDESC = tc::instr_desc(0u, 128u, (uint32_t)NR);  // kind::f16, A and B FP16
    constexpr uint32_t kBarReady = 1, kBarMma = 2, kBarThreads = S::THREADS;
    constexpr int BPLANE = CH * NR * 2;                      // bytes of one FP16 plane of B (2 KB)
    __shared__ __align__(128) float4 stage[ST][CH * F4];
    __shared__ __align__(128) unsigned char bbuf[2][2 * BPLANE];  // [buffer][hi | lo], K-major core matrices
    __shared__ __align__(16) float s_src[NC][4][CH];
    __shared__ NearChunkInfo info[ST];
    __shared__ __align__(8) uint64_t full[ST], mma_done[2];
    __shared__ uint32_t tmem_base;
    __shared__ uint32_t s_valid[kMaskWords];
    __shared__ int s_fail, s_nch;
    __shared__ float s_acc[NR][NC * 32];
    const int tl = threadIdx.x, warp = tl >> 5, lane = tl & 31;
    const int64_t blk = cta_block(a);
    const KernelParams kp = block_params(a, blk, kp_all);
    const int2 rg = a.blk[blk];
    const int t = rg.x + tl;
    const bool valid = warp < NC && t < rg.y;
    const uint32_t vword = __ballot_sync(0xffffffffu, valid);
    const int64_t e0 = a.near_off[blk], e1 = a.near_off[blk + 1];
    if (tl == 0) {
#pragma unroll
        for (int s = 0; s < ST; ++s) ptx::mbar_init(&full[s], 1);
        ptx::mbar_init(&mma_done[0], 1);
        ptx::mbar_init(&mma_done[1], 1);
        ptx::fence_mbar_init();
        s_fail = 0;
        s_nch = 0;
    }
    if (warp < NC && lane == 0) s_valid[warp] = vword;
    if (warp == 0) {
        tc::alloc(&tmem_base, S::TMEM_COLS);
        tc::relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    {   // the block's chunk count (both roles loop exactly this many rounds)
        int cnt = 0;
        for (int64_t e = e0 + tl; e < e1; e += S::THREADS) {
            const int leaf = a.near_ent[e].x;
            cnt += (a.nd_end[leaf] - a.nd_begin[leaf] + CH - 1) / CH;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0 && cnt) atomicAdd(&s_nch, cnt);
    }
    __syncthreads();
    const int nch = s_nch;
    const uint32_t tmem = tmem_base;
    __shared__ float s_wsc[NR];  // 2^-e_r per right-hand side
    if (tl < NR) s_wsc[tl] = tl < a.nr ? wscale_of(wmax[tl]) : 1.0f;
    __syncthreads();

    if (warp == NC) {
        // ---------------------------------------------------------------- producer / issuer
        int64_t wbase = e0;
        int wbeg = 0, wend = 0;
        uint32_t wm[kMaskWords] = {0u, 0u, 0u, 0u};
        auto load_window = [&]() {
            const int64_t e = wbase + lane;
            wbeg = wend = 0;
            if (e < e1) {
                const int2 ent = a.near_ent[e];
                wbeg = a.nd_begin[ent.x];
                wend = a.nd_end[ent.x];
#pragma unroll
                for (int w = 0; w < kMaskWords; ++w)
                    wm[w] = (ent.y < 0 ? 0xFFFFFFFFu : __ldg(&a.masks[(int64_t)ent.y * kMaskWords + w])) & s_valid[w];
            }
        };
        int ei = 0, cb = 0, cend = 0, issued = 0;
        bool pdone = wbase >= e1;
        auto settle = [&]() {  // warp-uniform: advance to the next entry with sources left
            while (!pdone && cb >= cend) {
                if (++ei == 32) {
                    wbase += 32;
                    ei = 0;
                    if (wbase >= e1) { pdone = true; break; }
                    load_window();
                }
                if (wbase + ei >= e1) { pdone = true; break; }
                cb = __shfl_sync(0xffffffffu, wbeg, ei);
                cend = __shfl_sync(0xffffffffu, wend, ei);
            }
        };
        auto produce = [&]() {  // warp-collective
            if (pdone) return;
            const int slot = issued % ST;
            const int n = min(CH, cend - cb);
            uint32_t on[kMaskWords];
#pragma unroll
            for (int w = 0; w < kMaskWords; ++w) on[w] = __shfl_sync(0xffffffffu, wm[w], ei);
            if (lane == 0) {
                NearChunkInfo& in = info[slot];
                in.n = n;
#pragma unroll
                for (int w = 0; w < kMaskWords; ++w) in.on[w] = on[w];
                const uint32_t bytes = (uint32_t)n * F4 * 16u;
                ptx::fence_proxy_async_smem();
                ptx::mbar_arrive_expect_tx(&full[slot], bytes);
                ptx::bulk_g2s(&stage[slot][0], a.rec + (int64_t)cb * F4, bytes, &full[slot]);
            }
            ++issued;
            cb += CH;
            settle();
        };
        if (!pdone) {
            load_window();
            cb = __shfl_sync(0xffffffffu, wbeg, 0);
            cend = __shfl_sync(0xffffffffu, wend, 0);
            settle();
        }
        for (int s = 0; s < ST; ++s) produce();
        int ncommit = 0;   // chunks whose MMAs were committed (0..c), in order while nothing failed
        int nwaited = 0;   // chunks whose MMAs were seen complete
        auto wait_chunk = [&](int c) {  // lane 0: MMAs of chunk c complete (bounded)
            if (c < 0 || c >= ncommit || c < nwaited) return;
            if (ptx::mbar_wait_bounded(&mma_done[c & 1], (uint32_t)((c >> 1) & 1), kWaitCycles)) nwaited = c + 1;
            else s_fail = 1;
        };
        for (int c = 0; c < nch; ++c) {
            const int slot = c % ST, b = c & 1;
            ptx::named_sync(kBarReady, kBarThreads);   // A and B buffers b hold chunk c
            if (lane == 0) {
                if (!s_fail) {
                    tc::fence_after_sync();
                    const NearChunkInfo in = info[slot];
                    const uint32_t off[kMaskWords] = {~in.on[0], ~in.on[1], ~in.on[2], ~in.on[3]};
                    const uint32_t dcol = tmem + S::COL_D + 32 * ((c / FLUSH) & 1);
                    const uint32_t ahi = tmem + S::COL_A + 32 * b, alo = ahi + 16;
                    const int nks = (in.n + 15) / 16;
                    for (int ks = 0; ks < nks; ++ks) {
                        const uint64_t bh = tc::smem_desc(&bbuf[b][ks * 1024], 512, 128);
                        const uint64_t bl = tc::smem_desc(&bbuf[b][BPLANE + ks * 1024], 512, 128);
                        tc::mma_bf16_ts_masked(dcol, ahi + ks * 8, bh, IDESC, off);
                        tc::mma_bf16_ts_masked(dcol, ahi + ks * 8, bl, IDESC, off);
                        tc::mma_bf16_ts_masked(dcol, alo + ks * 8, bh, IDESC, off);
                    }
                    tc::commit(&mma_done[b]);
                    ncommit = c + 1;
                }
                wait_chunk(c - 1);                     // frees A / B buffers (c - 1) & 1 for chunk c + 1
                tc::fence_before_sync();
            }
            __syncwarp();
            ptx::named_arrive(kBarMma, kBarThreads);
            // stage `slot` has been read by every target warp: refill it ST chunks ahead
            if (__all_sync(0xffffffffu, !s_fail)) produce();   // warp-uniform: produce() shuffles
        }
        if (nch >= 1) {
            if (lane == 0) {
                wait_chunk(nch - 1);
                tc::fence_before_sync();
            }
            __syncwarp();
            ptx::named_arrive(kBarMma, kBarThreads);   // every MMA of the block is complete
        }
        if (lane == 0 && s_fail) {
            atomicExch(a.err, 1);
            // the last copy of each stage may still be in flight; then the MMAs not seen complete
            for (int j = issued > ST ? issued - ST : 0; j < issued; ++j)
                ptx::mbar_wait_bounded(&full[j % ST], (uint32_t)((j / ST) & 1), kWaitCycles);
            if (nwaited < ncommit)  // the last commit covers every earlier MMA
                ptx::mbar_wait_bounded(&mma_done[(ncommit - 1) & 1], (uint32_t)(((ncommit - 1) >> 1) & 1), kWaitCycles);
        }
    } else {
        // ---------------------------------------------------------------- targets
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        float2 tx2[4];
        {
            const float4 x = valid ? a.xs[t] : make_float4(0.f, 0.f, 0.f, 0.f);
            tx2[0] = make_float2(x.x * kp.sig, x.x * kp.sig);
            tx2[1] = make_float2(x.y * kp.sig, x.y * kp.sig);
            tx2[2] = make_float2(x.z * kp.sig, x.z * kp.sig);
            tx2[3] = make_float2(x.w * kp.sig, x.w * kp.sig);
        }
        const float wsc = s_wsc[lane];  // this lane's right-hand side in the B operand
        tc::st32_zero(tmem + lane_base + S::COL_D);
        tc::st32_zero(tmem + lane_base + S::COL_D + 32);
        tc::wait_st();
#pragma unroll
        for (int r = 0; r < NR; ++r) s_acc[r][tl] = 0.f;
        auto flush = [&](int i) {  // accumulator i -> the float32 sums, then zero it
#pragma unroll
            for (int h = 0; h < NR; h += 16) {
                float d[16];
                tc::ld16(tmem + lane_base + S::COL_D + 32 * i + h, d);
#pragma unroll
                for (int r = 0; r < 16; ++r) s_acc[h + r][tl] += d[r];
            }
            tc::st32_zero(tmem + lane_base + S::COL_D + 32 * i);
        };
        unsigned dirty = 0u;  // bit i: this warp's rows of accumulator i hold products not yet summed
        for (int c = 0; c < nch; ++c) {
            const int slot = c % ST, b = c & 1;
            const bool got = ptx::mbar_wait_bounded(&full[slot], (uint32_t)((c / ST) & 1), a.wait_cycles);
            if (!__all_sync(0xffffffffu, got)) s_fail = 1;
            const int n = info[slot].n;
            const uint32_t mword = s_fail ? 0u : info[slot].on[warp];
            const float4* sb = &stage[slot][0];
            // this row's kernel values against the chunk, before waiting for the MMAs of chunk c-2
            uint32_t khi[CH / 2], klo[CH / 2];
            if (mword != 0u) {
                {   // this warp's SoA copy of the chunk's negated coordinates (zeros past the chunk's
                    // end: those columns meet zero weights in B)
                    const float4 r = lane < n ? sb[lane * F4] : make_float4(0.f, 0.f, 0.f, 0.f);
                    s_src[warp][0][lane] = -r.x;
                    s_src[warp][1][lane] = -r.y;
                    s_src[warp][2][lane] = -r.z;
                    if (dim_of(D) == 4) s_src[warp][3][lane] = -r.w;
                }
                __syncwarp();
#pragma unroll
                for (int j4 = 0; j4 < CH; j4 += 4) {
                    if (j4 < 16 || n > 16) {  // the MMAs read only ceil(n/16) K-steps
                        const float4 X = *reinterpret_cast<const float4*>(&s_src[warp][0][j4]);
                        const float4 Y = *reinterpret_cast<const float4*>(&s_src[warp][1][j4]);
                        const float4 Z = *reinterpret_cast<const float4*>(&s_src[warp][2][j4]);
                        float2 q[2];
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            const float2 dx = __fadd2_rn(tx2[0], hh ? make_float2(X.z, X.w) : make_float2(X.x, X.y));
                            const float2 dy = __fadd2_rn(tx2[1], hh ? make_float2(Y.z, Y.w) : make_float2(Y.x, Y.y));
                            const float2 dz = __fadd2_rn(tx2[2], hh ? make_float2(Z.z, Z.w) : make_float2(Z.x, Z.y));
                            q[hh] = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                        }
                        if (dim_of(D) == 4) {
                            const float4 W = *reinterpret_cast<const float4*>(&s_src[warp][3][j4]);
                            const float2 dw0 = __fadd2_rn(tx2[3], make_float2(W.x, W.y));
                            const float2 dw1 = __fadd2_rn(tx2[3], make_float2(W.z, W.w));
                            q[0] = __ffma2_rn(dw0, dw0, q[0]);
                            q[1] = __ffma2_rn(dw1, dw1, q[1]);
                        }
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh)
                            split_f16x2(kval2_k14<KIND>(q[hh], kp), khi[j4 / 2 + hh], klo[j4 / 2 + hh]);
                    } else {
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) khi[j4 / 2 + hh] = klo[j4 / 2 + hh] = 0u;
                    }
                }
            }
            if (c >= 1) ptx::named_sync(kBarMma, kBarThreads);  // the MMAs of chunk c-2 are complete
            tc::fence_after_sync();
            const bool work = !s_fail;
            bool stored = false;
            if (work && c % FLUSH == 1 && c > FLUSH) {  // the period before the current one is complete
                const int i = ((c / FLUSH) - 1) & 1;
                if ((dirty >> i) & 1u) {
                    flush(i);
                    dirty &= ~(1u << i);
                    stored = true;
                }
            }
            if (work) {
                // B operand: warp w rearranges sources 8w..8w+7 of the chunk, lane = right-hand side;
                // element (n, k) at byte (k / 8) * 512 + n * 16 + (k % 8) * 2 of each plane
                const int kg = warp;
                uint32_t h[4], l[4];
#pragma unroll
                for (int i2 = 0; i2 < 4; ++i2) {
                    const int k = 8 * kg + 2 * i2;
                    const float v0 = k < n ? reinterpret_cast<const float*>(sb + k * F4)[4 + lane] * wsc : 0.f;
                    const float v1 = k + 1 < n ? reinterpret_cast<const float*>(sb + (k + 1) * F4)[4 + lane] * wsc : 0.f;
                    split_f16x2(make_float2(v0, v1), h[i2], l[i2]);
                }
                *reinterpret_cast<uint4*>(&bbuf[b][kg * 512 + lane * 16]) = make_uint4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<uint4*>(&bbuf[b][BPLANE + kg * 512 + lane * 16]) = make_uint4(l[0], l[1], l[2], l[3]);
            }
            if (work && mword != 0u) {  // A operand: the row into tensor memory, buffer b
                const uint32_t ahi = tmem + lane_base + S::COL_A + 32 * b;
                tc::st16(ahi, khi);
                tc::st16(ahi + 16, klo);
                dirty |= 1u << ((c / FLUSH) & 1);
                stored = true;
            }
            if (stored) tc::wait_st();
            ptx::fence_proxy_async_smem();  // B planes -> the tensor core
            tc::fence_before_sync();
            __syncwarp();
            ptx::named_arrive(kBarReady, kBarThreads);
        }
        if (nch >= 1) {  // the MMAs of chunk nch-2, then of the last chunk, are complete
            ptx::named_sync(kBarMma, kBarThreads);
            ptx::named_sync(kBarMma, kBarThreads);
        }
        tc::fence_after_sync();
        const bool ok = !s_fail;
        if (ok) {
            if (dirty & 1u) flush(0);
            if (dirty & 2u) flush(1);
        }
        __syncwarp();
        if (ok && valid) {
            const float f = kp.scale * (1.0f / S::kKScale);
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if (r < a.nr) acc_store(a, r, t, s_acc[r][tl] * f / s_wsc[r]);
        }
        if (!ok && tl == 0) atomicExch(a.err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::dealloc(tmem, S::TMEM_COLS);
}

template <int D>
void launch_near_tc2_dim(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp,
                         const unsigned* wmax) {
    constexpr int TH = NearTc2Shape::THREADS;
    switch (kind) {
    case FKT_GAUSSIAN: near_tc2_kernel<D, FKT_GAUSSIAN><<<grid, TH, 0, st>>>(a, kp, wmax); break;
    case FKT_EXPONENTIAL: near_tc2_kernel<D, FKT_EXPONENTIAL><<<grid, TH, 0, st>>>(a, kp, wmax); break;
    case FKT_MATERN32: near_tc2_kernel<D, FKT_MATERN32><<<grid, TH, 0, st>>>(a, kp, wmax); break;
    case FKT_MATERN52: near_tc2_kernel<D, FKT_MATERN52><<<grid, TH, 0, st>>>(a, kp, wmax); break;
    case FKT_CAUCHY: near_tc2_kernel<D, FKT_CAUCHY><<<grid, TH, 0, st>>>(a, kp, wmax); break;
    default: near_tc2_kernel<D, FKT_RATQUAD><<<grid, TH, 0, st>>>(a, kp, wmax); break;
    }
}

}  // namespace fkt
