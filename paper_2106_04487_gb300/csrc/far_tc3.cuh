// Far field on the tensor cores, two far entries per thread (d = 3, BF16 / BF16 hi+lo).
//
// The same product as far_tc2_kernel -- per 128-target block z[t][r] += sum_b U_b[t][q] M_b[q][r],
// U_b[t][q] = Yt_kh(x_t - c_b) (s_b/r)^j R_kj(r) (Theorem 3.1, eq. finaltrunc) -- with the CUDA-core
// work of the basis rows halved: a thread (one target, one tensor-memory lane) generates its rows
// for two consecutive entries of its block's list at once, in packed float32 pairs (x = first
// entry, y = second), so every add, multiply and FMA of the jets, the radial sums, the harmonics
// and the term products is one FFMA2/FMUL2/FADD2 for both entries.  A warp does this for an
// entry pair when any of its targets takes either entry; the masks of the two entries overlap
// strongly, so the pairs cost about half as many warp passes as single entries.  Each entry's
// row goes to its own A buffer in tensor memory; the MMA issuer runs the entries' MMAs with their
// own row masks (rows outside an entry's mask disabled) into one float32 accumulator, which the
// target threads add into float32 sums in shared memory every kFlushPairs pairs (the tensor
// core's accumulation is not round-to-nearest).
//
// Tensor memory per CTA: accumulator 32 columns + 2 A buffers x (hi [+ lo]) x NTP/2 columns of
// packed BF16 pairs = 224 columns at p = 6 (BF16 hi/lo), allocated as 256: two CTAs per SM.
#pragma once

#include "far_tc.cuh"

namespace fkt {

// Far-field tables with every coefficient duplicated into both halves of a float2, so that a
// packed FMA takes it as one 64-bit operand.
struct FarTables2 {
    float2 That[36][11];
    float2 hA[11][11];
    float2 hB[11][11];
    float2 hSeed[11];
};

inline void make_far_tables2(const FarTables& T, FarTables2* out) {
    for (int i = 0; i < 36; ++i)
        for (int m = 0; m < 11; ++m) out->That[i][m] = make_float2(T.That[i][m], T.That[i][m]);
    for (int l = 0; l < 11; ++l) {
        for (int m = 0; m < 11; ++m) {
            out->hA[l][m] = make_float2(T.hA[l][m], T.hA[l][m]);
            out->hB[l][m] = make_float2(T.hB[l][m], T.hB[l][m]);
        }
        out->hSeed[l] = make_float2(T.hSeed[l], T.hSeed[l]);
    }
}

namespace f2 {
__device__ __forceinline__ float2 dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 exp(float2 a) { return make_float2(__expf(a.x), __expf(a.y)); }
__device__ __forceinline__ float2 rcp(float2 a) { return make_float2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y)); }
}  // namespace f2

// Packed kernel_jets: J_m = K^(m)(r) r^m / m! for two distances at once (same recurrences).
// sc = the kernel scale of each half; a zero scale zeroes that half (every J_m carries it).
template <int P>
__device__ __forceinline__ void kernel_jets2(const KernelParams& kp, float2 r, float2 rinv, float2 sc, float2 J[P + 1]) {
    using namespace f2;
    switch (kp.kind) {
    case FKT_GAUSSIAN: {
        const float2 a = mul(mul(r, r), dup(kp.c1));
        const float2 E = mul(sc, exp(neg(a)));
        float2 em2 = dup(0.f), em1 = dup(1.f);
        J[0] = E;
#pragma unroll
        for (int m = 1; m <= P; ++m) {
            const float2 em = mul(mul(a, dup(-2.0f / m)), add(em1, em2));
            J[m] = mul(E, em);
            em2 = em1;
            em1 = em;
        }
        break;
    }
    case FKT_EXPONENTIAL: {
        const float2 b = mul(r, dup(kp.c1));
        float2 v = mul(sc, exp(neg(b)));
        J[0] = v;
#pragma unroll
        for (int m = 1; m <= P; ++m) {
            v = mul(v, mul(b, dup(-1.0f / m)));
            J[m] = v;
        }
        break;
    }
    case FKT_MATERN32: {
        const float2 b = mul(r, dup(kp.c1));
        const float2 b1 = add(b, dup(1.f));
        float2 E = mul(sc, exp(neg(b)));
        J[0] = mul(b1, E);
#pragma unroll
        for (int m = 1; m <= P; ++m) {
            const float2 En = mul(E, mul(b, dup(-1.0f / m)));
            J[m] = fma(b1, En, mul(b, E));
            E = En;
        }
        break;
    }
    case FKT_MATERN52: {
        const float2 b = mul(r, dup(kp.c1));
        const float2 bb = mul(b, b);
        const float2 p0 = fma(bb, dup(1.0f / 3.0f), add(b, dup(1.f)));
        const float2 p1 = fma(bb, dup(2.0f / 3.0f), b);
        const float2 p2 = mul(bb, dup(1.0f / 3.0f));
        float2 Em2 = dup(0.f), Em1 = dup(0.f), E = mul(sc, exp(neg(b)));
#pragma unroll
        for (int m = 0; m <= P; ++m) {
            if (m > 0) {
                const float2 En = mul(E, mul(b, dup(-1.0f / m)));
                Em2 = Em1;
                Em1 = E;
                E = En;
            }
            J[m] = fma(p0, E, fma(p1, Em1, mul(p2, Em2)));
        }
        break;
    }
    case FKT_CAUCHY: {
        const float2 c = mul(mul(r, r), dup(kp.c1));
        const float2 inv = rcp(add(c, dup(1.f)));
        float2 qm2 = dup(0.f), qm1 = mul(sc, inv);
        const float2 c2 = mul(c, dup(-2.f)), cn = neg(c);
        J[0] = qm1;
#pragma unroll
        for (int m = 1; m <= P; ++m) {
            const float2 q = mul(fma(c2, qm1, mul(cn, qm2)), inv);
            J[m] = q;
            qm2 = qm1;
            qm1 = q;
        }
        break;
    }
    case FKT_RATQUAD: {
        const float2 c = mul(mul(r, r), dup(kp.c1));
        const float2 d0 = add(c, dup(1.f));
        const float2 d1 = mul(c, dup(2.f));
        const float beta = -kp.alpha;
        const float2 inv = rcp(d0);
        float2 fm2 = dup(0.f);
        float2 fm1 = mul(sc, make_float2(exp2f(beta * __log2f(d0.x)), exp2f(beta * __log2f(d0.y))));
        J[0] = fm1;
#pragma unroll
        for (int m = 1; m <= P; ++m) {
            const float2 t = fma(mul(d1, dup(beta - (m - 1))), fm1, mul(mul(c, dup(2.0f * beta - (m - 2))), fm2));
            const float2 f = mul(mul(t, inv), dup(1.0f / m));
            J[m] = f;
            fm2 = fm1;
            fm1 = f;
        }
        break;
    }
    default: {  // Laplace
        float2 v = mul(sc, rinv);
#pragma unroll
        for (int m = 0; m <= P; ++m) {
            J[m] = v;
            v = neg(v);
        }
        break;
    }
    }
}

// Degree L of the harmonics (and the levels above it, by compile-time recursion, so every array
// index is a constant): the Legendre-type values cur[m] of degree L from the two previous degrees,
// then put(q, Y_Lh G_Lj) for the terms of degree L in increasing q.
template <int P, int L, class F>
__device__ __forceinline__ void harmonic_level(float2 uz, const float2 (&C)[P + 1], const float2 (&S)[P + 1],
                                               float2 (&pm1)[P + 1], float2 (&pm2)[P + 1],
                                               const float2 (&G)[Layout<3, P>::npairs], const FarTables2& T, F&& put) {
    using namespace f2;
    using Lay = Layout<3, P>;
    float2 cur[L + 1];
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        if (m == L) cur[m] = T.hSeed[m];
        else if (m == L - 1) cur[m] = mul(T.hA[L][m], mul(uz, pm1[m]));
        else cur[m] = fma(T.hA[L][m], mul(uz, pm1[m]), neg(mul(T.hB[L][m], pm2[m])));
    }
    constexpr int o = Lay::off(L), nj = Lay::nj(L), g = Lay::pair(L);
#pragma unroll
    for (int jj = 0; jj < nj; ++jj) put(o + jj, mul(cur[0], G[g + jj]));
#pragma unroll
    for (int m = 1; m <= L; ++m) {
        const float2 yc = mul(cur[m], C[m]), ys = mul(cur[m], S[m]);
#pragma unroll
        for (int jj = 0; jj < nj; ++jj) put(o + (2 * m - 1) * nj + jj, mul(yc, G[g + jj]));
#pragma unroll
        for (int jj = 0; jj < nj; ++jj) put(o + 2 * m * nj + jj, mul(ys, G[g + jj]));
    }
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        pm2[m] = pm1[m];
        pm1[m] = cur[m];
    }
    if constexpr (L < P) harmonic_level<P, L + 1>(uz, C, S, pm1, pm2, G, T, put);
}

// Basis rows of one target for two far nodes at once (x: node 0, y: node 1): calls
// put(q, U[q]) for q = 0..NT-1 in increasing order.  Same expansion as far_basis<3, P>; the
// direction is a unit vector, so the homogeneous recurrence's |u|^2 factor is 1.
template <int P, class F>
__device__ __forceinline__ void far_basis2(const float4& xt, float2 cx, float2 cy, float2 cz, float2 s, float2 sc,
                                           const KernelParams& kp, const FarTables2& T, F&& put) {
    using namespace f2;
    using Lay = Layout<3, P>;
    const float2 dx = sub(dup(xt.x), cx), dy = sub(dup(xt.y), cy), dz = sub(dup(xt.z), cz);
    const float2 r2 = fma(dx, dx, fma(dy, dy, mul(dz, dz)));
    const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 r = mul(r2, rinv);
    const float2 u = mul(s, rinv);
    float2 G[Lay::npairs];
    {
        float2 J[P + 1];
        kernel_jets2<P>(kp, r, rinv, sc, J);
        float2 up[P + 1];
        up[0] = dup(1.f);
#pragma unroll
        for (int j = 1; j <= P; ++j) up[j] = mul(up[j - 1], u);
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int jj = 0; jj < Lay::nj(k); ++jj) {
                const int j = k + 2 * jj, q = Lay::pair(k) + jj, tq = Lay::tpair(k, jj);
                float2 R = mul(T.That[tq][0], J[0]);
#pragma unroll
                for (int m = 1; m <= j; ++m) R = fma(T.That[tq][m], J[m], R);
                G[q] = mul(up[j], R);
            }
    }
    const float2 ux = mul(dx, rinv), uy = mul(dy, rinv), uz = mul(dz, rinv);
    float2 C[P + 1], S[P + 1];
    C[0] = dup(1.f);
    S[0] = dup(0.f);
#pragma unroll
    for (int m = 1; m <= P; ++m) {
        C[m] = fma(ux, C[m - 1], neg(mul(uy, S[m - 1])));
        S[m] = fma(ux, S[m - 1], mul(uy, C[m - 1]));
    }
    float2 pm2[P + 1], pm1[P + 1];
#pragma unroll
    for (int m = 0; m <= P; ++m) pm2[m] = pm1[m] = dup(0.f);
    harmonic_level<P, 0>(uz, C, S, pm1, pm2, G, T, put);
}

template <int P, int PREC>
struct Tc3Shape {
    using S = TcShape<3, P, PREC>;
    static constexpr int NT = S::NT, NTP = S::NTP;
    static constexpr int PLANE_COLS = NTP / 2;                          // packed BF16 pairs per plane
    static constexpr int BUF_COLS = S::PLANES * PLANE_COLS;              // one entry's A buffer
    static constexpr int COL_A0 = 32, COL_A1 = 32 + BUF_COLS;
    static constexpr int USED = 32 + 2 * BUF_COLS;
    static constexpr int TMEM_COLS = USED <= 64 ? 64 : USED <= 128 ? 128 : USED <= 256 ? 256 : 512;
    static constexpr int ST = 6;                                         // multipole stages (entries)
    static constexpr int THREADS = 160;
    static constexpr size_t smem_bytes() { return (size_t)ST * S::B_BYTES + (size_t)kTcN * 128 * 4 + 128; }
    static constexpr bool supported = PREC != TC_TF32 && TMEM_COLS <= 256 && smem_bytes() <= 110 * 1024;
};

// Warp roles: warps 0-3 = targets (thread = target = TMEM lane), warp 4 = producer (metadata
// window, bulk copies of the multipoles ST entries ahead, MMA issue).  Round k handles entries 2k
// and 2k+1 (the second absent when the block's entry count is odd).  The hand-offs go through two
// named barriers -- targets -> issuer once the rows of pair k are stored, issuer -> targets once
// its MMAs are complete (one thread polls their commit) -- so waiting target warps are
// descheduled instead of polling.  Both roles run npairs rounds whatever happens; a copy wait that
// runs out (bounded) sets s_fail, which only skips work, and the producer drains what it issued
// before the CTA frees its tensor memory.
template <int P, int PREC>
__global__ void __launch_bounds__(160, Tc3Shape<P, PREC>::TMEM_COLS <= 128 ? 4 : 2) far_tc3_kernel(MvmArgs a, KernelParams kp_all,
                                                         const __grid_constant__ FarTables2 T,
                                                         const unsigned char* __restrict__ image, int nr_total) {
    using Sh = Tc3Shape<P, PREC>;
    using S = typename Sh::S;
    constexpr int NT = Sh::NT, NTP = Sh::NTP, ST = Sh::ST, BB = S::B_BYTES, BPLANE = kTcN * NTP * 2;
    constexpr int kFlushPairs = 2;   // 2 pairs = 4 entries = 72 MMAs (BF16 hi/lo) per accumulator flush
    constexpr uint32_t IDESC = tc::instr_desc(1u, 128u, (uint32_t)kTcN);
    // named barriers: targets -> issuer (rows stored), issuer -> targets (MMAs complete)
    constexpr uint32_t kBarReady = 1, kBarMma = 2, kBarThreads = Sh::THREADS;
    extern __shared__ __align__(128) unsigned char tc3_smem[];
    unsigned char* Bbuf = tc3_smem;                                  // [ST][B_BYTES]
    float* accs = reinterpret_cast<float*>(tc3_smem + ST * BB);      // [kTcN][128] float32 sums
    __shared__ FarTc2Info info[ST];
    __shared__ __align__(8) uint64_t full[ST], mma_done;
    __shared__ uint32_t tmem_base;
    __shared__ uint32_t s_valid[kMaskWords];
    __shared__ int s_fail;
    const int tl = threadIdx.x, warp = tl >> 5, lane = tl & 31;
    const int64_t blk = cta_block(a);
    const KernelParams kp = block_params(a, blk, kp_all);
    const int2 rg = a.blk[blk];
    const int t = rg.x + tl;
    const bool valid = warp < 4 && t < rg.y;
    const uint32_t vword = __ballot_sync(0xffffffffu, valid);
    const int64_t e0 = a.far_off[blk];
    const int ne = (int)(a.far_off[blk + 1] - e0);
    const int npairs = (ne + 1) / 2;
    if (tl == 0) {
#pragma unroll
        for (int s = 0; s < ST; ++s) ptx::mbar_init(&full[s], 1);
        ptx::mbar_init(&mma_done, 1);
        ptx::fence_mbar_init();
        s_fail = 0;
    }
    if (warp < 4 && lane == 0) s_valid[warp] = vword;
    if (warp == 0) {
        tc::alloc(&tmem_base, Sh::TMEM_COLS);
        tc::relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;

    if (warp == 4) {
        // ------------------------------------------------------------------ producer / issuer
        // The whole warp walks the entries through a 32-entry metadata window (one lane per
        // entry); lane 0 issues the bulk copies, the MMAs and the one poll of their completion.
        int wb = 0, wnode = 0;
        float4 wc = make_float4(0.f, 0.f, 0.f, 0.f);
        float ws = 0.f;
        uint32_t wm[kMaskWords] = {0u, 0u, 0u, 0u};
        auto load_window = [&]() {
            const int e = wb + lane;
            if (e < ne) {
                const int2 ent = a.far_ent[e0 + e];
                wnode = ent.x;
                wc = a.nd_cf[ent.x];
                ws = a.nd_scale[ent.x];
#pragma unroll
                for (int w = 0; w < kMaskWords; ++w)
                    wm[w] = (ent.y < 0 ? 0xFFFFFFFFu : __ldg(&a.masks[(int64_t)ent.y * kMaskWords + w])) & s_valid[w];
            }
        };
        int issued = 0;
        auto produce = [&]() {  // warp-collective: the next entry into its stage
            if (issued >= wb + 32) {
                wb += 32;
                load_window();
            }
            const int src = issued - wb, slot = issued % ST;
            const int node = __shfl_sync(0xffffffffu, wnode, src);
            const float cx = __shfl_sync(0xffffffffu, wc.x, src), cy = __shfl_sync(0xffffffffu, wc.y, src);
            const float cz = __shfl_sync(0xffffffffu, wc.z, src);
            const float sc = __shfl_sync(0xffffffffu, ws, src);
            uint32_t on[kMaskWords];
#pragma unroll
            for (int w = 0; w < kMaskWords; ++w) on[w] = __shfl_sync(0xffffffffu, wm[w], src);
            if (lane == 0) {
                FarTc2Info& in = info[slot];
                in.c = make_float4(cx, cy, cz, 0.f);
                in.s = sc;
#pragma unroll
                for (int w = 0; w < kMaskWords; ++w) in.on[w] = on[w];
                ptx::fence_proxy_async_smem();
                ptx::mbar_arrive_expect_tx(&full[slot], (uint32_t)BB);
                ptx::bulk_g2s(Bbuf + slot * BB, image + (int64_t)node * BB, (uint32_t)BB, &full[slot]);
            }
            ++issued;
        };
        if (ne > 0) load_window();
        while (issued < ST && issued < ne) produce();
        int committed = 0, waited = 0;
        for (int k = 0; k < npairs; ++k) {
            ptx::named_sync(kBarReady, kBarThreads);  // the rows of pair k are in tensor memory
            if (lane == 0 && !s_fail) {
                tc::fence_after_sync();
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int e = 2 * k + h;
                    if (e >= ne) break;
                    const int slot = e % ST;
                    uint32_t off[kMaskWords];
#pragma unroll
                    for (int w = 0; w < kMaskWords; ++w) off[w] = ~info[slot].on[w];
                    const unsigned char* B = Bbuf + slot * BB;
                    const uint32_t acol = h ? Sh::COL_A1 : Sh::COL_A0;
#pragma unroll 1
                    for (int ks = 0; ks < NTP / 16; ++ks) {
                        const uint64_t bh = tc::smem_desc(B + ks * 256, 128, S::SBO_A);
                        const uint32_t ahi = tmem + acol + ks * 8;
                        tc::mma_bf16_ts_masked(tmem, ahi, bh, IDESC, off);
                        if (PREC == TC_BF16X3) {
                            const uint64_t bl = tc::smem_desc(B + BPLANE + ks * 256, 128, S::SBO_A);
                            tc::mma_bf16_ts_masked(tmem, ahi, bl, IDESC, off);
                            tc::mma_bf16_ts_masked(tmem, tmem + acol + Sh::PLANE_COLS + ks * 8, bh, IDESC, off);
                        }
                    }
                }
                tc::commit(&mma_done);
                ++committed;
                if (ptx::mbar_wait_bounded(&mma_done, (uint32_t)((committed - 1) & 1), kWaitCycles)) waited = committed;
                else s_fail = 1;
                tc::fence_before_sync();
            }
            __syncwarp();
            ptx::named_arrive(kBarMma, kBarThreads);  // pair k's MMAs are complete (or skipped)
            // the stages of entries 2k and 2k+1 are free: refill them ST entries ahead
            if (__all_sync(0xffffffffu, !s_fail))  // warp-uniform: produce() shuffles
                while (issued < ne && issued <= 2 * k + 1 + ST) produce();
        }
        if (lane == 0 && s_fail) {
            atomicExch(a.err, 1);
            // the last copy of each stage may still be in flight; then the last MMAs
            for (int j = issued > ST ? issued - ST : 0; j < issued; ++j)
                ptx::mbar_wait_bounded(&full[j % ST], (uint32_t)((j / ST) & 1), kWaitCycles);
            if (waited < committed) ptx::mbar_wait_bounded(&mma_done, (uint32_t)(waited & 1), kWaitCycles);
        }
    } else {
        // ------------------------------------------------------------------ targets
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        const float4 xt = valid ? a.xs[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 m1 = make_float2(-1.f, -1.f);
        tc::st32_zero(tmem + lane_base);
        tc::wait_st();
#pragma unroll
        for (int r = 0; r < kTcN; ++r) accs[r * 128 + tl] = 0.f;
        auto flush = [&]() {
            float d[kTcN];
            tc::ld16(tmem + lane_base, d);
            tc::ld16(tmem + lane_base + 16, d + 16);
#pragma unroll
            for (int r = 0; r < kTcN; ++r) accs[r * 128 + tl] += d[r];
        };
        bool dirty = false;
        // Every thread runs npairs rounds of the two named barriers whatever happens: a copy
        // wait that runs out sets s_fail, which only skips work.
        for (int k = 0; k < npairs; ++k) {
            const int ea = 2 * k, eb = 2 * k + 1;
            const bool has_b = eb < ne;
            const int sa = ea % ST, sb = eb % ST;
            bool got = ptx::mbar_wait_bounded(&full[sa], (uint32_t)((ea / ST) & 1), a.wait_cycles);
            if (has_b) got = got && ptx::mbar_wait_bounded(&full[sb], (uint32_t)((eb / ST) & 1), a.wait_cycles);
            if (!__all_sync(0xffffffffu, got)) s_fail = 1;
            const bool work = !s_fail;
            bool waited = k == 0;
            auto wait_prev = [&]() {  // warp-uniform: the MMAs of pair k-1 are complete
                if (!waited) {
                    ptx::named_sync(kBarMma, kBarThreads);
                    waited = true;
                    tc::fence_after_sync();
                }
            };
            bool stored = false;
            if (k % kFlushPairs == 0 && dirty) {
                wait_prev();
                if (!s_fail) {
                    flush();
                    tc::st32_zero(tmem + lane_base);
                    stored = true;
                }
                dirty = false;
            }
            const uint32_t ma = work ? info[sa].on[warp] : 0u;
            const uint32_t mb = work && has_b ? info[sb].on[warp] : 0u;
            if ((ma | mb) != 0u) {
                const float4 ca = info[sa].c, cb = has_b ? info[sb].c : ca;
                const float sca = info[sa].s, scb = has_b ? info[sb].s : sca;
                // a lane outside an entry's mask computes its row for that entry with a zero
                // kernel scale; the entry's MMAs leave that row disabled whatever it holds
                const bool ina = (ma >> lane) & 1u, inb = (mb >> lane) & 1u;
                const float2 kscale = make_float2(ina ? kp.scale : 0.f, inb ? kp.scale : 0.f);
                float2 buf[16];
                auto store_group = [&](int g) {  // terms 16g..16g+15 of both entries
                    // hi = the BF16 rounding of each term, lo = the BF16 rounding of term - hi;
                    // v0 = (term 2i of entry a, of entry b), v1 = (term 2i+1 of a, of b)
                    uint32_t hia[8], loa[8], hib[8], lob[8];
#pragma unroll
                    for (int i2 = 0; i2 < 8; ++i2) {
                        const float2 v0 = buf[2 * i2], v1 = buf[2 * i2 + 1];
                        const uint32_t ha = bf2_bits(__floats2bfloat162_rn(v0.x, v1.x));
                        const uint32_t hb = bf2_bits(__floats2bfloat162_rn(v0.y, v1.y));
                        hia[i2] = ha;
                        hib[i2] = hb;
                        if (PREC == TC_BF16X3) {
                            const float2 h0 = make_float2(__uint_as_float(ha << 16), __uint_as_float(hb << 16));
                            const float2 h1 = make_float2(__uint_as_float(ha & 0xFFFF0000u),
                                                          __uint_as_float(hb & 0xFFFF0000u));
                            const float2 r0 = __ffma2_rn(h0, m1, v0), r1 = __ffma2_rn(h1, m1, v1);
                            loa[i2] = bf2_bits(__floats2bfloat162_rn(r0.x, r1.x));
                            lob[i2] = bf2_bits(__floats2bfloat162_rn(r0.y, r1.y));
                        }
                    }
                    if (g == 0) wait_prev();
                    if (ma != 0u) {
                        tc::st8(tmem + lane_base + Sh::COL_A0 + g * 8, hia);
                        if (PREC == TC_BF16X3) tc::st8(tmem + lane_base + Sh::COL_A0 + Sh::PLANE_COLS + g * 8, loa);
                    }
                    if (mb != 0u) {
                        tc::st8(tmem + lane_base + Sh::COL_A1 + g * 8, hib);
                        if (PREC == TC_BF16X3) tc::st8(tmem + lane_base + Sh::COL_A1 + Sh::PLANE_COLS + g * 8, lob);
                    }
                };
                far_basis2<P>(xt, make_float2(ca.x, cb.x), make_float2(ca.y, cb.y), make_float2(ca.z, cb.z),
                              make_float2(sca, scb), kscale, kp, T, [&](int q, float2 v) {
                                  buf[q & 15] = v;
                                  if (q == NT - 1) {
#pragma unroll
                                      for (int z = (q & 15) + 1; z < 16; ++z) buf[z] = make_float2(0.f, 0.f);
                                      store_group(q >> 4);
                                  } else if ((q & 15) == 15) {
                                      store_group(q >> 4);
                                  }
                              });
                dirty = true;
                stored = true;
            }
            wait_prev();
            if (stored) tc::wait_st();
            tc::fence_before_sync();
            __syncwarp();
            ptx::named_arrive(kBarReady, kBarThreads);
        }
        if (npairs >= 1) ptx::named_sync(kBarMma, kBarThreads);  // the last pair's MMAs are complete
        tc::fence_after_sync();
        const bool ok = !s_fail;
        if (ok && dirty) flush();
        __syncwarp();
        if (ok && valid)
#pragma unroll 4
            for (int r = 0; r < kTcN; ++r)
                if (r < nr_total) a.yfar[(int64_t)r * a.N + t] = accs[r * 128 + tl];
        if (!ok && tl == 0) atomicExch(a.err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::dealloc(tmem, Sh::TMEM_COLS);
}

}  // namespace fkt
