// Far field on the tensor cores, d = 3, BF16 / BF16 hi+lo, one far entry per thread and round
// (included by far_tc.cuh after Tc2Shape and FarTc2Info).
//
// Per 128-target block: z[t][r] += sum_b U_b[t][q] M_b[q][r], U_b[t][q] = Yt_kh(x_t - c_b)
// (s_b/r)^j R_kj(r) (Theorem 3.1, eq. finaltrunc).  Warps 0-3 (thread = target = tensor-memory
// lane) generate the basis row of each far entry that a target of their warp takes -- radial
// jets and sums first, then the harmonics in increasing term order -- and store it 16 terms at a
// time as packed BF16 pairs (hi and lo planes) into tensor memory, the A operand of
// tcgen05.mma.kind::f16.  Warp 4 resolves the entries through a 32-entry metadata window,
// bulk-copies each node's packed multipoles ST entries ahead, issues the entry's MMAs with the
// rows outside its mask disabled, and polls their completion (one thread).  The two hand-offs go
// through named barriers, so waiting target warps are descheduled instead of polling.  Every
// kFarFlush entries the targets add the accumulator into float32 sums in shared memory (the
// tensor core's accumulation is not round-to-nearest).  Tensor memory: 32 + 96 columns at p = 6,
// four CTAs per SM.
#pragma once

namespace fkt {

// Scalar harmonics of degree L and above (compile-time recursion: constant array indices), as
// harmonic_level for packed pairs.
template <int P, int LD, int L, class F>
__device__ __forceinline__ void harmonic_level1(float uz, const float (&C)[P + 1], const float (&S)[P + 1],
                                                float (&pm1)[P + 1], float (&pm2)[P + 1],
                                                const float (&G)[Layout<LD, P>::npairs], const FarTables& T, F&& put) {
    using Lay = Layout<LD, P>;
    float cur[L + 1];
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        if (m == L) cur[m] = T.hSeed[m];
        else if (m == L - 1) cur[m] = T.hA[L][m] * (uz * pm1[m]);
        else cur[m] = fmaf(T.hA[L][m], uz * pm1[m], -T.hB[L][m] * pm2[m]);
    }
    constexpr int o = Lay::off(L), nj = Lay::nj(L), g = Lay::pair(L);
#pragma unroll
    for (int jj = 0; jj < nj; ++jj) put(o + jj, cur[0] * G[g + jj]);
#pragma unroll
    for (int m = 1; m <= L; ++m) {
        const float yc = cur[m] * C[m], ys = cur[m] * S[m];
#pragma unroll
        for (int jj = 0; jj < nj; ++jj) put(o + (2 * m - 1) * nj + jj, yc * G[g + jj]);
#pragma unroll
        for (int jj = 0; jj < nj; ++jj) put(o + 2 * m * nj + jj, ys * G[g + jj]);
    }
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        pm2[m] = pm1[m];
        pm1[m] = cur[m];
    }
    if constexpr (L < P) harmonic_level1<P, LD, L + 1>(uz, C, S, pm1, pm2, G, T, put);
}

// The basis row of one (target, far node) pair, put(q, U[q]) for q = 0..NT-1 in increasing order
// (the expansion of far_basis<LD, P>, with |u|^2 = 1 in the recurrence of the unit direction).
// LD = 3 or kDiag3 (layout codes of fkt_kernels.cuh).
template <int P, int LD, class F>
__device__ __forceinline__ void far_basis1(const float4& xt, const float4& c, float s, const KernelParams& kp,
                                           const FarTables& T, F&& put) {
    using Lay = Layout<LD, P>;
    const float dx = xt.x - c.x, dy = xt.y - c.y, dz = xt.z - c.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float u = s * rinv;
    float G[Lay::npairs];
    {
        float J[P + 1];
        kernel_jets<P>(kp, r, rinv, J);
        float up[P + 1];
        up[0] = 1.f;
#pragma unroll
        for (int j = 1; j <= P; ++j) up[j] = up[j - 1] * u;
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int jj = 0; jj < Lay::nj(k); ++jj) {
                const int j = k + 2 * jj, q = Lay::pair(k) + jj, tq = Lay::tpair(k, jj);
                float R = T.That[tq][0] * J[0];
#pragma unroll
                for (int m = 1; m <= j; ++m) R = fmaf(T.That[tq][m], J[m], R);
                G[q] = up[j] * R;
            }
    }
    const float ux = dx * rinv, uy = dy * rinv, uz = dz * rinv;
    float C[P + 1], S[P + 1];
    C[0] = 1.f;
    S[0] = 0.f;
#pragma unroll
    for (int m = 1; m <= P; ++m) {
        C[m] = fmaf(ux, C[m - 1], -uy * S[m - 1]);
        S[m] = fmaf(ux, S[m - 1], uy * C[m - 1]);
    }
    float pm2[P + 1], pm1[P + 1];
#pragma unroll
    for (int m = 0; m <= P; ++m) pm2[m] = pm1[m] = 0.f;
    harmonic_level1<P, LD, 0>(uz, C, S, pm1, pm2, G, T, put);
}

// HOLD > 0: the first HOLD 16-term groups of a row are kept in registers and stored only after
// the MMAs of the previous entry complete, so that almost the whole row is computed while they
// run; the extra registers allow three CTAs per SM instead of four.
template <int P, int PREC, int LD = 3, int HOLD = 0>
__global__ void __launch_bounds__(160, HOLD > 0 ? 3
                                      : Tc2Shape<P, PREC, LD>::NTP <= 96 ? 4 : Tc2Shape<P, PREC, LD>::NTP <= 128 ? 3 : 2)
    far_tc2_kernel(MvmArgs a, KernelParams kp_all, const __grid_constant__ FarTables T,
                   const unsigned char* __restrict__ image, int nr_total) {
    using Sh = Tc2Shape<P, PREC, LD>;
    static_assert(HOLD <= 6, "held groups live in registers");
    using S = typename Sh::S;
    constexpr int NT = Sh::NT, NTP = Sh::NTP, ST = Sh::ST, BB = S::B_BYTES, BPLANE = kTcN * NTP * 2;
    constexpr int kFarFlush = 4;
    constexpr uint32_t IDESC = tc::instr_desc(1u, 128u, (uint32_t)kTcN);
    constexpr uint32_t kBarReady = 1, kBarMma = 2, kBarThreads = Sh::THREADS;
    extern __shared__ __align__(128) unsigned char tc2_smem[];
    unsigned char* Bbuf = tc2_smem;                                  // [ST][B_BYTES]
    float* accs = reinterpret_cast<float*>(tc2_smem + ST * BB);      // [kTcN][128] float32 sums
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
        const uint64_t desc0 = tc::smem_desc(Bbuf, 128, S::SBO_A);  // B hi of stage 0, K-step 0
        static_assert(BB % 16 == 0 && BPLANE % 16 == 0, "descriptor offsets in 16-byte units");
        int committed = 0, waited = 0;
        for (int i = 0; i < ne; ++i) {
            ptx::named_sync(kBarReady, kBarThreads);  // the rows of entry i are in tensor memory
            if (lane == 0 && !s_fail) {
                tc::fence_after_sync();
                const int slot = i % ST;
                uint32_t off[kMaskWords];
#pragma unroll
                for (int w = 0; w < kMaskWords; ++w) off[w] = ~info[slot].on[w];
                // descriptors: stage 0's base plus byte offsets / 16 in the start-address field
                // (shared addresses stay below 2^18 bytes, so the 14-bit field cannot carry)
                const uint64_t d0 = desc0 + (uint64_t)(slot * (BB >> 4));
#pragma unroll 1
                for (int ks = 0; ks < NTP / 16; ++ks) {
                    const uint64_t bh = d0 + (uint64_t)(ks * 16);
                    const uint32_t ahi = tmem + Sh::COL_AHI + ks * 8;
                    if (PREC == TC_BF16X3)
                        tc::mma3_bf16_ts_masked(tmem, ahi, tmem + Sh::COL_ALO + ks * 8, bh, bh + (uint64_t)(BPLANE >> 4),
                                                IDESC, off);
                    else
                        tc::mma_bf16_ts_masked(tmem, ahi, bh, IDESC, off);
                }
                tc::commit(&mma_done);
                ++committed;
                if (ptx::mbar_wait_bounded(&mma_done, (uint32_t)((committed - 1) & 1), kWaitCycles)) waited = committed;
                else s_fail = 1;
                tc::fence_before_sync();
            }
            __syncwarp();
            ptx::named_arrive(kBarMma, kBarThreads);  // entry i's MMAs are complete (or skipped)
            // entry i's stage is free: refill it ST entries ahead
            if (__all_sync(0xffffffffu, !s_fail))  // warp-uniform: produce() shuffles
                while (issued < ne && issued <= i + ST) produce();
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
        // Every thread runs ne rounds of the two named barriers whatever happens: a copy wait
        // that runs out sets s_fail, which only skips work.
        for (int i = 0; i < ne; ++i) {
            const int slot = i % ST;
            const bool got = ptx::mbar_wait_bounded(&full[slot], (uint32_t)((i / ST) & 1), a.wait_cycles);
            if (!__all_sync(0xffffffffu, got)) s_fail = 1;
            bool waited = i == 0;
            auto wait_prev = [&]() {  // warp-uniform: the MMAs of entry i-1 are complete
                if (!waited) {
                    ptx::named_sync(kBarMma, kBarThreads);
                    waited = true;
                    tc::fence_after_sync();
                }
            };
            bool stored = false;
            if (i % kFarFlush == 0 && dirty) {
                wait_prev();
                if (!s_fail) {
                    flush();
                    tc::st32_zero(tmem + lane_base);
                    stored = true;
                }
                dirty = false;
            }
            const uint32_t mword = s_fail ? 0u : info[slot].on[warp];
            if (mword != 0u) {
                const float4 c = info[slot].c;
                const float sc = info[slot].s;
                float2 buf[8];  // terms 16g..16g+15 as pairs (2i, 2i+1)
                constexpr int NG = NTP / 16;
                uint32_t held_hi[HOLD > 0 ? HOLD : 1][8], held_lo[HOLD > 0 ? HOLD : 1][8];
                auto store_held = [&](int upto) {
#pragma unroll
                    for (int gg = 0; gg < (HOLD > 0 ? HOLD : 1); ++gg)
                        if (gg < upto) {
                            tc::st8(tmem + lane_base + Sh::COL_AHI + gg * 8, held_hi[gg]);
                            if (PREC == TC_BF16X3) tc::st8(tmem + lane_base + Sh::COL_ALO + gg * 8, held_lo[gg]);
                        }
                };
                auto store_group = [&](int g) {
                    // hi = the BF16 rounding of each term, lo = the BF16 rounding of term - hi
                    uint32_t hi[8], lo[8];
#pragma unroll
                    for (int i2 = 0; i2 < 8; ++i2) {
                        const float2 v = buf[i2];
                        const uint32_t h = bf2_bits(__floats2bfloat162_rn(v.x, v.y));
                        hi[i2] = h;
                        if (PREC == TC_BF16X3) {
                            const float2 hf = make_float2(__uint_as_float(h << 16), __uint_as_float(h & 0xFFFF0000u));
                            const float2 rr = __ffma2_rn(hf, m1, v);
                            lo[i2] = bf2_bits(__floats2bfloat162_rn(rr.x, rr.y));
                        }
                    }
                    if (g < HOLD) {
#pragma unroll
                        for (int i2 = 0; i2 < 8; ++i2) {
                            held_hi[g < HOLD ? g : 0][i2] = hi[i2];
                            held_lo[g < HOLD ? g : 0][i2] = lo[i2];
                        }
                        if (g == NG - 1) {  // the whole row was held
                            wait_prev();
                            store_held(NG);
                        }
                        return;
                    }
                    if (g == HOLD) {
                        wait_prev();
                        store_held(HOLD);
                    }
                    tc::st8(tmem + lane_base + Sh::COL_AHI + g * 8, hi);
                    if (PREC == TC_BF16X3) tc::st8(tmem + lane_base + Sh::COL_ALO + g * 8, lo);
                };
                far_basis1<P, LD>(xt, c, sc, kp, T, [&](int q, float v) {
                    if (q & 1) buf[(q & 15) >> 1].y = v;
                    else buf[(q & 15) >> 1].x = v;
                    if (q == NT - 1) {
                        if (!(q & 1)) buf[(q & 15) >> 1].y = 0.f;
#pragma unroll
                        for (int z = ((q & 15) >> 1) + 1; z < 8; ++z) buf[z] = make_float2(0.f, 0.f);
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
        if (ne >= 1) ptx::named_sync(kBarMma, kBarThreads);  // the last entry's MMAs are complete
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
