// Near field of 32-wide passes on the 5th-generation tensor cores.
//
// For one block of 128 targets and one chunk of up to 32 sources of a near leaf the near field is
// the dense product (Algorithm 1, the near-field sum of eq. nbody over the leaf)
//     z[t][r] += sum_s K(|x_t - x_s|) w[s][r]        (128 x 32) += (128 x 32) (32 x 32).
// The CUDA cores evaluate the kernel values in float32, one target row per thread, and write the
// row straight into tensor memory as the A operand (tcgen05.st); one thread issues tcgen05.mma
// (kind::tf32, A from tensor memory, M = 128 targets, N = 32 right-hand sides, K = 8 sources per
// instruction) into a float32 accumulator in tensor memory.  The B operand (the chunk's weights,
// split hi/lo) and the chunk's source coordinates come ready-made from the pass's near-field
// image (near_image_kernel, once per pass): the bulk copy lands them in shared memory in the
// layout the MMA and the target threads read, so no thread rearranges weights per chunk.
//
// float32 accuracy from TF32 operands: every factor v is split into hi = v with 10 mantissa bits
// (the weights rounded to nearest once per pass; the kernel values truncated, one instruction
// per value) and lo = v - hi (exact in float32, |lo| <= 2^-10 |v|); the tensor core adds
// hi*hi + hi*lo + lo*hi.  The dropped lo*lo and the truncation of lo to TF32 leave at most about
// 2^-20 of each product.  The tensor core's own float32 accumulation is not
// round-to-nearest: summed over the thousands of MMAs of a target block it drifts by about 2^-24
// per MMA in one direction (measured: 2e-5 relative after ~600 MMAs).  So every few chunks each
// thread adds its accumulator row into float32 sums (round-to-nearest) and zeroes it.
#pragma once

#include "mvm_kernels.cuh"

namespace fkt {

struct NearTcShape {
    static constexpr int NR = 32;                     // right-hand sides (the MMA's N)
    static constexpr int CH = 32;                     // sources per chunk (4 MMA K-steps of 8)
    static constexpr int ST = 4;                      // chunk stages in flight
    static constexpr int CONSUMERS = 4;               // warps that own the 128 TMEM lanes / targets
    static constexpr int THREADS = 32 * (CONSUMERS + 1);  // + one producer / MMA-issuer warp
    static constexpr int TMEM_COLS = 128;             // accumulator 32 + A hi 32 + A lo 32 + float32 sums 32
    static constexpr int COL_AHI = 32, COL_ALO = 64, COL_SUM = 96;
    static constexpr int FLUSH = 4;                   // chunks (12 MMAs each) per float32 flush
    static constexpr int SMEM_BYTES = ST * kNearChunkBytes;  // chunk stages
};

namespace tc {

// 16 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void st16(uint32_t taddr, const uint32_t v[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

// D[tmem] += A[tmem] * B[smem]^T (BF16 operands), accumulator rows with a set bit in off[] untouched.
__device__ __forceinline__ void mma_bf16_ts_masked(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                                   const uint32_t off[4]) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, 1, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, {%4, %5, %6, %7}, p;\n"
        "}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(off[0]), "r"(off[1]), "r"(off[2]), "r"(off[3])
        : "memory");
}

// 4 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void st4(uint32_t taddr, const uint32_t v[4]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v[0]), "r"(v[1]),
                 "r"(v[2]), "r"(v[3])
                 : "memory");
}
// One K-step of the BF16 hi/lo product, D += Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T, as one asm block
// of three MMAs sharing their operands, rows with a set bit in off[] untouched.
__device__ __forceinline__ void mma3_bf16_ts_masked(uint32_t d_tmem, uint32_t ahi, uint32_t alo, uint64_t bhi,
                                                    uint64_t blo, uint32_t idesc, const uint32_t off[4]) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, 1, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %3, %5, {%6, %7, %8, %9}, p;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %4, %5, {%6, %7, %8, %9}, p;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%2], %3, %5, {%6, %7, %8, %9}, p;\n"
        "}\n" ::"r"(d_tmem),
        "r"(ahi), "r"(alo), "l"(bhi), "l"(blo), "r"(idesc), "r"(off[0]), "r"(off[1]), "r"(off[2]), "r"(off[3])
        : "memory");
}

// 8 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void st8(uint32_t taddr, const uint32_t v[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

// Zero 32 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void st32_zero(uint32_t taddr) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
        "r"(0u)
        : "memory");
}
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Every K-step of one near chunk (nks = 1..4 steps of 8 sources) in one asm block: for K-step k
// the hi/lo product D += Ahi_k Bhi_k^T + Ahi_k Blo_k^T + Alo_k Bhi_k^T, with A column offsets 8k
// and B descriptors bh + 136 k (hi) and bh + 136 k + 32 (lo) in 16-byte units (the near-field
// image's 2176-byte K-steps, lo plane 512 bytes after hi).  The operands enter once for all
// twelve MMAs; rows with a set bit in off[] are left untouched.
__device__ __forceinline__ void near_chunk_mma(uint32_t d_tmem, uint32_t ahi, uint32_t alo, uint64_t bh, int nks,
                                               uint32_t idesc, const uint32_t off[4]) {
    asm volatile(
        "{\n"
        ".reg .pred p, q1, q2, q3;\n"
        ".reg .b64 h0, l0, h1, l1, h2, l2, h3, l3;\n"
        ".reg .b32 ah1, al1, ah2, al2, ah3, al3;\n"
        "setp.ne.b32 p, 1, 0;\n"
        "setp.gt.s32 q1, %4, 1;\n"
        "setp.gt.s32 q2, %4, 2;\n"
        "setp.gt.s32 q3, %4, 3;\n"
        "mov.b64 h0, %3;\n"
        "add.s64 l0, %3, 32;\n"
        "add.s64 h1, %3, 136;\n"
        "add.s64 l1, %3, 168;\n"
        "add.s64 h2, %3, 272;\n"
        "add.s64 l2, %3, 304;\n"
        "add.s64 h3, %3, 408;\n"
        "add.s64 l3, %3, 440;\n"
        "add.u32 ah1, %1, 8;\n"
        "add.u32 al1, %2, 8;\n"
        "add.u32 ah2, %1, 16;\n"
        "add.u32 al2, %2, 16;\n"
        "add.u32 ah3, %1, 24;\n"
        "add.u32 al3, %2, 24;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], h0, %5, {%6, %7, %8, %9}, p;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], l0, %5, {%6, %7, %8, %9}, p;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%2], h0, %5, {%6, %7, %8, %9}, p;\n"
        "@q1 tcgen05.mma.cta_group::1.kind::tf32 [%0], [ah1], h1, %5, {%6, %7, %8, %9}, p;\n"
        "@q1 tcgen05.mma.cta_group::1.kind::tf32 [%0], [ah1], l1, %5, {%6, %7, %8, %9}, p;\n"
        "@q1 tcgen05.mma.cta_group::1.kind::tf32 [%0], [al1], h1, %5, {%6, %7, %8, %9}, p;\n"
        "@q2 tcgen05.mma.cta_group::1.kind::tf32 [%0], [ah2], h2, %5, {%6, %7, %8, %9}, p;\n"
        "@q2 tcgen05.mma.cta_group::1.kind::tf32 [%0], [ah2], l2, %5, {%6, %7, %8, %9}, p;\n"
        "@q2 tcgen05.mma.cta_group::1.kind::tf32 [%0], [al2], h2, %5, {%6, %7, %8, %9}, p;\n"
        "@q3 tcgen05.mma.cta_group::1.kind::tf32 [%0], [ah3], h3, %5, {%6, %7, %8, %9}, p;\n"
        "@q3 tcgen05.mma.cta_group::1.kind::tf32 [%0], [ah3], l3, %5, {%6, %7, %8, %9}, p;\n"
        "@q3 tcgen05.mma.cta_group::1.kind::tf32 [%0], [al3], h3, %5, {%6, %7, %8, %9}, p;\n"
        "}\n" ::"r"(d_tmem),
        "r"(ahi), "r"(alo), "l"(bh), "r"(nks), "r"(idesc), "r"(off[0]), "r"(off[1]), "r"(off[2]), "r"(off[3])
        : "memory");
}

}  // namespace tc

// v = hi + lo with hi representable in TF32 (round half away from zero on the 13 dropped bits).
__device__ __forceinline__ void split_tf32(float v, uint32_t& hi, uint32_t& lo) {
    const uint32_t h = (__float_as_uint(v) + 0x1000u) & 0xFFFFE000u;
    hi = h;
    lo = __float_as_uint(v - __uint_as_float(h));
}

// Kernel values of two pairs at once (the same formulas as kval, with the non-MUFU arithmetic on
// packed float32 pairs); q = squared distances in the kernel's own units.
template <int KIND>
__device__ __forceinline__ float2 kval2(float2 q, const KernelParams& kp) {
    constexpr float kLn2 = 0.69314718055994531f;
    if (KIND == FKT_GAUSSIAN) {
        return make_float2(ptx::ex2(-q.x), ptx::ex2(-q.y));
    } else if (KIND == FKT_EXPONENTIAL) {
        return make_float2(ptx::ex2(-ptx::sqrt_approx(q.x)), ptx::ex2(-ptx::sqrt_approx(q.y)));
    } else if (KIND == FKT_MATERN32) {
        const float2 u = make_float2(ptx::sqrt_approx(q.x), ptx::sqrt_approx(q.y));
        const float2 e = make_float2(ptx::ex2(-u.x), ptx::ex2(-u.y));
        return __fmul2_rn(__ffma2_rn(u, make_float2(kLn2, kLn2), make_float2(1.f, 1.f)), e);
    } else if (KIND == FKT_MATERN52) {
        const float2 u = make_float2(ptx::sqrt_approx(q.x), ptx::sqrt_approx(q.y));
        const float2 e = make_float2(ptx::ex2(-u.x), ptx::ex2(-u.y));
        const float2 t = __fmul2_rn(u, make_float2(kLn2, kLn2));
        const float2 poly = __ffma2_rn(t, __ffma2_rn(t, make_float2(1.f / 3.f, 1.f / 3.f), make_float2(1.f, 1.f)),
                                       make_float2(1.f, 1.f));
        return __fmul2_rn(poly, e);
    } else if (KIND == FKT_CAUCHY) {
        const float2 b = __fadd2_rn(q, make_float2(1.f, 1.f));
        return make_float2(ptx::rcp_approx(b.x), ptx::rcp_approx(b.y));
    } else if (KIND == FKT_RATQUAD) {
        const float2 b = __fadd2_rn(q, make_float2(1.f, 1.f));
        if (kp.alpha == 1.0f) return make_float2(ptx::rcp_approx(b.x), ptx::rcp_approx(b.y));
        return make_float2(ptx::ex2(-kp.alpha * ptx::lg2(b.x)), ptx::ex2(-kp.alpha * ptx::lg2(b.y)));
    } else {
        return make_float2(q.x > 0.0f ? ptx::rsqrt_approx(q.x) : 0.0f, q.y > 0.0f ? ptx::rsqrt_approx(q.y) : 0.0f);
    }
}

// Two kernel values -> their TF32 hi parts (bits: v truncated to 10 mantissa bits) and float32
// lo = v - hi (exact, same sign as v, |lo| < 2^-10 |v|).
__device__ __forceinline__ void split2(float2 v, uint32_t& h0, uint32_t& h1, uint32_t& l0, uint32_t& l1) {
    h0 = __float_as_uint(v.x) & 0xFFFFE000u;
    h1 = __float_as_uint(v.y) & 0xFFFFE000u;
    const float2 lo = __ffma2_rn(make_float2(__uint_as_float(h0), __uint_as_float(h1)), make_float2(-1.f, -1.f), v);
    l0 = __float_as_uint(lo.x);
    l1 = __float_as_uint(lo.y);
}

__device__ __forceinline__ void acc_store(const MvmArgs& a, int r, int t, float v) { a.ynear[(int64_t)r * a.N + t] = v; }

// acc[r] += this thread's accumulator row (32 columns at taddr).
__device__ __forceinline__ void add_partial(uint32_t taddr, float acc[32]) {
    float d[32];
    tc::ld16(taddr, d);
    tc::ld16(taddr + 16, d + 16);
#pragma unroll
    for (int r = 0; r < 32; ++r) acc[r] += d[r];
}

// Per chunk stage: what the producer resolved for the chunk it holds.
struct NearChunkInfo {
    int n;                     // sources in the chunk
    uint32_t on[kMaskWords];   // targets (TMEM lanes) that use the chunk's leaf
};

// One CTA per 128-target block, warp-specialised:
//   warps 0-3 (consumers, thread = target = TMEM lane): per chunk c of up to 32 sources, wait for
//     its image stage; a warp with a target in the chunk's mask evaluates its rows (float32
//     kernel values against the stage's coordinates, split hi/lo) into registers; wait (named
//     barrier) until the MMAs of chunk c-1 are complete, which frees the A columns; every FLUSH
//     chunks add the accumulator rows into the float32 sums and zero them; store the rows into
//     tensor memory; then arrive on the ready barrier.
//   warp 4 (producer / MMA issuer, lane 0 works): resolves chunk metadata from the lists and
//     bulk-copies image chunks ST ahead; per chunk syncs on the ready barrier, issues 3 MMAs per
//     8 sources (B straight from the stage; rows outside the mask disabled), waits for them,
//     arrives on the MMA barrier and refills the stage.
// Hand-offs between the roles use named barriers, so waiting warps are descheduled instead of
// polling.  Both roles run the same number of rounds (the block's chunk count, counted by all
// threads up front) whatever happens: a bounded mbarrier wait that runs out sets s_fail, which
// only skips work, and the producer drains what it issued before the CTA frees tensor memory.
template <int D, int KIND>
__global__ void __launch_bounds__(NearTcShape::THREADS, 4) near_tc_kernel(MvmArgs a, KernelParams kp_all) {
    using S = NearTcShape;
    constexpr int CH = S::CH, ST = S::ST, NR = S::NR, NC = S::CONSUMERS, GF = kNearGroupFloats;
    constexpr uint32_t IDESC = tc::instr_desc(2u, 128u, (uint32_t)NR);
    constexpr uint32_t kBarReady = 1, kBarMma = 2, kBarThreads = S::THREADS;
    extern __shared__ __align__(128) unsigned char near_smem[];
    float* stage = reinterpret_cast<float*>(near_smem);  // [ST][8 groups][GF]
    __shared__ NearChunkInfo info[ST];
    __shared__ __align__(8) uint64_t full[ST], mma_done;
    __shared__ uint32_t tmem_base;
    __shared__ uint32_t s_valid[kMaskWords];
    __shared__ int s_fail, s_nch;
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
        ptx::mbar_init(&mma_done, 1);
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

    if (warp == NC) {
        // ---------------------------------------------------------------- producer / issuer
        // The whole warp walks the chunk sequence in step: every lane holds the image position,
        // source count and row mask of one entry of a 32-entry window (loaded together, one
        // memory latency per 32 entries), lane 0 issues the copies.
        int64_t wbase = e0;
        int wimg = 0, wn = 0;
        uint32_t wm[kMaskWords] = {0u, 0u, 0u, 0u};
        auto load_window = [&]() {
            const int64_t e = wbase + lane;
            wimg = wn = 0;
            if (e < e1) {
                const int2 ent = a.near_ent[e];
                wimg = a.nd_img[ent.x];
                wn = a.nd_end[ent.x] - a.nd_begin[ent.x];
#pragma unroll
                for (int w = 0; w < kMaskWords; ++w)
                    wm[w] = (ent.y < 0 ? 0xFFFFFFFFu : __ldg(&a.masks[(int64_t)ent.y * kMaskWords + w])) & s_valid[w];
            }
        };
        int ei = 0, img0 = 0, cb = 0, cend = 0, issued = 0;
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
                img0 = __shfl_sync(0xffffffffu, wimg, ei);
                cend = __shfl_sync(0xffffffffu, wn, ei);
                cb = 0;
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
                const uint32_t bytes = (uint32_t)((n + 7) / 8) * 2u * kNearGroupBytes;
                ptx::mbar_arrive_expect_tx(&full[slot], bytes);
                ptx::bulk_g2s(stage + slot * 8 * GF, a.nimg + (int64_t)((img0 + cb) / 4) * GF, bytes, &full[slot]);
            }
            ++issued;
            cb += CH;
            settle();
        };
        if (!pdone) {
            load_window();
            img0 = __shfl_sync(0xffffffffu, wimg, 0);
            cend = __shfl_sync(0xffffffffu, wn, 0);
            cb = 0;
            settle();
        }
        for (int s = 0; s < ST; ++s) produce();
        const uint64_t desc0 = tc::smem_desc(stage, kNearGroupBytes, 128);  // B hi of stage 0, K-step 0
        int waited_mma = 0, committed = 0;
        for (int c = 0; c < nch; ++c) {
            const int slot = c % ST;
            ptx::named_sync(kBarReady, kBarThreads);
            if (lane == 0 && !s_fail) {
                tc::fence_after_sync();
                const NearChunkInfo in = info[slot];
                const uint32_t off[kMaskWords] = {~in.on[0], ~in.on[1], ~in.on[2], ~in.on[3]};
                const int nks = (in.n + 7) / 8;
                // descriptors: the stage base plus byte offsets / 16 in the start-address field
                // (shared addresses stay below 2^18 bytes, so the 14-bit field cannot carry)
                const uint64_t d0 = desc0 + (uint64_t)(slot * (kNearChunkBytes >> 4));
                static_assert(2 * kNearGroupBytes / 16 == 136 && 128 * 4 / 16 == 32, "near_chunk_mma offsets");
                tc::near_chunk_mma(tmem, tmem + S::COL_AHI, tmem + S::COL_ALO, d0, nks, IDESC, off);
                tc::commit(&mma_done);
                ++committed;
                if (ptx::mbar_wait_bounded(&mma_done, (uint32_t)((committed - 1) & 1), kWaitCycles)) waited_mma = committed;
                else s_fail = 1;
                tc::fence_before_sync();
            }
            __syncwarp();
            ptx::named_arrive(kBarMma, kBarThreads);
            // after releasing the consumers: every consumer has read stage `slot` and its MMAs
            // are complete, refill it ST chunks ahead
            if (__all_sync(0xffffffffu, !s_fail)) {  // warp-uniform: produce() shuffles
                if (lane == 0) ptx::fence_proxy_async_smem();
                produce();
            }
        }
        if (lane == 0 && s_fail) {
            atomicExch(a.err, 1);
            // the last copy of each stage may still be in flight; then the last MMAs
            for (int j = issued > ST ? issued - ST : 0; j < issued; ++j)
                ptx::mbar_wait_bounded(&full[j % ST], (uint32_t)((j / ST) & 1), kWaitCycles);
            if (waited_mma < committed) ptx::mbar_wait_bounded(&mma_done, (uint32_t)(waited_mma & 1), kWaitCycles);
        }
    } else {
        // ---------------------------------------------------------------- consumers
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        float2 tx2[4];  // this target (scaled by sigma), duplicated for the packed pair arithmetic
        {
            const float4 x = valid ? a.xs[t] : make_float4(0.f, 0.f, 0.f, 0.f);
            tx2[0] = make_float2(x.x * kp.sig, x.x * kp.sig);
            tx2[1] = make_float2(x.y * kp.sig, x.y * kp.sig);
            tx2[2] = make_float2(x.z * kp.sig, x.z * kp.sig);
            tx2[3] = make_float2(x.w * kp.sig, x.w * kp.sig);
        }
        tc::st32_zero(tmem + lane_base);  // accumulator rows start at zero; every MMA accumulates
        tc::st32_zero(tmem + lane_base + S::COL_SUM);
        tc::wait_st();
        // accumulator row -> the float32 sums (tensor-memory columns COL_SUM..), 8 columns at a time
        auto flush = [&]() {
#pragma unroll
            for (int h = 0; h < NR; h += 4) {
                float d[4], sum[4];
                tc::ld4x2(tmem + lane_base + h, tmem + lane_base + S::COL_SUM + h, d, sum);
                uint32_t u[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) u[r] = __float_as_uint(sum[r] + d[r]);
                tc::st4(tmem + lane_base + S::COL_SUM + h, u);
            }
        };
        bool dirty = false;  // this warp's accumulator rows hold products not yet added to the sums
        for (int c = 0; c < nch; ++c) {
            const int slot = c % ST;
            const bool got = ptx::mbar_wait_bounded(&full[slot], (uint32_t)((c / ST) & 1), a.wait_cycles);
            if (!__all_sync(0xffffffffu, got)) s_fail = 1;
            const int n = info[slot].n;
            const uint32_t mword = s_fail ? 0u : info[slot].on[warp];
            const float* sg = stage + slot * 8 * GF + 256;  // coordinates of the stage's first group
            // this row's kernel values against the chunk, before waiting for the MMAs of chunk
            // c-1: the wait then overlaps useful work (registers; rows of targets outside the
            // mask are computed anyway when their warp is busy, and left out by the MMA).
            // Columns past the chunk's end meet zero weights (zero-padded groups) or are never
            // read (K-steps past ceil(n/8)).
            uint32_t khi[CH], klo[CH];
            if (mword != 0u) {
#pragma unroll
                for (int j4 = 0; j4 < CH; j4 += 4) {
                    if (j4 < 16 || n > 16) {  // the MMA reads only ceil(n/8) K-steps
                        const float* g = sg + (j4 / 4) * GF;
                        const float4 X = *reinterpret_cast<const float4*>(g);
                        const float4 Y = *reinterpret_cast<const float4*>(g + 4);
                        const float4 Z = *reinterpret_cast<const float4*>(g + 8);
                        float2 q[2];
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            const float2 dx = __fadd2_rn(tx2[0], hh ? make_float2(X.z, X.w) : make_float2(X.x, X.y));
                            const float2 dy = __fadd2_rn(tx2[1], hh ? make_float2(Y.z, Y.w) : make_float2(Y.x, Y.y));
                            const float2 dz = __fadd2_rn(tx2[2], hh ? make_float2(Z.z, Z.w) : make_float2(Z.x, Z.y));
                            q[hh] = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                        }
                        if (D == 4) {
                            const float4 W = *reinterpret_cast<const float4*>(g + 12);
                            const float2 dw0 = __fadd2_rn(tx2[3], make_float2(W.x, W.y));
                            const float2 dw1 = __fadd2_rn(tx2[3], make_float2(W.z, W.w));
                            q[0] = __ffma2_rn(dw0, dw0, q[0]);
                            q[1] = __ffma2_rn(dw1, dw1, q[1]);
                        }
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            const float2 kv = kval2<KIND>(q[hh], kp);
                            split2(kv, khi[j4 + 2 * hh], khi[j4 + 2 * hh + 1], klo[j4 + 2 * hh], klo[j4 + 2 * hh + 1]);
                        }
                    }
                }
            }
            if (c >= 1) ptx::named_sync(kBarMma, kBarThreads);  // the MMAs of chunk c-1 are done
            tc::fence_after_sync();
            const bool work = !s_fail;
            bool stored = false;
            if (work && c % S::FLUSH == 0 && dirty) {
                flush();
                tc::st32_zero(tmem + lane_base);
                dirty = false;
                stored = true;
            }
            if (work && mword != 0u) {  // A operand: the row into tensor memory
                tc::st16(tmem + lane_base + S::COL_AHI, khi);
                tc::st16(tmem + lane_base + S::COL_ALO, klo);
                if (n > 16) {
                    tc::st16(tmem + lane_base + S::COL_AHI + 16, khi + 16);
                    tc::st16(tmem + lane_base + S::COL_ALO + 16, klo + 16);
                }
                dirty = true;
                stored = true;
            }
            if (stored) tc::wait_st();
            // publish the A rows to the issuer
            tc::fence_before_sync();
            __syncwarp();
            ptx::named_arrive(kBarReady, kBarThreads);
        }
        if (nch >= 1) ptx::named_sync(kBarMma, kBarThreads);  // the MMAs of the last chunk are done
        tc::fence_after_sync();
        const bool ok = !s_fail;
        if (ok && dirty) {
            flush();
            tc::wait_st();
        }
        if (ok) {
#pragma unroll
            for (int h = 0; h < NR; h += 16) {
                float sum[16];
                tc::ld16(tmem + lane_base + S::COL_SUM + h, sum);
                if (valid)
#pragma unroll
                    for (int r = 0; r < 16; ++r)
                        if (h + r < a.nr) acc_store(a, h + r, t, sum[r] * kp.scale);
            }
        }
        if (!ok && tl == 0) atomicExch(a.err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::dealloc(tmem, S::TMEM_COLS);
}

// Near-field image of one 32-wide pass from its source records (layout: kNearGroupFloats).
// One CTA per node (non-leaves return); warp w packs the leaf's groups w, w + 8, ...: lane n
// loads the weights of right-hand side n of the group's 4 sources (coalesced along the record),
// splits them into TF32 hi / lo and stores 16 bytes of each plane; lanes 0-15 store the negated
// coordinates.  Positions past the leaf's last source get zero weights and coordinates.
__global__ void near_image_kernel(int64_t nnodes, const int32_t* __restrict__ nd_leaf,
                                  const int32_t* __restrict__ nd_begin, const int32_t* __restrict__ nd_end,
                                  const int32_t* __restrict__ nd_img, const float4* __restrict__ rec, int rec_f4,
                                  float* __restrict__ img);

// One launch of a near_tc_kernel instantiation with its dynamic shared memory (the attribute is
// set on the first launch of each instantiation).
template <void (*K)(MvmArgs, KernelParams)>
void launch_near_tc_one(unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, NearTcShape::SMEM_BYTES);
        attr = true;
    }
    K<<<grid, NearTcShape::THREADS, NearTcShape::SMEM_BYTES, st>>>(a, kp);
}

template <int D>
void launch_near_tc_dim(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp) {
    switch (kind) {
    case FKT_GAUSSIAN: launch_near_tc_one<near_tc_kernel<D, FKT_GAUSSIAN>>(grid, st, a, kp); break;
    case FKT_EXPONENTIAL: launch_near_tc_one<near_tc_kernel<D, FKT_EXPONENTIAL>>(grid, st, a, kp); break;
    case FKT_MATERN32: launch_near_tc_one<near_tc_kernel<D, FKT_MATERN32>>(grid, st, a, kp); break;
    case FKT_MATERN52: launch_near_tc_one<near_tc_kernel<D, FKT_MATERN52>>(grid, st, a, kp); break;
    case FKT_CAUCHY: launch_near_tc_one<near_tc_kernel<D, FKT_CAUCHY>>(grid, st, a, kp); break;
    case FKT_RATQUAD: launch_near_tc_one<near_tc_kernel<D, FKT_RATQUAD>>(grid, st, a, kp); break;
    default: launch_near_tc_one<near_tc_kernel<D, FKT_LAPLACE>>(grid, st, a, kp); break;
    }
}

}  // namespace fkt
