// Far field on the 5th-generation tensor cores (the precision form of the far field).
//
// For one block of 128 targets the far field is a product accumulated over its far nodes b:
//     z[t][r] += sum_q U_b[t][q] M_b[q][r],   U_b[t][q] = Yt_kh(x_t - c_b) (s/r)^j R_kj(r)
// (the same basis as far_kernel).  CUDA cores generate the 128 x NTP basis tile U_b into shared
// memory, converted to BF16 (or split into BF16 hi + lo, or TF32); the node's multipoles, packed
// beforehand into the tensor-core operand image, arrive by a bulk copy; one thread issues
// tcgen05.mma (M = 128 targets, N = 32 right-hand sides, K = 16 terms per instruction) into a
// float32 accumulator in tensor memory, which the epilogue reads back with tcgen05.ld.
//
// Operand layout (both K-major, no swizzle): core matrices of 8 rows x 16 bytes stored
// contiguously; the core matrices of one 8-row group follow each other along K (128 bytes
// apart, the leading-dimension offset), and 8-row groups are SBO = (NTP * elem / 16) * 128 bytes
// apart (the stride-dimension offset).
#pragma once

#include <cuda_bf16.h>

#include "near_tc.cuh"

namespace fkt {

enum TcPrec { TC_BF16 = 0, TC_BF16X3 = 1, TC_TF32 = 2 };

constexpr int kTcN = 32;  // right-hand-side columns per pass

template <int D, int P, int PREC>
struct TcShape {
    static constexpr int NT = Layout<D, P>::nterms;
    static constexpr int NTP = (NT + 15) / 16 * 16;                 // K padded to whole MMA steps
    static constexpr int EL = PREC == TC_TF32 ? 4 : 2;              // bytes per operand element
    static constexpr int PER16 = 16 / EL;                           // elements per 16-byte core row
    static constexpr int SBO_A = NTP / PER16 * 128;                 // bytes between 8-row groups
    static constexpr int PLANES = PREC == TC_BF16X3 ? 2 : 1;        // hi (+ lo)
    static constexpr int A_BYTES = 128 * NTP * EL * PLANES;
    static constexpr int B_BYTES = kTcN * NTP * EL * PLANES;
    // ROW: the target's whole basis row is kept in registers and written as 16-byte core rows
    // (NTP <= 128); otherwise each term is stored as it is generated.
    static constexpr bool ROW = NTP <= 128;
    static constexpr size_t smem_bytes() { return (size_t)A_BYTES + 2 * (size_t)B_BYTES + 128; }
    static constexpr bool supported = smem_bytes() <= 200 * 1024;
    // byte offset of element (row, k) of one plane
    __host__ __device__ static constexpr int off(int row, int k) {
        return (row / 8) * SBO_A + (k / PER16) * 128 + (row % 8) * 16 + (k % PER16) * EL;
    }
};

template <int PREC>
__device__ __forceinline__ void tc_store(unsigned char* plane0, int plane_bytes, int off, float v) {
    if (PREC == TC_TF32) {
        *reinterpret_cast<float*>(plane0 + off) = v;  // the tensor core reads the top 19 bits
    } else {
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        *reinterpret_cast<__nv_bfloat16*>(plane0 + off) = hi;
        if (PREC == TC_BF16X3)
            *reinterpret_cast<__nv_bfloat16*>(plane0 + plane_bytes + off) =
                __float2bfloat16_rn(v - __bfloat162float(hi));
    }
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) {
    uint32_t u;
    memcpy(&u, &v, sizeof(u));
    return u;
}

// One 16-byte core-matrix row (16 / elem consecutive terms) of one target: a single
// conflict-free 16-byte shared store per plane.
template <int PREC>
__device__ __forceinline__ void tc_store_row16(unsigned char* plane0, int plane_bytes, int off, const float* u) {
    if constexpr (PREC == TC_TF32) {
        *reinterpret_cast<float4*>(plane0 + off) = make_float4(u[0], u[1], u[2], u[3]);
    } else {
        __nv_bfloat162 h[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(u[2 * i], u[2 * i + 1]);
        *reinterpret_cast<uint4*>(plane0 + off) = make_uint4(bf2_bits(h[0]), bf2_bits(h[1]), bf2_bits(h[2]), bf2_bits(h[3]));
        if constexpr (PREC == TC_BF16X3) {
            __nv_bfloat162 l[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 f = __bfloat1622float2(h[i]);
                l[i] = __floats2bfloat162_rn(u[2 * i] - f.x, u[2 * i + 1] - f.y);
            }
            *reinterpret_cast<uint4*>(plane0 + plane_bytes + off) =
                make_uint4(bf2_bits(l[0]), bf2_bits(l[1]), bf2_bits(l[2]), bf2_bits(l[3]));
        }
    }
}

// Pack node multipoles (float32, [group][node][NT][8]) into the B-operand image of one pass of
// kTcN right-hand sides: rows = right-hand sides, columns = terms (K-major).
template <int D, int P, int PREC>
__global__ void tc_pack_kernel(int64_t nnodes, const int64_t* __restrict__ item_off, const float* __restrict__ mult,
                               int64_t group_stride, int nr_total, unsigned char* __restrict__ image) {
    using S = TcShape<D, P, PREC>;
    const int64_t node = blockIdx.x;
    if (item_off[node] == item_off[node + 1]) return;  // no target uses this node
    unsigned char* img = image + node * (int64_t)S::B_BYTES;
    const int plane = kTcN * S::NTP * S::EL;
    for (int e = threadIdx.x; e < kTcN * S::NTP; e += blockDim.x) {
        const int n = e / S::NTP, k = e - n * S::NTP;
        float v = 0.f;
        if (k < S::NT && n < nr_total) v = mult[(n / 8) * group_stride + (node * S::NT + k) * 8 + (n % 8)];
        // B rows are right-hand sides: same core-matrix rule with kTcN rows
        tc_store<PREC>(img, plane, S::off(n, k), v);
    }
}

// Basis of one (target, far node) pair: calls put(q, value) for every term q < NT, in
// increasing q for D = 3.  U[t][q] = Yt_kh(x_t - c) (s/r)^j R_kj(r).
template <int D, int P, class F>
__device__ __forceinline__ void far_basis(const float4& xt, const float4& c, float s, const KernelParams& kp,
                                          const FarTables& T, F&& put) {
    using Lay = Layout<D, P>;
    const float dx = xt.x - c.x, dy = xt.y - c.y, dz = xt.z - c.z, dw = dim_of(D) == 4 ? xt.w - c.w : 0.f;
    const float r2 = dx * dx + dy * dy + dz * dz + dw * dw;
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float u = s * rinv;
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
        for (int jj = 0; jj < Lay::nj(k); ++jj) put(o + jj, Y * G[Lay::pair(k) + jj]);
    });
}

// Per target block: for each far entry i, the CTA writes the 128 x NTP basis tile into shared
// memory and one thread issues the MMAs against the node's packed multipoles (bulk-copied into
// a 2-slot ring one entry ahead).  In ROW mode each thread computes its basis row for entry i
// in registers while the MMAs of entry i - 1 still read the tile, and stores it after they
// complete.  Every wait is bounded; a wait that runs out sets the error word and the CTA
// drains what it issued before leaving.
template <int D, int P, int PREC>
__global__ void __launch_bounds__(kTB) far_tc_kernel(MvmArgs a, KernelParams kp_all, const __grid_constant__ FarTables T,
                                                      const unsigned char* __restrict__ image, int nr_total) {
    using S = TcShape<D, P, PREC>;
    constexpr int NT = S::NT, NTP = S::NTP, PER16 = S::PER16;
    constexpr int APLANE = 128 * NTP * S::EL, BPLANE = kTcN * NTP * S::EL;
    constexpr uint32_t IDESC = tc::instr_desc(PREC == TC_TF32 ? 2u : 1u, 128u, (uint32_t)kTcN);
    extern __shared__ __align__(128) unsigned char tc_smem[];
    unsigned char* A = tc_smem;                                      // [A_BYTES]
    unsigned char* Bbuf = tc_smem + S::A_BYTES;                      // [2][B_BYTES]
    __shared__ __align__(8) uint64_t bar_b[2], bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int tl = threadIdx.x, warp = tl >> 5;
    const int64_t blk = cta_block(a);
    const KernelParams kp = block_params(a, blk, kp_all);
    const int2 rg = a.blk[blk];
    const int t = rg.x + tl;
    const bool valid = t < rg.y;
    const float4 xt = valid ? a.xs[t] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t e0 = a.far_off[blk], e1 = a.far_off[blk + 1];
    const int ne = (int)(e1 - e0);
    if (tl == 0) {
        ptx::mbar_init(&bar_b[0], 1);
        ptx::mbar_init(&bar_b[1], 1);
        ptx::mbar_init(&bar_mma, 1);
        ptx::fence_mbar_init();
        s_fail = 0;
    }
    if (warp == 0) {
        tc::alloc(&tmem_base, 32);
        tc::relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    // thread 0's bookkeeping of what it issued (to drain on failure)
    int nb_issued = 0, nb_done = 0, n_commit = 0;
    auto issue_b = [&](int i) {
        const int slot = i & 1;
        ptx::mbar_arrive_expect_tx(&bar_b[slot], (uint32_t)S::B_BYTES);
        ptx::bulk_g2s(Bbuf + slot * S::B_BYTES, image + (int64_t)a.far_ent[e0 + i].x * S::B_BYTES,
                      (uint32_t)S::B_BYTES, &bar_b[slot]);
        ++nb_issued;
    };
    if (tl == 0 && ne > 0) issue_b(0);
    bool ok = true;
    for (int i = 0; i < ne; ++i) {
        const int2 ent = a.far_ent[e0 + i];
        const bool active = valid && entry_active(ent.y, a.masks, tl);
        float U[S::ROW ? NTP : 1];
        if constexpr (S::ROW) {
            if (active) {  // inactive rows are stored as zeros below, without a basis
                far_basis<D, P>(xt, a.nd_cf[ent.x], a.nd_scale[ent.x], kp, T, [&](int q, float v) { U[q] = v; });
#pragma unroll
                for (int q = NT; q < NTP; ++q) U[q] = 0.f;
            }
        }
        // the MMAs of entry i - 1 are done: the tile and the other multipole slot are free
        if (i > 0) ok = ptx::mbar_wait_bounded(&bar_mma, (uint32_t)((i - 1) & 1), kWaitCycles);
        if (!__syncthreads_and(ok && !s_fail)) { ok = false; break; }
        if (tl == 0 && i + 1 < ne) issue_b(i + 1);
        if constexpr (S::ROW) {
            if (active) {
#pragma unroll
                for (int g = 0; g < NTP / PER16; ++g)
                    tc_store_row16<PREC>(A, APLANE, S::off(tl, g * PER16), U + g * PER16);
            } else {
#pragma unroll
                for (int g = 0; g < NTP / PER16; ++g)
#pragma unroll
                    for (int pl = 0; pl < S::PLANES; ++pl)
                        *reinterpret_cast<uint4*>(A + pl * APLANE + S::off(tl, g * PER16)) = make_uint4(0u, 0u, 0u, 0u);
            }
        } else {
            if (active) {
                far_basis<D, P>(xt, a.nd_cf[ent.x], a.nd_scale[ent.x], kp, T,
                                [&](int q, float v) { tc_store<PREC>(A, APLANE, S::off(tl, q), v); });
#pragma unroll
                for (int q = NT; q < NTP; ++q) tc_store<PREC>(A, APLANE, S::off(tl, q), 0.f);
            } else {
#pragma unroll 4
                for (int q = 0; q < NTP; ++q) tc_store<PREC>(A, APLANE, S::off(tl, q), 0.f);
            }
        }
        ptx::fence_proxy_async_smem();  // generic-proxy stores -> visible to the tensor core
        __syncthreads();
        if (tl == 0) {
            const bool got = ptx::mbar_wait_bounded(&bar_b[i & 1], (uint32_t)((i >> 1) & 1), kWaitCycles);
            if (got) {
                ++nb_done;
                tc::fence_after_sync();
                const unsigned char* B = Bbuf + (i & 1) * S::B_BYTES;
                constexpr int KSTEP_BYTES = 256;  // one MMA consumes 2 core matrices (32 bytes) of K
                constexpr int NSTEP = PREC == TC_TF32 ? NTP / 8 : NTP / 16;
#pragma unroll 1
                for (int ks = 0; ks < NSTEP; ++ks) {
                    const uint64_t da = tc::smem_desc(A + ks * KSTEP_BYTES, 128, S::SBO_A);
                    const uint64_t db = tc::smem_desc(B + ks * KSTEP_BYTES, 128, S::SBO_A);
                    const bool acc = (i > 0) || (ks > 0);
                    if (PREC == TC_TF32) {
                        tc::mma_tf32(tmem, da, db, IDESC, acc);
                    } else {
                        tc::mma_bf16(tmem, da, db, IDESC, acc);
                        if (PREC == TC_BF16X3) {
                            const uint64_t da_lo = tc::smem_desc(A + APLANE + ks * KSTEP_BYTES, 128, S::SBO_A);
                            const uint64_t db_lo = tc::smem_desc(B + BPLANE + ks * KSTEP_BYTES, 128, S::SBO_A);
                            tc::mma_bf16(tmem, da, db_lo, IDESC, true);
                            tc::mma_bf16(tmem, da_lo, db, IDESC, true);
                        }
                    }
                }
            } else {
                s_fail = 1;
            }
            tc::commit(&bar_mma);  // arrives when the MMAs above (if any) are done
            ++n_commit;
        }
    }
    // wait for the last MMA group, then read the accumulator rows
    if (ok && ne > 0) ok = ptx::mbar_wait_bounded(&bar_mma, (uint32_t)((ne - 1) & 1), kWaitCycles);
    const bool all_ok = __syncthreads_and(ok && !s_fail) != 0;
    tc::fence_after_sync();
    float acc[kTcN];
#pragma unroll
    for (int r = 0; r < kTcN; ++r) acc[r] = 0.f;
    if (ne > 0 && all_ok) {
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        tc::ld16(lane_addr, acc);
        tc::ld16(lane_addr + 16, acc + 16);
    }
    if (!all_ok && tl == 0) {
        atomicExch(a.err, 1);
        // let the bulk copies and MMAs still in flight finish before the CTA leaves (bounded)
        for (int j = nb_done; j < nb_issued; ++j)
            ptx::mbar_wait_bounded(&bar_b[j & 1], (uint32_t)((j >> 1) & 1), kWaitCycles);
        if (n_commit > 0) ptx::mbar_wait_bounded(&bar_mma, (uint32_t)((n_commit - 1) & 1), kWaitCycles);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::dealloc(tmem, 32);
    if (valid && all_ok)
        for (int r = 0; r < nr_total; ++r) a.yfar[(int64_t)r * a.N + t] = acc[r];  // tree order, coalesced
}

// ----------------------------------------------------------------------------------------
// d = 3, BF16 / BF16 hi+lo: the basis rows go straight into tensor memory (A operand) instead
// of shared memory, warp-specialised like the near field.
//   warps 0-3 (thread = target = TMEM lane): per far entry i, wait for its info; a warp with a
//     target in the entry's mask generates its rows (radial part first, then the harmonics in
//     increasing term order) and stores them 16 terms at a time as packed BF16 pairs (hi, lo
//     planes) with tcgen05.st -- waiting for the MMAs of entry i-1 only just before its first
//     store; every kFarFlush entries the accumulator rows are added into float32 sums in shared
//     memory and zeroed; every warp has seen the MMAs of entry i-1 complete before it arrives on
//     aready for entry i.
//   warp 4 (lane 0 issues): per entry, the node's centre, scale and the entry's row mask go to a
//     stage with a bulk copy of the node's packed multipoles (ST - 1 entries ahead; the metadata
//     of 32 entries at a time is loaded by the whole warp, one lane per entry); waits aready,
//     issues the MMAs (rows outside the mask disabled) and commits them to mma_done.
// The accumulator is flushed because the tensor core's float32 accumulation drifts over
// thousands of MMAs.  Every wait is bounded.
template <int P, int PREC, int LD = 3>
struct Tc2Shape {
    using S = TcShape<LD, P, PREC>;
    static constexpr int NT = S::NT, NTP = S::NTP;
    static constexpr int PLANE_COLS = NTP / 2;                     // packed BF16 pairs per plane
    static constexpr int COL_AHI = 32, COL_ALO = 32 + PLANE_COLS;
    static constexpr int USED = 32 + S::PLANES * PLANE_COLS;
    static constexpr int TMEM_COLS = USED <= 32 ? 32 : USED <= 64 ? 64 : USED <= 128 ? 128 : USED <= 256 ? 256 : 512;
    static constexpr int ST = 3;                                    // multipole stages in flight
    static constexpr int THREADS = 160;
    static constexpr size_t smem_bytes() { return (size_t)ST * S::B_BYTES + (size_t)kTcN * 128 * 4 + 128; }
    static constexpr bool supported = PREC != TC_TF32 && TMEM_COLS <= 256 && smem_bytes() <= 160 * 1024;
};

struct FarTc2Info {
    float4 c;                  // node centre
    float s;                   // node length scale
    uint32_t on[kMaskWords];   // targets (TMEM lanes) that use the entry
};

}  // namespace fkt

#include "far_tc2.cuh"

namespace fkt {
}  // namespace fkt

#include "far_tc3.cuh"

namespace fkt {

struct TcLaunch {
    const MvmArgs* a;
    const KernelParams* kp;
    const FarTables* T;
    int64_t nblocks, nnodes;
    int64_t group_stride;        // floats between right-hand-side groups of the multipoles
    int nr_total;                // right-hand sides in this pass (<= kTcN)
    unsigned char* image;        // packed B operands, [nodes][B_BYTES]
    cudaStream_t s_pack, s_far;
    int far_kernel;              // d = 3 BF16 forms: 0 = two entries per thread (far_tc3) where
                                 // supported, 1 = one entry per thread (far_tc2)
};

template <int D, int P, int PREC>
int launch_tc_t(const TcLaunch& L) {
    using S = TcShape<D, P, PREC>;
    if constexpr (!S::supported) {
        return FKT_ERR_UNSUPPORTED;
    } else {
        tc_pack_kernel<D, P, PREC><<<(unsigned)L.nnodes, 256, 0, L.s_pack>>>(
            L.nnodes, L.a->s2m_item_off, L.a->mult, L.group_stride, L.nr_total, L.image);
        FKT_CUDA_TRY(cudaGetLastError());
        return FKT_OK;
    }
}

template <int D, int P, int PREC>
int launch_tc_far_t(const TcLaunch& L) {
    using S = TcShape<D, P, PREC>;
    if constexpr (D == 3 && Tc3Shape<P, PREC>::supported) {
        if (L.far_kernel == 0) {
            using Sh = Tc3Shape<P, PREC>;
            const size_t smem = Sh::smem_bytes();
            static bool attr3 = false;
            if (!attr3) {
                FKT_CUDA_TRY(cudaFuncSetAttribute(far_tc3_kernel<P, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)smem));
                attr3 = true;
            }
            FarTables2 T2;
            make_far_tables2(*L.T, &T2);
            far_tc3_kernel<P, PREC><<<(unsigned)L.nblocks, Sh::THREADS, smem, L.s_far>>>(*L.a, *L.kp, T2, L.image,
                                                                                        L.nr_total);
            FKT_CUDA_TRY(cudaGetLastError());
            return FKT_OK;
        }
    }
    if constexpr (dim_of(D) == 3 && Tc2Shape<P, PREC, D>::supported) {
        using Sh = Tc2Shape<P, PREC, D>;
        const size_t smem = Sh::smem_bytes();
        if (L.far_kernel == 2) {  // rows held in registers until the previous entry's MMAs complete
            static bool attr_h = false;
            if (!attr_h) {
                FKT_CUDA_TRY(cudaFuncSetAttribute(far_tc2_kernel<P, PREC, D, 4>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                attr_h = true;
            }
            far_tc2_kernel<P, PREC, D, 4><<<(unsigned)L.nblocks, Sh::THREADS, smem, L.s_far>>>(*L.a, *L.kp, *L.T, L.image,
                                                                                              L.nr_total);
            FKT_CUDA_TRY(cudaGetLastError());
            return FKT_OK;
        }
        static bool attr = false;
        if (!attr) {
            FKT_CUDA_TRY(cudaFuncSetAttribute(far_tc2_kernel<P, PREC, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
            attr = true;
        }
        far_tc2_kernel<P, PREC, D><<<(unsigned)L.nblocks, Sh::THREADS, smem, L.s_far>>>(*L.a, *L.kp, *L.T, L.image, L.nr_total);
        FKT_CUDA_TRY(cudaGetLastError());
        return FKT_OK;
    } else if constexpr (!S::supported) {
        return FKT_ERR_UNSUPPORTED;
    } else {
        const size_t smem = S::smem_bytes();
        static bool attr = false;
        if (!attr) {
            FKT_CUDA_TRY(cudaFuncSetAttribute(far_tc_kernel<D, P, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
            attr = true;
        }
        far_tc_kernel<D, P, PREC><<<(unsigned)L.nblocks, kTB, smem, L.s_far>>>(*L.a, *L.kp, *L.T, L.image, L.nr_total);
        FKT_CUDA_TRY(cudaGetLastError());
        return FKT_OK;
    }
}

template <int D, int PLO, int PHI>
int launch_tc_range(int p, int prec, bool far, const TcLaunch& L) {
    if (p == PHI) {
        if (prec == TC_BF16) return far ? launch_tc_far_t<D, PHI, TC_BF16>(L) : launch_tc_t<D, PHI, TC_BF16>(L);
        if (prec == TC_BF16X3) return far ? launch_tc_far_t<D, PHI, TC_BF16X3>(L) : launch_tc_t<D, PHI, TC_BF16X3>(L);
        return far ? launch_tc_far_t<D, PHI, TC_TF32>(L) : launch_tc_t<D, PHI, TC_TF32>(L);
    }
    if constexpr (PHI > PLO) return launch_tc_range<D, PLO, PHI - 1>(p, prec, far, L);
    return FKT_ERR_INVALID_ARG;
}

// Bytes of the packed B-operand image per node.
inline int tc_b_bytes(int nt, int prec) {
    const int ntp = (nt + 15) / 16 * 16;
    const int el = prec == TC_TF32 ? 4 : 2;
    return kTcN * ntp * el * (prec == TC_BF16X3 ? 2 : 1);
}

}  // namespace fkt
