// __global__ kernels of the FKT matrix-vector product (Algorithm 1).
//   permute_kernel   w (caller order) -> sorted weights of one group of NR right-hand sides
//   s2m_kernel       per (node, <=1024-point chunk): partial multipoles (source2mult)
//   s2m_reduce       per node: sum of its chunks' partials (deterministic order)
//   near_kernel      per target block: dense K(near, leaf) * w[leaf] over the near leaves
//   far_kernel       per target block: m2t * multipole over the far nodes, plus the near
//                    result, scattered back to the caller's order
//   dense_kernel     exact all-pairs product (eq. nbody), for checks and baselines
#pragma once

#include "fkt_kernels.cuh"

namespace fkt {

constexpr int kNearChunk = 256;   // sources staged per shared-memory pass

template <int NR>
__global__ void permute_kernel(int64_t N, const int32_t* __restrict__ perm, const float* __restrict__ w, int nr,
                               float* __restrict__ ws) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int64_t j = perm[i];
#pragma unroll
    for (int r = 0; r < NR; ++r) ws[r * N + i] = r < nr ? __ldg(&w[r * N + j]) : 0.0f;
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
    float acc[TPL][NR];
#pragma unroll
    for (int i = 0; i < TPL; ++i)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[i][r] = 0.f;
    for (int base = it.y + warp * 32; base < it.z; base += WARPS * 32) {
        const int s = base + lane;
        const bool ok = s < it.z;
        float4 x = ok ? a.xs[s] : c;
        float x0 = (x.x - c.x) * inv_s, x1 = (x.y - c.y) * inv_s, x2 = (x.z - c.z) * inv_s;
        float x3 = D == 4 ? (x.w - c.w) * inv_s : 0.f;
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
        for (int r = 0; r < NR; ++r) wt[lane * NR + r] = ok ? a.ws[(int64_t)r * a.N + s] : 0.f;
        __syncwarp();
#pragma unroll 4
        for (int row = 0; row < 32; ++row) {
            float wr[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) wr[r] = wt[row * NR + r];
#pragma unroll
            for (int i = 0; i < TPL; ++i) {
                const int t = lane + 32 * i;
                if (t < NT) {
                    float b = tile[row * ROW + t];
#pragma unroll
                    for (int r = 0; r < NR; ++r) acc[i][r] = fmaf(b, wr[r], acc[i][r]);
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
            for (int r = 0; r < NR; ++r) red[(warp * NT + t) * NR + r] = acc[i][r];
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
template <int D, int KIND, int NR>
__global__ void __launch_bounds__(kTB) near_kernel(MvmArgs a, KernelParams kp) {
    __shared__ float4 sx[kNearChunk];
    __shared__ float sw[NR][kNearChunk];
    const int64_t blk = blockIdx.x;
    const int2 rg = a.blk[blk];
    const int tl = threadIdx.x;
    const int t = rg.x + tl;
    const bool valid = t < rg.y;
    const float4 xt = valid ? a.xs[t] : make_float4(0.f, 0.f, 0.f, 0.f);
    float acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.f;
    const int64_t e0 = a.near_off[blk], e1 = a.near_off[blk + 1];
    for (int64_t e = e0; e < e1; ++e) {
        const int2 ent = a.near_ent[e];
        const bool active = valid && entry_active(ent.y, a.masks, tl);
        const int s0 = a.nd_begin[ent.x], s1 = a.nd_end[ent.x];
        for (int cb = s0; cb < s1; cb += kNearChunk) {
            const int n = min(kNearChunk, s1 - cb);
            __syncthreads();
            for (int i = tl; i < n; i += kTB) {
                sx[i] = a.xs[cb + i];
#pragma unroll
                for (int r = 0; r < NR; ++r) sw[r][i] = a.ws[(int64_t)r * a.N + cb + i];
            }
            __syncthreads();
            if (active) {
#pragma unroll 4
                for (int i = 0; i < n; ++i) {
                    const float4 xs = sx[i];
                    float dx = xt.x - xs.x, dy = xt.y - xs.y, dz = xt.z - xs.z;
                    float r2 = dx * dx + dy * dy + dz * dz;
                    if (D == 4) { float dw = xt.w - xs.w; r2 += dw * dw; }
                    const float kv = kernel_r2<KIND>(r2, kp);
#pragma unroll
                    for (int r = 0; r < NR; ++r) acc[r] = fmaf(kv, sw[r][i], acc[r]);
                }
            }
        }
    }
    if (valid)
#pragma unroll
        for (int r = 0; r < NR; ++r) a.ynear[(int64_t)r * a.N + t] = acc[r];
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
__global__ void __launch_bounds__(kTB) far_kernel(MvmArgs a, KernelParams kp, const __grid_constant__ FarTables T) {
    using Lay = Layout<D, P>;
    using Sh = FarShape<D, P, NR>;
    constexpr int NT = Sh::NT, FB = Sh::FB;
    extern __shared__ float sM[];
    __shared__ float4 s_c[FB];
    __shared__ float s_s[FB];
    __shared__ int s_m[FB];
    const int64_t blk = blockIdx.x;
    const int2 rg = a.blk[blk];
    const int tl = threadIdx.x;
    const int t = rg.x + tl;
    const bool valid = t < rg.y;
    const float4 xt = valid ? a.xs[t] : make_float4(0.f, 0.f, 0.f, 0.f);
    float acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.f;
    const int64_t e0 = a.far_off[blk], e1 = a.far_off[blk + 1];
    for (int64_t eb = e0; eb < e1; eb += FB) {
        const int nb = (int)min((int64_t)FB, e1 - eb);
        __syncthreads();
        for (int i = tl; i < nb * NT * NR; i += kTB) {
            const int e = i / (NT * NR), q = i - e * NT * NR;
            const int node = a.far_ent[eb + e].x;
            sM[i] = a.mult[(int64_t)node * NT * NR + q];
        }
        if (tl < nb) {
            const int2 ent = a.far_ent[eb + tl];
            s_c[tl] = a.nd_cf[ent.x];
            s_s[tl] = a.nd_scale[ent.x];
            s_m[tl] = ent.y;
        }
        __syncthreads();
        for (int e = 0; e < nb; ++e) {
            if (!(valid && entry_active(s_m[e], a.masks, tl))) continue;
            const float4 c = s_c[e];
            const float dx = xt.x - c.x, dy = xt.y - c.y, dz = xt.z - c.z, dw = D == 4 ? xt.w - c.w : 0.f;
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
                    const int j = k + 2 * jj, q = Lay::pair(k) + jj;
                    float R = 0.f;
#pragma unroll
                    for (int m = 0; m <= j; ++m) R = fmaf(T.That[q][m], J[m], R);
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
        const int64_t o = a.perm[t];
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (r < a.nr) a.y[(int64_t)r * a.N + o] = a.ynear[(int64_t)r * a.N + t] + acc[r];
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
__global__ void __launch_bounds__(kTB) far_mr_kernel(MvmArgs a, KernelParams kp, const __grid_constant__ FarTables T) {
    using Lay = Layout<D, P>;
    constexpr int NT = Lay::nterms, ROW = FarMrShape<D, P>::ROW;
    extern __shared__ float sm[];
    float* U = sm;
    float4* Ms = reinterpret_cast<float4*>(sm + kTB * ROW);  // kTB * ROW is a multiple of 128 floats
    __shared__ float4 s_c;
    __shared__ float s_s;
    __shared__ int s_m;
    const int64_t blk = blockIdx.x;
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
        const float dx = xt.x - c.x, dy = xt.y - c.y, dz = xt.z - c.z, dw = D == 4 ? xt.w - c.w : 0.f;
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
                const int j = k + 2 * jj, q = Lay::pair(k) + jj;
                float R = 0.f;
#pragma unroll
                for (int m = 0; m <= j; ++m) R = fmaf(T.That[q][m], J[m], R);
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
        const int64_t o = a.perm[t];
#pragma unroll
        for (int r = 0; r < 8; ++r)
            if (r < a.nr) a.y[(int64_t)r * a.N + o] = a.ynear[(int64_t)r * a.N + t] + acc[r];
    }
}

// ---------------------------------------------------------------- dense
template <int D, int KIND, int NR>
__global__ void __launch_bounds__(kTB) dense_kernel(MvmArgs a, KernelParams kp) {
    __shared__ float4 sx[kNearChunk];
    __shared__ float sw[NR][kNearChunk];
    const int t = blockIdx.x * kTB + threadIdx.x;
    const bool valid = t < a.N;
    const float4 xt = valid ? a.xs[t] : make_float4(0.f, 0.f, 0.f, 0.f);
    float acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.f;
    for (int64_t cb = 0; cb < a.N; cb += kNearChunk) {
        const int n = (int)min((int64_t)kNearChunk, a.N - cb);
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += kTB) {
            sx[i] = a.xs[cb + i];
#pragma unroll
            for (int r = 0; r < NR; ++r) sw[r][i] = a.ws[(int64_t)r * a.N + cb + i];
        }
        __syncthreads();
        for (int i = 0; i < n; ++i) {
            const float4 xs = sx[i];
            float dx = xt.x - xs.x, dy = xt.y - xs.y, dz = xt.z - xs.z;
            float r2 = dx * dx + dy * dy + dz * dz;
            if (D == 4) { float dw = xt.w - xs.w; r2 += dw * dw; }
            const float kv = kernel_r2<KIND>(r2, kp);
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] = fmaf(kv, sw[r][i], acc[r]);
        }
    }
    if (valid) {
        const int64_t o = a.perm[t];
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (r < a.nr) a.y[(int64_t)r * a.N + o] = acc[r];
    }
}

}  // namespace fkt
