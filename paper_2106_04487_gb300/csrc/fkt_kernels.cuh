// Device code of the FKT matrix-vector product (Algorithm 1), templated on the
// dimension D (3 or 4), the truncation order P and the number of right-hand sides
// NR handled per pass.
//
// Expansion used (Theorem 3.1, eq. finaltrunc, with the node length scale s):
//   K(|x - x'|) ~ sum_{k<=P} sum_h Yt_kh(x/|x|) (s/r)^j R_kj(r) * (r'/s)^(j-k) St_kh(x'/s)
//   over j = k, k+2, ..., <= P, where
//     x = target - c, r = |x|; x' = source - c, r' = |x'|
//     St_kh(y) = |y|^k Yt_kh(y/|y|)  (normalised solid harmonic, sum_h Yt_kh(u) Yt_kh(v) = C_k(u.v))
//     R_kj(r)  = sum_{m<=j} That_{kjm} J_m(r),  J_m = K^(m)(r) r^m / m!   (That = m! Tbar)
// so the source side is a polynomial in x'/s (no square roots) and every factor is
// bounded: r' <= rho <= s, and far pairs have s/r < theta when s = rho.
#pragma once

#include "fkt_internal.h"

namespace fkt {

// ----------------------------------------------------------------- layout
// Layout code D of the expansion: 2, 3 or 4 = every radial term j = k, k+2, ..., <= P of each
// degree k in that dimension; kDiag3 = d = 3 with the j = k term only.  The latter is the radial
// compression of the Laplace kernel 1/r in d = 3: its degree-k radial part has rank 1 (Table 3),
// being r'^k / r^(k+1) alone (the Legendre multipole expansion of Sec. 3.3, eq. electro), so the
// terms j > k vanish identically and are dropped from s2m, the multipoles and m2t.
constexpr int kDiag3 = 103;
__host__ __device__ constexpr int dim_of(int D) { return D % 100; }
__host__ __device__ constexpr bool diag_of(int D) { return D >= 100; }

template <int D, int P>
struct Layout {
    static constexpr int nj(int k) { return diag_of(D) ? 1 : (P - k) / 2 + 1; }
    static constexpr int dk(int k) {
        return dim_of(D) == 2 ? (k == 0 ? 1 : 2) : dim_of(D) == 3 ? 2 * k + 1 : (k + 1) * (k + 1);
    }
    // row of the expansion tables (built for the full layout) of radial pair (k, j = k + 2 jj)
    static constexpr int tpair(int k, int jj) {
        int o = 0;
        for (int i = 0; i < k; ++i) o += (P - i) / 2 + 1;
        return o + jj;
    }
    static constexpr int off(int k) {
        int o = 0;
        for (int i = 0; i < k; ++i) o += dk(i) * nj(i);
        return o;
    }
    static constexpr int pair(int k) {  // index of the first (k, j) radial pair of degree k
        int o = 0;
        for (int i = 0; i < k; ++i) o += nj(i);
        return o;
    }
    static constexpr int nterms = off(P + 1);
    static constexpr int npairs = pair(P + 1);
};

// -------------------------------------------------------- kernel values
template <int KIND>
__device__ __forceinline__ float kernel_r2(float r2, const KernelParams& kp) {
    if (KIND == FKT_GAUSSIAN) {
        return kp.scale * __expf(-r2 * kp.c1);
    } else if (KIND == FKT_EXPONENTIAL) {
        float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
        return kp.scale * __expf(-r * kp.c1);
    } else if (KIND == FKT_MATERN32) {
        float t = r2 * rsqrtf(fmaxf(r2, 1e-30f)) * kp.c1;
        return kp.scale * (1.0f + t) * __expf(-t);
    } else if (KIND == FKT_MATERN52) {
        float t = r2 * rsqrtf(fmaxf(r2, 1e-30f)) * kp.c1;
        return kp.scale * (1.0f + t + t * t * (1.0f / 3.0f)) * __expf(-t);
    } else if (KIND == FKT_CAUCHY) {
        return __fdividef(kp.scale, 1.0f + r2 * kp.c1);
    } else if (KIND == FKT_RATQUAD) {
        float b = 1.0f + r2 * kp.c1;
        return kp.alpha == 1.0f ? __fdividef(kp.scale, b) : kp.scale * exp2f(-kp.alpha * __log2f(b));
    } else {  // FKT_LAPLACE: r = 0 pairs contribute nothing
        return r2 > 0.0f ? kp.scale * rsqrtf(r2) : 0.0f;
    }
}

// Scaled Taylor coefficients J_m = K^(m)(r) r^m / m! of t -> K(r (1 + t)), m = 0..P,
// from closed-form recurrences per kernel (float32).
template <int P>
__device__ __forceinline__ void kernel_jets(const KernelParams& kp, float r, float rinv, float J[P + 1]) {
    switch (kp.kind) {
    case FKT_GAUSSIAN: {  // exp(-a (1+t)^2): e_m = -(2a/m)(e_{m-1} + e_{m-2})
        float a = r * r * kp.c1;
        float E = kp.scale * __expf(-a);
        float em2 = 0.f, em1 = 1.f;
        J[0] = E;
#pragma unroll
        for (int m = 1; m <= P; ++m) {
            float em = -(2.0f * a / m) * (em1 + em2);
            J[m] = E * em;
            em2 = em1;
            em1 = em;
        }
        break;
    }
    case FKT_EXPONENTIAL: {  // exp(-b (1+t)): (-b)^m / m!
        float b = r * kp.c1;
        float v = kp.scale * __expf(-b);
        J[0] = v;
#pragma unroll
        for (int m = 1; m <= P; ++m) { v *= -b / m; J[m] = v; }
        break;
    }
    case FKT_MATERN32: {  // (1 + b + b t) exp(-b) exp(-b t)
        float b = r * kp.c1;
        float E[P + 1];
        E[0] = kp.scale * __expf(-b);
#pragma unroll
        for (int m = 1; m <= P; ++m) E[m] = E[m - 1] * (-b / m);
        J[0] = (1.0f + b) * E[0];
#pragma unroll
        for (int m = 1; m <= P; ++m) J[m] = (1.0f + b) * E[m] + b * E[m - 1];
        break;
    }
    case FKT_MATERN52: {  // (1 + b(1+t) + b^2 (1+t)^2 / 3) exp(-b (1+t))
        float b = r * kp.c1;
        float p0 = 1.0f + b + b * b * (1.0f / 3.0f), p1 = b + b * b * (2.0f / 3.0f), p2 = b * b * (1.0f / 3.0f);
        float E[P + 1];
        E[0] = kp.scale * __expf(-b);
#pragma unroll
        for (int m = 1; m <= P; ++m) E[m] = E[m - 1] * (-b / m);
#pragma unroll
        for (int m = 0; m <= P; ++m) J[m] = p0 * E[m] + (m >= 1 ? p1 * E[m - 1] : 0.f) + (m >= 2 ? p2 * E[m - 2] : 0.f);
        break;
    }
    case FKT_CAUCHY: {  // 1 / ((1+c) + 2c t + c t^2)
        float c = r * r * kp.c1;
        float inv = __fdividef(1.0f, 1.0f + c);
        float qm2 = 0.f, qm1 = kp.scale * inv;
        J[0] = qm1;
#pragma unroll
        for (int m = 1; m <= P; ++m) {
            float q = -(2.0f * c * qm1 + c * qm2) * inv;
            J[m] = q;
            qm2 = qm1;
            qm1 = q;
        }
        break;
    }
    case FKT_RATQUAD: {  // ((1+c) + 2c t + c t^2)^(-alpha):  m d0 f_m = sum_i (beta i - (m - i)) d_i f_{m-i}
        float c = r * r * kp.c1;
        float d0 = 1.0f + c, d1 = 2.0f * c, d2 = c, beta = -kp.alpha;
        float inv = __fdividef(1.0f, d0);
        float fm2 = 0.f, fm1 = kp.scale * exp2f(beta * __log2f(d0));
        J[0] = fm1;
#pragma unroll
        for (int m = 1; m <= P; ++m) {
            float f = ((beta - (m - 1)) * d1 * fm1 + (2.0f * beta - (m - 2)) * d2 * fm2) * inv / m;
            J[m] = f;
            fm2 = fm1;
            fm1 = f;
        }
        break;
    }
    default: {  // FKT_LAPLACE: s / (r (1+t))
        float v = kp.scale * rinv;
#pragma unroll
        for (int m = 0; m <= P; ++m) { J[m] = v; v = -v; }
        break;
    }
    }
}

// ---------------------------------------------------- solid harmonics
// Calls f(k, h, value) for every normalised solid harmonic St_kh(x) of degree k <= P,
// in an l-major order.  r2_3 = x0^2 + x1^2 + x2^2, r2 = |x|^2 (r2 = r2_3 when D = 3).
// D = 2: the circular harmonics Re, Im of (x0 + i x1)^k (1 at k = 0), whose products add up to
// T_k of the angle between two unit vectors (the 2-D addition theorem).
// The recurrences are those of Legendre-type polynomials in homogeneous form (no
// square roots), so the same routine serves s2m (arbitrary x') and m2t (unit x).
template <int D, int P, class F>
__device__ __forceinline__ void solid_harmonics(float x0, float x1, float x2, float x3, float r2_3, float r2,
                                                const FarTables& T, F&& f) {
    float C[P + 1], S[P + 1];
    C[0] = 1.f;
    S[0] = 0.f;
#pragma unroll
    for (int m = 1; m <= P; ++m) {
        C[m] = x0 * C[m - 1] - x1 * S[m - 1];
        S[m] = x0 * S[m - 1] + x1 * C[m - 1];
    }
    if constexpr (dim_of(D) == 2) {
        f(0, 0, 1.f);
#pragma unroll
        for (int k = 1; k <= P; ++k) {
            f(k, 0, C[k]);
            f(k, 1, S[k]);
        }
        return;
    }
    float pm2[P + 1], pm1[P + 1], cur[P + 1];
#pragma unroll
    for (int m = 0; m <= P; ++m) { pm2[m] = 0.f; pm1[m] = 0.f; cur[m] = 0.f; }
#pragma unroll
    for (int l = 0; l <= P; ++l) {
#pragma unroll
        for (int m = 0; m <= l; ++m) {
            if (m == l) cur[m] = T.hSeed[m];
            else if (m == l - 1) cur[m] = T.hA[l][m] * x2 * pm1[m];
            else cur[m] = T.hA[l][m] * x2 * pm1[m] - T.hB[l][m] * r2_3 * pm2[m];
        }
        if (dim_of(D) == 3) {
            f(l, 0, cur[0]);
#pragma unroll
            for (int m = 1; m <= l; ++m) {
                f(l, 2 * m - 1, cur[m] * C[m]);
                f(l, 2 * m, cur[m] * S[m]);
            }
        } else {
            // Gegenbauer chain factor Q_n^(l+1)(x3, r2), normalised, for k = l + n
            float Q[P + 1];
            Q[0] = T.gSeed[l];
#pragma unroll
            for (int n = 1; n + l <= P; ++n)
                Q[n] = T.gA[l][n] * x3 * Q[n - 1] - (n >= 2 ? T.gB[l][n] * r2 * Q[n - 2] : 0.f);
#pragma unroll
            for (int n = 0; n + l <= P; ++n) {
                const int k = l + n, hb = l * l;
                f(k, hb, Q[n] * cur[0]);
#pragma unroll
                for (int m = 1; m <= l; ++m) {
                    f(k, hb + 2 * m - 1, Q[n] * cur[m] * C[m]);
                    f(k, hb + 2 * m, Q[n] * cur[m] * S[m]);
                }
            }
        }
#pragma unroll
        for (int m = 0; m <= P; ++m) { pm2[m] = pm1[m]; pm1[m] = cur[m]; }
    }
}

// --------------------------------------------------------------- arguments
struct MvmArgs {
    int64_t N;
    const float4* xs;          // sorted points
    const int32_t* perm;       // sorted -> original
    const int2* blk;           // target blocks
    const int64_t* far_off;
    const int2* far_ent;
    const int64_t* near_off;
    const int2* near_ent;
    const uint32_t* masks;
    const int32_t* nd_begin;
    const int32_t* nd_end;
    const float4* nd_cf;
    const float* nd_scale;
    const int4* s2m_items;
    const int64_t* s2m_item_off;
    const int32_t* nd_img;     // image position of each leaf's first source (near-field image)
    int64_t nnodes;
    // per pass (one group of NR right-hand sides)
    const float4* rec;         // source records in tree order: rec_f4 float4 per point (point, then weights)
    int rec_f4;                // float4s per source record
    int woff;                  // float index, within a record, of this group's first weight (s2m)
    float* ynear;              // sorted near-field result of this group, [NR][N]
    float* mult;               // multipoles of this group, [nodes][nterms][NR]
    float* part;               // s2m partials, [items][nterms][NR]
    float* y;                  // output (original order), [nrhs][N]; this group starts at y
    float* yfar;               // far-field result of this group (tree order), [NR][N]
    const float* nimg;         // near-field image of this pass (32-wide tensor-core passes)
    int nr;                    // right-hand sides actually present in this group (<= NR)
    int near_split;            // single-RHS near field: CTAs per target block, each taking every
                               // near_split-th entry and writing its own partial row of ynear
    int far_split;             // the same for the single-RHS float32 far field (partial rows of yfar)
    int* err;                  // device error word: 1 = a bounded wait ran out
    // batches of independent problems (all null for a single problem)
    const KernelParams* kps;   // kernel parameters per problem
    const int32_t* blk_prob;   // problem of each target block
    const int32_t* blk_list;   // grid index -> target block (work ordered largest first)
    const float* pt_sig;       // near-field coordinate scale of each point's problem
    // limit, in SM clocks, of the pipeline waits of the tensor-core kernels (record / multipole
    // copies landing, the consumers' hand-off to the MMA issuer); the waits that drain work in
    // flight before a CTA exits always use kWaitCycles
    long long wait_cycles;
};

// Target block handled by this CTA and its kernel parameters (per problem in a batch).
__device__ __forceinline__ int64_t cta_block(const MvmArgs& a) {
    return a.blk_list ? (int64_t)a.blk_list[blockIdx.x] : (int64_t)blockIdx.x;
}
__device__ __forceinline__ KernelParams block_params(const MvmArgs& a, int64_t blk, const KernelParams& kp) {
    return a.kps ? a.kps[a.blk_prob[blk]] : kp;
}

// Source record of one point for a pass of NR right-hand sides: (x, y, z, w) when d = 3 and
// NR = 1, otherwise (x, y, z, u) followed by the NR weights, padded to whole float4s.
template <int D, int NR>
struct Rec {
    static constexpr int F4 = (D == 3 && NR == 1) ? 1 : (4 + NR + 3) / 4;  // float4s per point
    static constexpr int WOFF = (D == 3 && NR == 1) ? 3 : 4;                // float index of weight 0
};

// (d = 2 uses the d = 3 records: its third coordinate is zero)
inline int rec_f4(int d, int nrb) { return (d <= 3 && nrb == 1) ? 1 : (4 + nrb + 3) / 4; }
inline int rec_woff(int d, int nrb) { return (d <= 3 && nrb == 1) ? 3 : 4; }

__device__ __forceinline__ bool entry_active(int mask, const uint32_t* __restrict__ masks, int t) {
    return mask < 0 || ((__ldg(&masks[(int64_t)mask * kMaskWords + (t >> 5)]) >> (t & 31)) & 1u);
}

}  // namespace fkt
