// Learned low-rank correction of the block-Jacobi preconditioner (include/fkt.h describes the
// teacher, the network and the loss).  Kernels:
//   teacher_kernel   T_b = A_by A_yy^{-1} A_yb, the coupling of block b to its neighbours y folded
//                    into the block (Cholesky of A_yy and triangular solves in shared memory), one
//                    CTA per training block
//   learn_kernel     forward pass, loss and full backward pass for one training block; gradients
//                    summed per CTA and added to the global gradient
//   adam_kernel      Adam step (Kingma & Ba 2015, bias-corrected moments)
//   vectors_kernel   V_b for every block; the corrected blocks A_bb + beta^2 V_b V_b^T are then
//                    factored and inverted by the block-Jacobi set-up kernel (solve.cu)
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <random>
#include <vector>

#include "mvm_kernels.cuh"

namespace fkt {
namespace {

constexpr int kNbrHalf = 32;               // neighbours taken from each adjacent block
constexpr int kMaxPts = kTB + 2 * kNbrHalf;  // block + neighbours
constexpr int kLdS = kTB + 1;
constexpr int kLdY = 2 * kNbrHalf + 1;
constexpr int kMaxH = 64, kMaxR = 16;

struct NetShape {
    int d, H, R;
    __host__ __device__ int oW1() const { return 0; }
    __host__ __device__ int ob1() const { return d * H; }
    __host__ __device__ int oW2() const { return d * H + H; }
    __host__ __device__ int ob2() const { return d * H + H + H * H; }
    __host__ __device__ int oWo() const { return d * H + 2 * H + H * H; }
    __host__ __device__ int obo() const { return oWo() + 3 * H * R; }
    __host__ __device__ int obeta() const { return obo() + R; }
    __host__ __device__ int n() const { return obeta() + 1; }
};

__device__ float kernel_value_any(int kind, float q, const KernelParams& kp) {
    switch (kind) {
    case FKT_GAUSSIAN: return kp.scale * kval<FKT_GAUSSIAN>(q, kp);
    case FKT_EXPONENTIAL: return kp.scale * kval<FKT_EXPONENTIAL>(q, kp);
    case FKT_MATERN32: return kp.scale * kval<FKT_MATERN32>(q, kp);
    case FKT_MATERN52: return kp.scale * kval<FKT_MATERN52>(q, kp);
    case FKT_CAUCHY: return kp.scale * kval<FKT_CAUCHY>(q, kp);
    case FKT_RATQUAD: return kp.scale * kval<FKT_RATQUAD>(q, kp);
    default: return kp.scale * kval<FKT_LAPLACE>(q, kp);
    }
}

// Points of block b followed by its neighbours (tree order); returns n (block) and m (neighbours).
__device__ void gather_points(const int2* __restrict__ blk, int64_t nblocks, int64_t b, const float4* __restrict__ xs,
                              float4* pts, int* n_out, int* m_out) {
    const int2 rg = blk[b];
    const int n = rg.y - rg.x;
    int lo_prev = 0, n_prev = 0, n_next = 0, lo_next = 0;
    if (b > 0) {
        const int2 r = blk[b - 1];
        n_prev = min(kNbrHalf, r.y - r.x);
        lo_prev = r.y - n_prev;
    }
    if (b + 1 < nblocks) {
        const int2 r = blk[b + 1];
        n_next = min(kNbrHalf, r.y - r.x);
        lo_next = r.x;
    }
    for (int i = threadIdx.x; i < n + n_prev + n_next; i += blockDim.x) {
        int src;
        if (i < n) src = rg.x + i;
        else if (i < n + n_prev) src = lo_prev + (i - n);
        else src = lo_next + (i - n - n_prev);
        pts[i] = xs[src];
    }
    *n_out = n;
    *m_out = n_prev + n_next;
}

// In-place lower Cholesky of the n x n matrix A (leading dimension ld); sets *bad on a
// non-positive pivot.  Called by the whole CTA.
__device__ void chol_inplace(float* A, int ld, int n, int* bad) {
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            float dkk = A[k * ld + k];
            if (!(dkk > 0.f)) { *bad = 1; dkk = 1e-30f; }
            A[k * ld + k] = sqrtf(dkk);
        }
        __syncthreads();
        const float dk = A[k * ld + k];
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[i * ld + k] /= dk;
        __syncthreads();
        const int m = n - k - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int i = k + 1 + e / m, j = k + 1 + e % m;
            if (j <= i) A[i * ld + j] -= A[i * ld + k] * A[j * ld + k];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
teacher_kernel(const int2* __restrict__ blk, int64_t nblocks, const int64_t* __restrict__ train, const float4* __restrict__ xs,
               KernelParams kp, float sigma2, float* __restrict__ D, int* err) {
    extern __shared__ float sm[];
    float* Ayb = sm;                      // [2*kNbrHalf][kLdS]
    float* Ayy = Ayb + 2 * kNbrHalf * kLdS;  // [2*kNbrHalf][kLdY]
    __shared__ float4 pts[kMaxPts];
    __shared__ int bad;
    __shared__ int s_n, s_m;
    const int64_t b = train[blockIdx.x];
    if (threadIdx.x == 0) bad = 0;
    {
        int n, m;
        gather_points(blk, nblocks, b, xs, pts, &n, &m);
        if (threadIdx.x == 0) { s_n = n; s_m = m; }
    }
    __syncthreads();
    const int n = s_n, m = s_m;
    auto kv = [&](int i, int j) {
        const float4 a = pts[i], c = pts[j];
        const float dx = (a.x - c.x) * kp.sig, dy = (a.y - c.y) * kp.sig, dz = (a.z - c.z) * kp.sig,
                    dw = (a.w - c.w) * kp.sig;
        float v = kernel_value_any(kp.kind, dx * dx + dy * dy + dz * dz + dw * dw, kp);
        if (i == j) v = (kp.kind == FKT_LAPLACE ? 0.f : v) + sigma2;
        return v;
    };
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        Ayb[i * kLdS + j] = kv(n + i, j);
    }
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        Ayy[i * kLdY + j] = kv(n + i, n + j);
    }
    __syncthreads();
    if (m > 0) {
        chol_inplace(Ayy, kLdY, m, &bad);
        // C = L_y^{-1} A_yb, column by column (forward substitution), in place
        for (int j = threadIdx.x; j < n; j += blockDim.x)
            for (int i = 0; i < m; ++i) {
                float s = Ayb[i * kLdS + j];
                for (int k = 0; k < i; ++k) s -= Ayy[i * kLdY + k] * Ayb[k * kLdS + j];
                Ayb[i * kLdS + j] = s / Ayy[i * kLdY + i];
            }
        __syncthreads();
    }
    // T = C^T C = A_by A_yy^{-1} A_yb  (zero without neighbours)
    float* out = D + (int64_t)blockIdx.x * kTB * kTB;
    for (int e = threadIdx.x; e < kTB * kTB; e += blockDim.x) {
        const int i = e / kTB, j = e % kTB;
        float v = 0.f;
        if (i < n && j < n)
            for (int k = 0; k < m; ++k) v += Ayb[k * kLdS + i] * Ayb[k * kLdS + j];
        out[e] = v;
    }
    if (threadIdx.x == 0 && bad) atomicExch(err, 2);
}

// sum |D_b|_F^2 and sum trace(D_b) / n_b over the training blocks
__global__ void teacher_stats_kernel(const float* __restrict__ D, const int2* __restrict__ blk,
                                     const int64_t* __restrict__ train, double* out) {
    const float* Db = D + (int64_t)blockIdx.x * kTB * kTB;
    const int2 rg = blk[train[blockIdx.x]];
    const int n = rg.y - rg.x;
    double f = 0.0, t = 0.0;
    for (int e = threadIdx.x; e < kTB * kTB; e += blockDim.x) {
        const double v = Db[e];
        f += v * v;
        if (e / kTB == e % kTB) t += v / n;
    }
    for (int off = 16; off; off >>= 1) {
        f += __shfl_xor_sync(0xffffffffu, f, off);
        t += __shfl_xor_sync(0xffffffffu, t, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], f);
        atomicAdd(&out[1], t);
    }
}

struct LearnSmem {
    float* U;    // [kMaxPts][4]
    float* Z1;   // [kMaxPts][H]
    float* PHI;  // [kMaxPts][H]
    float* dPHI; // [kMaxPts][H]
    float* dZ1;  // [kMaxPts][H]
    float* V;    // [kTB][R]
    float* dV;   // [kTB][R]
    float* gh;   // [2H] pooled features g, h
    float* sdV;  // [R]
};

__host__ __device__ inline size_t learn_smem_floats(int H, int R) {
    return (size_t)kMaxPts * 4 + 4 * (size_t)kMaxPts * H + 2 * (size_t)kTB * R + 2 * (size_t)H + R + 8;
}

__device__ LearnSmem carve(float* sm, int H, int R) {
    LearnSmem s;
    s.U = sm;
    s.Z1 = s.U + kMaxPts * 4;
    s.PHI = s.Z1 + kMaxPts * H;
    s.dPHI = s.PHI + kMaxPts * H;
    s.dZ1 = s.dPHI + kMaxPts * H;
    s.V = s.dZ1 + kMaxPts * H;
    s.dV = s.V + kTB * R;
    s.gh = s.dV + kTB * R;
    s.sdV = s.gh + 2 * H;
    return s;
}

// Forward pass up to V for the CTA's block; leaves U, Z1, PHI, gh, V in shared memory.
__device__ void net_forward(const NetShape& S, const float* __restrict__ prm, const float4* pts, int n, int m,
                            float inv_ell, LearnSmem& s) {
    const int d = S.d, H = S.H, R = S.R, P = n + m;
    __shared__ float cen[4];
    if (threadIdx.x < 4) {
        float c = 0.f;
        for (int i = 0; i < n; ++i) {
            const float4 x = pts[i];
            c += threadIdx.x == 0 ? x.x : threadIdx.x == 1 ? x.y : threadIdx.x == 2 ? x.z : x.w;
        }
        cen[threadIdx.x] = c / n;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const float4 x = pts[p];
        s.U[p * 4 + 0] = (x.x - cen[0]) * inv_ell;
        s.U[p * 4 + 1] = (x.y - cen[1]) * inv_ell;
        s.U[p * 4 + 2] = (x.z - cen[2]) * inv_ell;
        s.U[p * 4 + 3] = d == 4 ? (x.w - cen[3]) * inv_ell : 0.f;
    }
    __syncthreads();
    const float* W1 = prm + S.oW1();
    const float* b1 = prm + S.ob1();
    const float* W2 = prm + S.oW2();
    const float* b2 = prm + S.ob2();
    const float* Wo = prm + S.oWo();
    const float* bo = prm + S.obo();
    for (int e = threadIdx.x; e < P * H; e += blockDim.x) {
        const int p = e / H, h = e % H;
        float a = b1[h];
        for (int c = 0; c < d; ++c) a = fmaf(W1[c * H + h], s.U[p * 4 + c], a);
        s.Z1[e] = tanhf(a);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < P * H; e += blockDim.x) {
        const int p = e / H, h = e % H;
        float a = b2[h];
        for (int k = 0; k < H; ++k) a = fmaf(W2[k * H + h], s.Z1[p * H + k], a);
        s.PHI[e] = tanhf(a);
    }
    __syncthreads();
    for (int h = threadIdx.x; h < 2 * H; h += blockDim.x) {
        const int hh = h % H;
        const bool nb = h >= H;
        const int p0 = nb ? n : 0, p1 = nb ? P : n;
        float acc = 0.f;
        for (int p = p0; p < p1; ++p) acc += s.PHI[p * H + hh];
        s.gh[h] = p1 > p0 ? acc / (p1 - p0) : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * R; e += blockDim.x) {
        const int i = e / R, r = e % R;
        float v = bo[r];
        for (int h = 0; h < H; ++h) v = fmaf(Wo[h * R + r], s.PHI[i * H + h], v);
        for (int h = 0; h < 2 * H; ++h) v = fmaf(Wo[(H + h) * R + r], s.gh[h], v);
        s.V[e] = v;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kTB)
learn_kernel(NetShape S, const float* __restrict__ prm, const int2* __restrict__ blk, int64_t nblocks,
             const int64_t* __restrict__ train, const float4* __restrict__ xs, float inv_ell,
             const float* __restrict__ D, float inv_normD, float* __restrict__ grad, double* __restrict__ loss) {
    extern __shared__ float sm[];
    __shared__ float4 pts[kMaxPts];
    __shared__ int s_n, s_m;
    const int H = S.H, R = S.R, d = S.d;
    LearnSmem s = carve(sm, H, R);
    const int64_t b = train[blockIdx.x];
    {
        int n, m;
        gather_points(blk, nblocks, b, xs, pts, &n, &m);
        if (threadIdx.x == 0) { s_n = n; s_m = m; }
    }
    __syncthreads();
    const int n = s_n, m = s_m, P = n + m;
    net_forward(S, prm, pts, n, m, inv_ell, s);
    const float beta = prm[S.obeta()];
    const float b2f = beta * beta;
    // E = beta^2 V V^T - D (row i per thread), loss and dV = 4 beta^2 E V / |D|^2
    const float* Db = D + (int64_t)blockIdx.x * kTB * kTB;
    double lrow = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        float dv[kMaxR];
        for (int r = 0; r < R; ++r) dv[r] = 0.f;
        for (int j = 0; j < n; ++j) {
            float vv = 0.f;
            for (int r = 0; r < R; ++r) vv = fmaf(s.V[i * R + r], s.V[j * R + r], vv);
            const float e = b2f * vv - Db[i * kTB + j];
            lrow += (double)e * e;
            for (int r = 0; r < R; ++r) dv[r] = fmaf(e, s.V[j * R + r], dv[r]);
        }
        for (int r = 0; r < R; ++r) s.dV[i * R + r] = 4.f * b2f * inv_normD * dv[r];
    }
    for (int off = 16; off; off >>= 1) lrow += __shfl_xor_sync(0xffffffffu, lrow, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, lrow * inv_normD);
    __syncthreads();
    const float* W2 = prm + S.oW2();
    const float* Wo = prm + S.oWo();
    // head: dbo, dWo, dPHI (direct + pooled)
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        float a = 0.f;
        for (int i = 0; i < n; ++i) a += s.dV[i * R + r];
        s.sdV[r] = a;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += blockDim.x) atomicAdd(&grad[S.obo() + r], s.sdV[r]);
    for (int e = threadIdx.x; e < 3 * H * R; e += blockDim.x) {
        const int h = e / R, r = e % R;
        float a;
        if (h < H) {
            a = 0.f;
            for (int i = 0; i < n; ++i) a = fmaf(s.PHI[i * H + h], s.dV[i * R + r], a);
        } else {
            a = s.gh[h - H] * s.sdV[r];
        }
        atomicAdd(&grad[S.oWo() + e], a);
    }
    for (int e = threadIdx.x; e < P * H; e += blockDim.x) {
        const int p = e / H, h = e % H;
        float a = 0.f;
        if (p < n) {
            for (int r = 0; r < R; ++r) a = fmaf(Wo[h * R + r], s.dV[p * R + r], a);
            float g = 0.f;
            for (int r = 0; r < R; ++r) g = fmaf(Wo[(H + h) * R + r], s.sdV[r], g);
            a += g / n;
        } else {
            float g = 0.f;
            for (int r = 0; r < R; ++r) g = fmaf(Wo[(2 * H + h) * R + r], s.sdV[r], g);
            a = g / m;
        }
        const float phi = s.PHI[e];
        s.dPHI[e] = a * (1.f - phi * phi);  // gradient wrt the layer-2 pre-activation
    }
    __syncthreads();
    // layer 2: db2, dW2, dZ1 -> layer-1 pre-activation
    for (int e = threadIdx.x; e < H * H + H; e += blockDim.x) {
        float a = 0.f;
        if (e < H * H) {
            const int k = e / H, h = e % H;
            for (int p = 0; p < P; ++p) a = fmaf(s.Z1[p * H + k], s.dPHI[p * H + h], a);
            atomicAdd(&grad[S.oW2() + e], a);
        } else {
            const int h = e - H * H;
            for (int p = 0; p < P; ++p) a += s.dPHI[p * H + h];
            atomicAdd(&grad[S.ob2() + h], a);
        }
    }
    for (int e = threadIdx.x; e < P * H; e += blockDim.x) {
        const int p = e / H, k = e % H;
        float a = 0.f;
        for (int h = 0; h < H; ++h) a = fmaf(W2[k * H + h], s.dPHI[p * H + h], a);
        const float z = s.Z1[e];
        s.dZ1[e] = a * (1.f - z * z);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < d * H + H; e += blockDim.x) {
        float a = 0.f;
        if (e < d * H) {
            const int c = e / H, h = e % H;
            for (int p = 0; p < P; ++p) a = fmaf(s.U[p * 4 + c], s.dZ1[p * H + h], a);
            atomicAdd(&grad[S.oW1() + e], a);
        } else {
            const int h = e - d * H;
            for (int p = 0; p < P; ++p) a += s.dZ1[p * H + h];
            atomicAdd(&grad[S.ob1() + h], a);
        }
    }
}

__global__ void adam_kernel(int n, int n_train, float* __restrict__ prm, const float* __restrict__ g,
                            float* __restrict__ m1, float* __restrict__ m2, float lr, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_train) return;  // the last parameter (beta) stays fixed
    const float gi = g[i];
    const float a = 0.9f * m1[i] + 0.1f * gi;
    const float v = 0.999f * m2[i] + 0.001f * gi * gi;
    m1[i] = a;
    m2[i] = v;
    prm[i] -= lr * (a / c1) / (sqrtf(v / c2) + 1e-8f);
    (void)n;
}

__global__ void __launch_bounds__(kTB)
vectors_kernel(NetShape S, const float* __restrict__ prm, const int2* __restrict__ blk, int64_t nblocks,
               const float4* __restrict__ xs, float inv_ell, float* __restrict__ Vout) {
    extern __shared__ float sm[];
    __shared__ float4 pts[kMaxPts];
    __shared__ int s_n, s_m;
    LearnSmem s = carve(sm, S.H, S.R);
    const int64_t b = blockIdx.x;
    {
        int n, m;
        gather_points(blk, nblocks, b, xs, pts, &n, &m);
        if (threadIdx.x == 0) { s_n = n; s_m = m; }
    }
    __syncthreads();
    const int n = s_n, m = s_m, R = S.R;
    net_forward(S, prm, pts, n, m, inv_ell, s);
    const float beta = prm[S.obeta()];
    float* vb = Vout + b * kTB * R;
    for (int e = threadIdx.x; e < kTB * R; e += blockDim.x) vb[e] = (e / R < n) ? beta * s.V[e] : 0.f;
}

}  // namespace

struct LearnState {
    NetShape S{};
    int64_t ntrain = 0;
    int64_t* train = nullptr;   // device
    float* D = nullptr;         // device [ntrain][kTB][kTB]
    float* prm = nullptr;       // device parameters
    float* grad = nullptr;
    float* m1 = nullptr;
    float* m2 = nullptr;
    double* acc = nullptr;      // device scalars
    float inv_normD = 1.f;
    float inv_ell = 1.f;
    double sigma2 = -1.0;
};

void free_learn(fkt_plan_s* P) {
    LearnState* L = static_cast<LearnState*>(P->learn);
    if (!L) return;
    cudaFree(L->train);
    cudaFree(L->D);
    cudaFree(L->prm);
    cudaFree(L->grad);
    cudaFree(L->m1);
    cudaFree(L->m2);
    cudaFree(L->acc);
    delete L;
    P->learn = nullptr;
    cudaFree(P->pc_learned);
    P->pc_learned = nullptr;
}

static int learn_loss_grad(fkt_plan_s* P, LearnState* L, const float* prm_dev, double* loss, bool want_grad) {
    cudaStream_t st = P->stream;
    const size_t smem = sizeof(float) * learn_smem_floats(L->S.H, L->S.R);
    FKT_CUDA_TRY(cudaFuncSetAttribute(learn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FKT_CUDA_TRY(cudaMemsetAsync(L->grad, 0, sizeof(float) * L->S.n(), st));
    FKT_CUDA_TRY(cudaMemsetAsync(L->acc, 0, sizeof(double) * 4, st));
    learn_kernel<<<(unsigned)L->ntrain, kTB, smem, st>>>(L->S, prm_dev, P->blk_range, P->nblocks, L->train, P->xs,
                                                         L->inv_ell, L->D, L->inv_normD, L->grad, L->acc);
    FKT_CUDA_TRY(cudaGetLastError());
    if (loss) {
        FKT_CUDA_TRY(cudaMemcpyAsync(loss, L->acc, sizeof(double), cudaMemcpyDeviceToHost, st));
        FKT_CUDA_TRY(cudaStreamSynchronize(st));
    }
    (void)want_grad;
    return FKT_OK;
}

int precond_learn(fkt_plan_s* P, double sigma2, const fkt_learn_opts* opts_in, fkt_learn_info* info) {
    if (P->nprob) return FKT_ERR_UNSUPPORTED;
    auto t0 = std::chrono::steady_clock::now();
    fkt_learn_opts o{8, 32, 300, 3e-3f, 512, 1, 0};
    if (opts_in) o = *opts_in;
    if (o.rank < 1 || o.rank > kMaxR || o.hidden < 8 || o.hidden > kMaxH || o.steps < 0 || !(o.lr > 0.f) ||
        o.train_blocks < 1)
        return FKT_ERR_INVALID_ARG;
    int rc = precond_setup(P, sigma2);
    if (rc) return rc;
    free_learn(P);
    LearnState* L = new LearnState();
    P->learn = L;
    L->S = NetShape{P->d, o.hidden, o.rank};
    L->sigma2 = sigma2;
    L->inv_ell = (float)(1.0 / P->kernel.lengthscale);
    cudaStream_t st = P->stream;
    // training blocks: every stride-th block
    const int64_t stride = std::max<int64_t>(1, P->nblocks / o.train_blocks);
    std::vector<int64_t> tr;
    for (int64_t b = 0; b < P->nblocks && (int64_t)tr.size() < o.train_blocks; b += stride) tr.push_back(b);
    L->ntrain = (int64_t)tr.size();
    const int np = L->S.n();
    FKT_CUDA_TRY(cudaMalloc(&L->train, 8 * L->ntrain));
    FKT_CUDA_TRY(cudaMalloc(&L->D, sizeof(float) * kTB * kTB * L->ntrain));
    FKT_CUDA_TRY(cudaMalloc(&L->prm, sizeof(float) * np));
    FKT_CUDA_TRY(cudaMalloc(&L->grad, sizeof(float) * np));
    FKT_CUDA_TRY(cudaMalloc(&L->m1, sizeof(float) * np));
    FKT_CUDA_TRY(cudaMalloc(&L->m2, sizeof(float) * np));
    FKT_CUDA_TRY(cudaMalloc(&L->acc, sizeof(double) * 4));
    FKT_CUDA_TRY(cudaMemcpy(L->train, tr.data(), 8 * L->ntrain, cudaMemcpyHostToDevice));
    // teacher
    const size_t tsmem = sizeof(float) * ((size_t)2 * kNbrHalf * kLdS + (size_t)2 * kNbrHalf * kLdY);
    FKT_CUDA_TRY(cudaFuncSetAttribute(teacher_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem));
    teacher_kernel<<<(unsigned)L->ntrain, 256, tsmem, st>>>(P->blk_range, P->nblocks, L->train, P->xs, P->kp,
                                                            (float)sigma2, L->D, P->d_err);
    FKT_CUDA_TRY(cudaGetLastError());
    FKT_CUDA_TRY(cudaMemsetAsync(L->acc, 0, sizeof(double) * 4, st));
    teacher_stats_kernel<<<(unsigned)L->ntrain, 256, 0, st>>>(L->D, P->blk_range, L->train, L->acc);
    double hs[2];
    FKT_CUDA_TRY(cudaMemcpyAsync(hs, L->acc, sizeof(hs), cudaMemcpyDeviceToHost, st));
    FKT_CUDA_TRY(cudaStreamSynchronize(st));
    int herr = 0;
    FKT_CUDA_TRY(cudaMemcpy(&herr, P->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) {
        FKT_CUDA_TRY(cudaMemset(P->d_err, 0, sizeof(int)));
        free_learn(P);
        return FKT_ERR_INVALID_ARG;  // a neighbourhood matrix was not positive definite in float32
    }
    L->inv_normD = hs[0] > 0 ? (float)(1.0 / hs[0]) : 1.f;
    const double mean_diag = hs[1] / std::max<int64_t>(L->ntrain, 1);
    // initial parameters: N(0, 1/fan_in) weights, zero biases, small output layer
    std::vector<float> h(np, 0.f);
    std::mt19937 gen((unsigned)o.seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    const NetShape& S = L->S;
    for (int i = 0; i < S.d * S.H; ++i) h[S.oW1() + i] = nd(gen) / sqrtf((float)S.d);
    for (int i = 0; i < S.H * S.H; ++i) h[S.oW2() + i] = nd(gen) / sqrtf((float)S.H);
    for (int i = 0; i < 3 * S.H * S.R; ++i) h[S.oWo() + i] = 0.1f * nd(gen) / sqrtf((float)(3 * S.H));
    h[S.obeta()] = (float)sqrt(std::max(mean_diag, 1e-12));
    FKT_CUDA_TRY(cudaMemcpy(L->prm, h.data(), sizeof(float) * np, cudaMemcpyHostToDevice));
    FKT_CUDA_TRY(cudaMemset(L->m1, 0, sizeof(float) * np));
    FKT_CUDA_TRY(cudaMemset(L->m2, 0, sizeof(float) * np));
    double loss0 = 0, loss1 = 0;
    if ((rc = learn_loss_grad(P, L, L->prm, &loss0, true))) return rc;
    for (int step = 1; step <= o.steps; ++step) {
        if (step > 1 && (rc = learn_loss_grad(P, L, L->prm, nullptr, true))) return rc;
        const float c1 = 1.f - powf(0.9f, (float)step), c2 = 1.f - powf(0.999f, (float)step);
        adam_kernel<<<(np + 255) / 256, 256, 0, st>>>(np, np - 1, L->prm, L->grad, L->m1, L->m2, o.lr, c1, c2);
        FKT_CUDA_TRY(cudaGetLastError());
    }
    if ((rc = learn_loss_grad(P, L, L->prm, &loss1, true))) return rc;
    // install A_bb^{-1} + beta^2 V V^T for every block
    if (!P->pc_learned) FKT_CUDA_TRY(cudaMalloc(&P->pc_learned, sizeof(float) * kTB * kTB * P->nblocks));
    if (o.install_teacher) {
        if (L->ntrain != P->nblocks) return FKT_ERR_INVALID_ARG;  // every block needs its teacher
        if ((rc = precond_build(P, sigma2, nullptr, 0, L->D, P->pc_learned))) return rc;
    } else {
        float* V = nullptr;
        FKT_CUDA_TRY(cudaMalloc(&V, sizeof(float) * kTB * S.R * P->nblocks));
        const size_t smem = sizeof(float) * learn_smem_floats(S.H, S.R);
        FKT_CUDA_TRY(cudaFuncSetAttribute(vectors_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        vectors_kernel<<<(unsigned)P->nblocks, kTB, smem, st>>>(S, L->prm, P->blk_range, P->nblocks, P->xs, L->inv_ell, V);
        FKT_CUDA_TRY(cudaGetLastError());
        rc = precond_build(P, sigma2, V, S.R, nullptr, P->pc_learned);
        cudaFree(V);
        if (rc) return rc;
    }
    FKT_CUDA_TRY(cudaStreamSynchronize(st));
    P->pc_learned_sigma2 = sigma2;
    if (info) {
        info->nparams = np;
        info->ntrain = (int)L->ntrain;
        info->loss_initial = loss0;
        info->loss_final = loss1;
        info->train_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return FKT_OK;
}

int learn_params(fkt_plan_s* P, float* out, int* nparams) {
    LearnState* L = static_cast<LearnState*>(P->learn);
    if (!L || !nparams) return FKT_ERR_INVALID_ARG;
    *nparams = L->S.n();
    if (out) FKT_CUDA_TRY(cudaMemcpy(out, L->prm, sizeof(float) * L->S.n(), cudaMemcpyDeviceToHost));
    return FKT_OK;
}

int learn_eval(fkt_plan_s* P, const float* params, double* loss, float* grad) {
    LearnState* L = static_cast<LearnState*>(P->learn);
    if (!L || !params) return FKT_ERR_INVALID_ARG;
    const int np = L->S.n();
    float* tmp = nullptr;
    FKT_CUDA_TRY(cudaMalloc(&tmp, sizeof(float) * np));
    FKT_CUDA_TRY(cudaMemcpy(tmp, params, sizeof(float) * np, cudaMemcpyHostToDevice));
    double l = 0;
    int rc = learn_loss_grad(P, L, tmp, &l, true);
    if (!rc && grad) {
        cudaError_t e = cudaMemcpy(grad, L->grad, sizeof(float) * np, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = FKT_ERR_CUDA;
    }
    cudaFree(tmp);
    if (loss) *loss = l;
    return rc;
}

int learn_teacher(fkt_plan_s* P, int64_t* blocks, float* D) {
    LearnState* L = static_cast<LearnState*>(P->learn);
    if (!L) return FKT_ERR_INVALID_ARG;
    if (blocks) FKT_CUDA_TRY(cudaMemcpy(blocks, L->train, 8 * L->ntrain, cudaMemcpyDeviceToHost));
    if (D) FKT_CUDA_TRY(cudaMemcpy(D, L->D, sizeof(float) * kTB * kTB * L->ntrain, cudaMemcpyDeviceToHost));
    return FKT_OK;
}

}  // namespace fkt
