// Preconditioned conjugate gradients for (Ktilde + sigma2 I) x = b (the GP solve the paper
// performs with FKT products, Sec. C) and its block-Jacobi preconditioner.
//
// Precision: the FKT product runs in float32; iterates x and residuals r, all inner
// products and the residual updates run in float64; search directions p, products q and
// preconditioned residuals z are float32.  The preconditioner blocks are the plan's target
// blocks (<= 128 consecutive tree-ordered points of one leaf); each block matrix
// K(X_b, X_b) + sigma2 I is built, Cholesky-factored and inverted in shared memory.
#include <math.h>

#include <algorithm>
#include <vector>

#include "mvm_kernels.cuh"

namespace fkt {
namespace {

constexpr int kPcThreads = 256;
constexpr int kPcLd = kTB + 1;  // padded row stride in shared memory

template <int KIND>
__device__ float kernel_exact(float q, const KernelParams& kp) {
    return kp.scale * kval<KIND>(q, kp);
}

__device__ float kernel_any(int kind, float q, const KernelParams& kp) {
    switch (kind) {
    case FKT_GAUSSIAN: return kernel_exact<FKT_GAUSSIAN>(q, kp);
    case FKT_EXPONENTIAL: return kernel_exact<FKT_EXPONENTIAL>(q, kp);
    case FKT_MATERN32: return kernel_exact<FKT_MATERN32>(q, kp);
    case FKT_MATERN52: return kernel_exact<FKT_MATERN52>(q, kp);
    case FKT_CAUCHY: return kernel_exact<FKT_CAUCHY>(q, kp);
    case FKT_RATQUAD: return kernel_exact<FKT_RATQUAD>(q, kp);
    default: return kernel_exact<FKT_LAPLACE>(q, kp);
    }
}

// One CTA per target block: A = K(X_b, X_b) + sigma2 I (+ a correction: V V^T from addV, rank R,
// or a full matrix addT), A = L L^T, A^{-1} = L^{-T} L^{-1}.  Singular kernels have no finite
// diagonal; there K(0) is taken as 0 (the r = 0 rule).
__global__ void __launch_bounds__(kPcThreads)
precond_setup_kernel(const int2* __restrict__ blk, const float4* __restrict__ xs, KernelParams kp, float sigma2,
                     const float* __restrict__ addV, int R, const float* __restrict__ addT, float* __restrict__ inv,
                     int* err) {
    extern __shared__ float sm[];
    float* A = sm;                  // [kTB][kPcLd], lower triangle = L after the factorisation
    float* Li = sm + kTB * kPcLd;   // [kTB][kPcLd], L^{-1}
    __shared__ float4 px[kTB];
    const int2 rg = blk[blockIdx.x];
    const int n = rg.y - rg.x;
    const int tid = threadIdx.x;
    for (int i = tid; i < n; i += kPcThreads) {
        const float4 x = xs[rg.x + i];
        px[i] = make_float4(x.x * kp.sig, x.y * kp.sig, x.z * kp.sig, x.w * kp.sig);
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += kPcThreads) {
        const int i = e / n, j = e - i * n;
        if (j > i) continue;
        const float4 a = px[i], b = px[j];
        const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, dw = a.w - b.w;
        const float q = dx * dx + dy * dy + dz * dz + dw * dw;
        float v = kernel_any(kp.kind, q, kp);
        if (i == j) v = (kp.kind == FKT_LAPLACE ? 0.f : v) + sigma2;
        if (addV) {
            const float* vb = addV + (int64_t)blockIdx.x * kTB * R;
            for (int r = 0; r < R; ++r) v = fmaf(vb[i * R + r], vb[j * R + r], v);
        }
        if (addT) v += addT[(int64_t)blockIdx.x * kTB * kTB + i * kTB + j];
        A[i * kPcLd + j] = v;
    }
    __syncthreads();
    // right-looking Cholesky
    __shared__ int bad;
    if (tid == 0) bad = 0;
    for (int k = 0; k < n; ++k) {
        if (tid == 0) {
            float d = A[k * kPcLd + k];
            if (!(d > 0.f)) { bad = 1; d = 1e-30f; }
            A[k * kPcLd + k] = sqrtf(d);
        }
        __syncthreads();
        const float dk = A[k * kPcLd + k];
        for (int i = k + 1 + tid; i < n; i += kPcThreads) A[i * kPcLd + k] /= dk;
        __syncthreads();
        const int m = n - k - 1;
        for (int e = tid; e < m * m; e += kPcThreads) {
            const int i = k + 1 + e / m, j = k + 1 + e % m;
            if (j <= i) A[i * kPcLd + j] -= A[i * kPcLd + k] * A[j * kPcLd + k];
        }
        __syncthreads();
    }
    // L^{-1}, one column per thread (forward substitution)
    for (int j = tid; j < n; j += kPcThreads) {
        for (int i = 0; i < j; ++i) Li[i * kPcLd + j] = 0.f;
        Li[j * kPcLd + j] = 1.0f / A[j * kPcLd + j];
        for (int i = j + 1; i < n; ++i) {
            float s = 0.f;
            for (int k = j; k < i; ++k) s += A[i * kPcLd + k] * Li[k * kPcLd + j];
            Li[i * kPcLd + j] = -s / A[i * kPcLd + i];
        }
    }
    __syncthreads();
    // A^{-1}_ij = sum_{k >= max(i,j)} Li_ki Li_kj, stored [kTB][kTB] (rows and columns >= n are zero)
    float* out = inv + (int64_t)blockIdx.x * kTB * kTB;
    for (int e = tid; e < kTB * kTB; e += kPcThreads) {
        const int i = e / kTB, j = e - i * kTB;
        float s = 0.f;
        if (i < n && j < n)
            for (int k = max(i, j); k < n; ++k) s += Li[k * kPcLd + i] * Li[k * kPcLd + j];
        out[e] = s;
    }
    if (tid == 0 && bad) atomicExch(err, 2);
}

// z[perm[t]] = sum_j inv_b[t][j] r[perm[j]] per target block, for up to 8 right-hand sides.
// r comes either as float32 (r32) or float64 (r64).
__global__ void __launch_bounds__(kTB)
precond_apply_kernel(const int2* __restrict__ blk, const int32_t* __restrict__ perm, const float* __restrict__ inv,
                     int64_t N, int nr, const float* __restrict__ r32, const double* __restrict__ r64,
                     float* __restrict__ z) {
    __shared__ float rs[8][kTB];
    const int2 rg = blk[blockIdx.x];
    const int n = rg.y - rg.x;
    const int i = threadIdx.x;
    if (i < n) {
        const int64_t o = perm[rg.x + i];
        for (int r = 0; r < nr; ++r) rs[r][i] = r32 ? r32[r * N + o] : (float)r64[r * N + o];
    }
    __syncthreads();
    if (i >= n) return;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const float* col = inv + (int64_t)blockIdx.x * kTB * kTB + i;  // symmetric: row i = column i
    for (int j = 0; j < n; ++j) {
        const float a = col[(int64_t)j * kTB];
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[r] = fmaf(a, rs[r][j], acc[r]);
    }
    const int64_t o = perm[rg.x + i];
    for (int r = 0; r < nr; ++r) z[r * N + o] = acc[r];
}

// ----------------------------------------------------------------- CG steps
// Scalars (float64, [slot][kMaxRhs]): 0 rz(A) 1 rz(B) 2 pq 3 rr 4 bb 5 alpha-active flags
constexpr int kRzA = 0, kRzB = 1, kPq = 2, kRr = 3, kBb = 4, kAct = 5;

__device__ __forceinline__ void block_add(double v, double* dst) {
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(dst, v);
}

// x = 0, r = b, |b|^2
__global__ void cg_init_kernel(int64_t N, int nrhs, const float* __restrict__ b, double* __restrict__ x,
                               double* __restrict__ r, double* __restrict__ sc) {
    const int rh = blockIdx.y;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = b[rh * N + i];
        x[rh * N + i] = 0.0;
        r[rh * N + i] = v;
        s += v * v;
    }
    block_add(s, &sc[kBb * kMaxRhs + rh]);
}

// dst = sum a.b (float32 a, b or float64 a with float32 b)
__global__ void cg_dot_kernel(int64_t N, const double* __restrict__ a64, const float* __restrict__ a32,
                              const float* __restrict__ b, double* __restrict__ dst) {
    const int rh = blockIdx.y;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double av = a64 ? a64[rh * N + i] : (double)a32[rh * N + i];
        s += av * (double)b[rh * N + i];
    }
    block_add(s, &dst[rh]);
}

// q += sigma2 p and pq = p.q
__global__ void cg_shift_dot_kernel(int64_t N, float sigma2, const float* __restrict__ p, float* __restrict__ q,
                                    double* __restrict__ sc) {
    const int rh = blockIdx.y;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float pv = p[rh * N + i];
        const float qv = fmaf(sigma2, pv, q[rh * N + i]);
        q[rh * N + i] = qv;
        s += (double)pv * (double)qv;
    }
    block_add(s, &sc[kPq * kMaxRhs + rh]);
}

// alpha = rz / pq; x += alpha p; r -= alpha q; rr = r.r  (right-hand sides already converged are frozen)
__global__ void cg_update_kernel(int64_t N, const float* __restrict__ p, const float* __restrict__ q,
                                 double* __restrict__ x, double* __restrict__ r, double* __restrict__ sc,
                                 const double* __restrict__ rz) {
    const int rh = blockIdx.y;
    const double pq = sc[kPq * kMaxRhs + rh];
    const bool act = sc[kAct * kMaxRhs + rh] != 0.0 && pq > 0.0;
    const double alpha = act ? rz[rh] / pq : 0.0;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = rh * N + i;
        x[k] += alpha * (double)p[k];
        const double rv = r[k] - alpha * (double)q[k];
        r[k] = rv;
        s += rv * rv;
    }
    block_add(s, &sc[kRr * kMaxRhs + rh]);
}

// beta = rz_new / rz_old; p = z + beta p  (beta = 0 starts the recurrence)
__global__ void cg_direction_kernel(int64_t N, const float* __restrict__ z, float* __restrict__ p,
                                    const double* __restrict__ rz_new, const double* __restrict__ rz_old,
                                    const double* __restrict__ sc, int first) {
    const int rh = blockIdx.y;
    const bool act = sc[kAct * kMaxRhs + rh] != 0.0;
    const double beta = (first || !act || rz_old[rh] == 0.0) ? 0.0 : rz_new[rh] / rz_old[rh];
    const float bf = (float)beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = rh * N + i;
        p[k] = act ? fmaf(bf, first ? 0.f : p[k], z[k]) : 0.f;
    }
}

__global__ void cg_to_float_kernel(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// x = hi + lo: hi = x rounded to float32, lo = the float32 rounding of the remainder
__global__ void cg_split_kernel(int64_t n, const double* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float h = (float)x[i];
        hi[i] = h;
        lo[i] = (float)(x[i] - (double)h);
    }
}

// true residual: rr = |b - (q + q2 + sigma2 x)|^2 with q (+ q2) = Ktilde x (q2 may be null)
__global__ void cg_true_residual_kernel(int64_t N, float sigma2, const float* __restrict__ b,
                                        const double* __restrict__ x, const float* __restrict__ q,
                                        const float* __restrict__ q2, double* __restrict__ dst) {
    const int rh = blockIdx.y;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = rh * N + i;
        const double kx = (double)q[k] + (q2 ? (double)q2[k] : 0.0);
        const double v = (double)b[k] - (kx + (double)sigma2 * x[k]);
        s += v * v;
    }
    block_add(s, &dst[rh]);
}

}  // namespace

void free_solve(fkt_plan_s* P) {
    free_coarse(P);
    cudaFree(P->pc_inv);
    cudaFree(P->cg_x);
    cudaFree(P->cg_r);
    cudaFree(P->cg_p);
    cudaFree(P->cg_q);
    cudaFree(P->cg_z);
    cudaFree(P->cg_s);
    P->pc_inv = nullptr;
    P->cg_x = P->cg_r = P->cg_s = nullptr;
    P->cg_p = P->cg_q = P->cg_z = nullptr;
    P->cg_cap = 0;
    P->pc_sigma2 = -1.0;
}

int precond_build(fkt_plan_s* P, double sigma2, const float* addV, int R, const float* addT, float* out) {
    const size_t smem = sizeof(float) * 2 * kTB * kPcLd;
    FKT_CUDA_TRY(cudaFuncSetAttribute(precond_setup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    precond_setup_kernel<<<(unsigned)P->nblocks, kPcThreads, smem, P->stream>>>(P->blk_range, P->xs, P->kp,
                                                                                (float)sigma2, addV, R, addT, out,
                                                                                P->d_err);
    FKT_CUDA_TRY(cudaGetLastError());
    FKT_CUDA_TRY(cudaStreamSynchronize(P->stream));
    int h = 0;
    FKT_CUDA_TRY(cudaMemcpy(&h, P->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h == 2) {  // a block was not positive definite in float32
        FKT_CUDA_TRY(cudaMemset(P->d_err, 0, sizeof(int)));
        return FKT_ERR_INVALID_ARG;
    }
    return FKT_OK;
}

int precond_setup(fkt_plan_s* P, double sigma2) {
    if (!(sigma2 > 0.0) || !isfinite(sigma2)) return FKT_ERR_INVALID_ARG;
    if (P->pc_inv && P->pc_sigma2 == sigma2) return FKT_OK;
    if (!P->pc_inv) FKT_CUDA_TRY(cudaMalloc(&P->pc_inv, sizeof(float) * kTB * kTB * P->nblocks));
    P->pc_sigma2 = -1.0;
    const int rc = precond_build(P, sigma2, nullptr, 0, nullptr, P->pc_inv);
    if (rc) return rc;
    P->pc_sigma2 = sigma2;
    return FKT_OK;
}

int precond_apply(fkt_plan_s* P, const float* r, const double* r64, float* z, int nrhs) {
    if (P->pc_mode == 0) {  // identity
        const int64_t n = (int64_t)nrhs * P->N;
        if (r) FKT_CUDA_TRY(cudaMemcpyAsync(z, r, sizeof(float) * n, cudaMemcpyDeviceToDevice, P->stream));
        else cg_to_float_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, P->stream>>>(n, r64, z);
        FKT_CUDA_TRY(cudaGetLastError());
        return FKT_OK;
    }
    if (!P->pc_inv || P->pc_sigma2 < 0) return FKT_ERR_INVALID_ARG;
    const float* inv = P->pc_inv;
    if (P->pc_mode == 2) {
        if (!P->pc_learned || P->pc_learned_sigma2 != P->pc_sigma2) return FKT_ERR_INVALID_ARG;
        inv = P->pc_learned;
    }
    for (int g = 0; g < nrhs; g += 8) {
        const int nr = std::min(8, nrhs - g);
        precond_apply_kernel<<<(unsigned)P->nblocks, kTB, 0, P->stream>>>(
            P->blk_range, P->perm, inv, P->N, nr, r ? r + (size_t)g * P->N : nullptr,
            r64 ? r64 + (size_t)g * P->N : nullptr, z + (size_t)g * P->N);
        FKT_CUDA_TRY(cudaGetLastError());
    }
    return FKT_OK;
}

static int solve_once(fkt_plan_s* P, double sigma2, const float* b, float* x, double* x64, int nrhs, double tol,
                      int max_iter, fkt_solve_info* info);

// With the learned correction, a run that does not converge is repeated with plain block-Jacobi.
int solve(fkt_plan_s* P, double sigma2, const float* b, float* x, double* x64, int nrhs, double tol, int max_iter,
          fkt_solve_info* info) {
    if (P->pc_mode != 2) return solve_once(P, sigma2, b, x, x64, nrhs, tol, max_iter, info);
    if (!P->pc_learned || P->pc_learned_sigma2 != sigma2) return FKT_ERR_INVALID_ARG;
    int rc = solve_once(P, sigma2, b, x, x64, nrhs, tol, max_iter, info);
    if (rc != FKT_ERR_NOT_CONVERGED) return rc;
    P->pc_mode = 1;
    rc = solve_once(P, sigma2, b, x, x64, nrhs, tol, max_iter, info);
    P->pc_mode = 2;
    if (info) info->used_fallback = 1;
    return rc;
}

// z = P^{-1} r: the first-level preconditioner alone, or inside the two-level coarse correction.
static int apply_pc(fkt_plan_s* P, const double* r64, float* z, int nrhs) {
    return P->coarse_rank > 0 ? coarse_apply(P, r64, z, nrhs) : precond_apply(P, nullptr, r64, z, nrhs);
}

// x (float32) or x64 (float64): exactly one is non-null.
static int solve_once(fkt_plan_s* P, double sigma2, const float* b, float* x, double* x64, int nrhs, double tol,
                      int max_iter, fkt_solve_info* info) {
    int rc = P->pc_mode ? precond_setup(P, sigma2) : FKT_OK;
    if (rc) return rc;
    if (P->coarse_rank > 0 && (rc = coarse_setup(P, sigma2))) return rc;
    const int64_t N = P->N;
    cudaStream_t st = P->stream;
    if (P->cg_cap < nrhs) {
        cudaFree(P->cg_x); cudaFree(P->cg_r); cudaFree(P->cg_p); cudaFree(P->cg_q); cudaFree(P->cg_z);
        P->cg_cap = 0;
        const size_t n = (size_t)nrhs * N;
        FKT_CUDA_TRY(cudaMalloc(&P->cg_x, 8 * n));
        FKT_CUDA_TRY(cudaMalloc(&P->cg_r, 8 * n));
        FKT_CUDA_TRY(cudaMalloc(&P->cg_p, 4 * n));
        FKT_CUDA_TRY(cudaMalloc(&P->cg_q, 4 * n));
        FKT_CUDA_TRY(cudaMalloc(&P->cg_z, 4 * n));
        P->cg_cap = nrhs;
    }
    if (!P->cg_s) FKT_CUDA_TRY(cudaMalloc(&P->cg_s, sizeof(double) * 8 * kMaxRhs));
    double* sc = P->cg_s;
    const dim3 grid((unsigned)std::min<int64_t>((N + 255) / 256, 152 * 4), (unsigned)nrhs);
    const float s2 = (float)sigma2;
    std::vector<double> act(kMaxRhs, 0.0), host(8 * kMaxRhs, 0.0);
    for (int i = 0; i < nrhs; ++i) act[i] = 1.0;
    FKT_CUDA_TRY(cudaMemsetAsync(sc, 0, sizeof(double) * 8 * kMaxRhs, st));
    FKT_CUDA_TRY(cudaMemcpyAsync(sc + kAct * kMaxRhs, act.data(), sizeof(double) * kMaxRhs, cudaMemcpyHostToDevice, st));
    cg_init_kernel<<<grid, 256, 0, st>>>(N, nrhs, b, P->cg_x, P->cg_r, sc);
    // z = M^{-1} r, rz = r.z, p = z
    if ((rc = apply_pc(P, P->cg_r, P->cg_z, nrhs))) return rc;
    double* rz_cur = sc + kRzA * kMaxRhs;
    double* rz_nxt = sc + kRzB * kMaxRhs;
    cg_dot_kernel<<<grid, 256, 0, st>>>(N, P->cg_r, nullptr, P->cg_z, rz_cur);
    cg_direction_kernel<<<grid, 256, 0, st>>>(N, P->cg_z, P->cg_p, rz_cur, rz_cur, sc, 1);
    FKT_CUDA_TRY(cudaGetLastError());
    FKT_CUDA_TRY(cudaMemcpyAsync(host.data(), sc, sizeof(double) * 8 * kMaxRhs, cudaMemcpyDeviceToHost, st));
    FKT_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<double> bb(nrhs);
    for (int i = 0; i < nrhs; ++i) bb[i] = host[kBb * kMaxRhs + i];
    const int check_every = 5;
    int it = 0;
    bool all_conv = false;
    double worst = 1.0;
    while (it < max_iter) {
        ++it;
        // q = Ktilde p, then q += sigma2 p, pq = p.q
        if ((rc = launch_mvm(P, P->cg_p, P->cg_q, nrhs))) return rc;
        FKT_CUDA_TRY(cudaMemsetAsync(sc + kPq * kMaxRhs, 0, sizeof(double) * kMaxRhs, st));
        FKT_CUDA_TRY(cudaMemsetAsync(sc + kRr * kMaxRhs, 0, sizeof(double) * kMaxRhs, st));
        FKT_CUDA_TRY(cudaMemsetAsync(rz_nxt, 0, sizeof(double) * kMaxRhs, st));
        cg_shift_dot_kernel<<<grid, 256, 0, st>>>(N, s2, P->cg_p, P->cg_q, sc);
        cg_update_kernel<<<grid, 256, 0, st>>>(N, P->cg_p, P->cg_q, P->cg_x, P->cg_r, sc, rz_cur);
        if ((rc = apply_pc(P, P->cg_r, P->cg_z, nrhs))) return rc;
        cg_dot_kernel<<<grid, 256, 0, st>>>(N, P->cg_r, nullptr, P->cg_z, rz_nxt);
        cg_direction_kernel<<<grid, 256, 0, st>>>(N, P->cg_z, P->cg_p, rz_nxt, rz_cur, sc, 0);
        FKT_CUDA_TRY(cudaGetLastError());
        std::swap(rz_cur, rz_nxt);
        if (it % check_every == 0 || it == max_iter) {
            FKT_CUDA_TRY(cudaMemcpyAsync(host.data(), sc, sizeof(double) * 8 * kMaxRhs, cudaMemcpyDeviceToHost, st));
            FKT_CUDA_TRY(cudaStreamSynchronize(st));
            all_conv = true;
            worst = 0.0;
            for (int i = 0; i < nrhs; ++i) {
                const double rel = bb[i] > 0 ? sqrt(host[kRr * kMaxRhs + i] / bb[i]) : 0.0;
                worst = std::max(worst, rel);
                if (rel <= tol) act[i] = 0.0;
                else all_conv = false;
            }
            FKT_CUDA_TRY(cudaMemcpyAsync(sc + kAct * kMaxRhs, act.data(), sizeof(double) * kMaxRhs,
                                         cudaMemcpyHostToDevice, st));
            if (all_conv) break;
        }
    }
    // the solution, and its true residual with one more product (float32 x), or two (float64 x:
    // Ktilde x = Ktilde hi + Ktilde lo, so the rounding of x to float32 does not enter)
    FKT_CUDA_TRY(cudaMemsetAsync(sc + kRr * kMaxRhs, 0, sizeof(double) * kMaxRhs, st));
    if (x64) {
        FKT_CUDA_TRY(cudaMemcpyAsync(x64, P->cg_x, sizeof(double) * (size_t)nrhs * N, cudaMemcpyDeviceToDevice, st));
        cg_split_kernel<<<grid.x * nrhs, 256, 0, st>>>((int64_t)nrhs * N, P->cg_x, P->cg_z, P->cg_p);
        if ((rc = launch_mvm(P, P->cg_z, P->cg_q, nrhs))) return rc;
        if ((rc = launch_mvm(P, P->cg_p, P->cg_z, nrhs))) return rc;
        cg_true_residual_kernel<<<grid, 256, 0, st>>>(N, s2, b, P->cg_x, P->cg_q, P->cg_z, sc + kRr * kMaxRhs);
    } else {
        cg_to_float_kernel<<<grid.x * nrhs, 256, 0, st>>>((int64_t)nrhs * N, P->cg_x, x);
        if ((rc = launch_mvm(P, x, P->cg_q, nrhs))) return rc;
        cg_true_residual_kernel<<<grid, 256, 0, st>>>(N, s2, b, P->cg_x, P->cg_q, nullptr, sc + kRr * kMaxRhs);
    }
    FKT_CUDA_TRY(cudaGetLastError());
    FKT_CUDA_TRY(cudaMemcpyAsync(host.data(), sc, sizeof(double) * 8 * kMaxRhs, cudaMemcpyDeviceToHost, st));
    FKT_CUDA_TRY(cudaStreamSynchronize(st));
    double true_worst = 0.0;
    for (int i = 0; i < nrhs; ++i)
        true_worst = std::max(true_worst, bb[i] > 0 ? sqrt(host[kRr * kMaxRhs + i] / bb[i]) : 0.0);
    if (info) {
        info->iterations = it;
        info->converged = all_conv ? 1 : 0;
        info->rel_residual = worst;
        info->true_rel_residual = true_worst;
    }
    return all_conv ? FKT_OK : FKT_ERR_NOT_CONVERGED;
}

}  // namespace fkt
