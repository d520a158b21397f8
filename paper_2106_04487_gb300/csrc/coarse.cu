// Two-level (balancing) coarse correction of fkt_solve's preconditioner.
//
// CG on (Ktilde + sigma2 I) x = b with a smooth kernel and a small sigma2 is slowed by the
// smooth global modes of K: many eigenvalues spread between sigma2 and |K|, carried by
// functions that vary slowly over the whole point set.  A block-diagonal preconditioner
// cannot represent them (it acts inside one target block at a time).  The coarse space Q
// (N x R, orthonormal columns) spans R random Fourier features of the kernel,
// z_c(x) = cos(omega_c . x + phi_c) with omega_c drawn from the kernel's spectral density
// (Bochner's theorem: K(x - y) / K(0) = E[cos(omega . (x - y))]), so span(Q) approximates the
// leading eigenspace of K.  With A = Ktilde + sigma2 I, W = A Q and E = Q^T W (R x R) the
// preconditioner is the balancing two-level form
//     P = Q E^-1 Q^T + (I - Q E^-1 W^T) M (I - W E^-1 Q^T),
// M = the chosen first-level preconditioner (identity, block-Jacobi or the learned blocks).
// P is symmetric positive semi-definite whenever E and M are (E is symmetrised), even though
// Ktilde itself is only approximately symmetric.  Applied to r:
//     c = Q^T r,  t = r - W E^-1 c,  m = M t,  z = m + Q E^-1 (c - W^T m).
// The paper solves its GP systems with plain CG on FKT products (Sec. C); this
// preconditioner is not from the paper.
//
// Set-up (once per sigma2, rank and seed): the R features in caller order, their Gram matrix
// (float64 sums), Q = Z L^-T from its Cholesky factor (host, float64), W = fkt_mvm(Q) +
// sigma2 Q (R / 64 products), E = Q^T W, E^-1 (host, float64).  Per CG iteration: two
// skinny products Q^T r and W^T m, two R x R solves, two expansions.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "fkt_internal.h"

namespace fkt {
namespace {

constexpr int kMaxCoarse = 256;

struct CoarseState {
    int R = 0;               // requested rank (cache key)
    int Re = 0;              // columns of Q: features independent on these points
    int dropped = 0;         // eigen-directions of E left out of E^+
    uint64_t seed = 0;
    double sigma2 = -1.0;
    float* feat = nullptr;   // [R][5]: omega (d entries, zero-padded to 4), phase
    float* Q = nullptr;      // [R][N] orthonormal coarse basis, caller order
    float* W = nullptr;      // [R][N] (Ktilde + sigma2 I) Q; holds the raw features during set-up
    float* Y = nullptr;      // [R][kMaxCoarse] float32 coefficients for the expansions
    double* G = nullptr;     // [R][kMaxCoarse] float64 sums (Gram matrices, Q^T r, W^T m)
    double* G2 = nullptr;    // [R][kMaxRhs]
    double* Einv = nullptr;  // [Re][Re] E^+
    float* t = nullptr;      // [tcap][N] first-level input
    int tcap = 0;
};

CoarseState* state(fkt_plan_s* P) { return static_cast<CoarseState*>(P->coarse); }

void release(CoarseState* C) {
    if (!C) return;
    cudaFree(C->feat);
    cudaFree(C->Q);
    cudaFree(C->W);
    cudaFree(C->Y);
    cudaFree(C->G);
    cudaFree(C->G2);
    cudaFree(C->Einv);
    cudaFree(C->t);
    *C = CoarseState{};
}

// Z[c][perm[t]] = cos(omega_c . x_t + phi_c): features of the sorted points written in the
// caller's order.
__global__ void coarse_features_kernel(int64_t N, int R, const float4* __restrict__ xs,
                                       const int32_t* __restrict__ perm, const float* __restrict__ feat,
                                       float* __restrict__ Z) {
    __shared__ float f[kMaxCoarse * 5];
    for (int i = threadIdx.x; i < R * 5; i += blockDim.x) f[i] = feat[i];
    __syncthreads();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
        const float4 x = xs[t];
        const int64_t o = perm[t];
        for (int c = 0; c < R; ++c) {
            const float* w = f + 5 * c;
            const float a = fmaf(w[0], x.x, fmaf(w[1], x.y, fmaf(w[2], x.z, fmaf(w[3], x.w, w[4]))));
            Z[(int64_t)c * N + o] = cosf(a);
        }
    }
}

// C[c][j] += sum_i A[c][i] B[j][i] for c < R, j < nb: 32 x 32 output tiles, the i range split
// over gridDim.z chunks; float32 sums per chunk, float64 atomics across chunks.
template <typename TB>
__global__ void __launch_bounds__(256) coarse_tdot_kernel(int64_t N, int R, int nb, const float* __restrict__ A,
                                                         const TB* __restrict__ B, int64_t chunk,
                                                         double* __restrict__ C, int ldc) {
    __shared__ float As[32][33], Bs[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int c0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int64_t i_begin = blockIdx.z * chunk, i_end = min(N, i_begin + chunk);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t i0 = i_begin; i0 < i_end; i0 += 32) {
        const int64_t i = i0 + tx;
        const bool in = i < i_end;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int row = ty + 8 * k;
            As[row][tx] = (in && c0 + row < R) ? A[(int64_t)(c0 + row) * N + i] : 0.f;
            Bs[row][tx] = (in && j0 + row < nb) ? (float)B[(int64_t)(j0 + row) * N + i] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const float b = Bs[tx][kk];
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] = fmaf(As[ty + 8 * k][kk], b, acc[k]);
        }
        __syncthreads();
    }
    const int j = j0 + tx;
    if (j < nb)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = c0 + ty + 8 * k;
            if (c < R) atomicAdd(&C[(int64_t)c * ldc + j], (double)acc[k]);
        }
}

// y[c][j] = sum_k Einv[c][k] (u[k][j] - v[k][j]) (v may be null), float64 sums, float32 out.
__global__ void coarse_solve_kernel(int R, int nb, const double* __restrict__ Einv, const double* __restrict__ u,
                                    int ldu, const double* __restrict__ v, int ldv, float* __restrict__ y, int ldy) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= R * nb) return;
    const int c = e / nb, j = e - c * nb;
    double s = 0.0;
    for (int k = 0; k < R; ++k) s = fma(Einv[(int64_t)c * R + k], u[(int64_t)k * ldu + j] - (v ? v[(int64_t)k * ldv + j] : 0.0), s);
    y[(int64_t)c * ldy + j] = (float)s;
}

// out[j][i] = base[j][i] + sgn * sum_c A[c][i] Y[c][j] for j in this CTA's group of 16 (base:
// float64 base64, float32 base32 -- may alias out -- or none).
constexpr int kExpNb = 16;
__global__ void __launch_bounds__(256) coarse_expand_kernel(int64_t N, int R, int nb, const float* __restrict__ A,
                                                           const float* __restrict__ Y, int ldy, float sgn,
                                                           const double* __restrict__ base64, const float* base32,
                                                           float* out) {
    __shared__ float Ys[kMaxCoarse][kExpNb];
    const int j0 = blockIdx.y * kExpNb;
    for (int e = threadIdx.x; e < R * kExpNb; e += blockDim.x) {
        const int c = e / kExpNb, jj = e - c * kExpNb;
        Ys[c][jj] = j0 + jj < nb ? sgn * Y[(int64_t)c * ldy + j0 + jj] : 0.f;
    }
    __syncthreads();
    const int jn = min(kExpNb, nb - j0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        float acc[kExpNb];
#pragma unroll
        for (int jj = 0; jj < kExpNb; ++jj) acc[jj] = 0.f;
        for (int c = 0; c < R; ++c) {
            const float a = A[(int64_t)c * N + i];
#pragma unroll
            for (int jj = 0; jj < kExpNb; ++jj) acc[jj] = fmaf(a, Ys[c][jj], acc[jj]);
        }
#pragma unroll
        for (int jj = 0; jj < kExpNb; ++jj) {
            if (jj < jn) {
                const int64_t k = (int64_t)(j0 + jj) * N + i;
                const float b = base64 ? (float)base64[k] : base32 ? base32[k] : 0.f;
                out[k] = b + acc[jj];
            }
        }
    }
}

// W += sigma2 Q
__global__ void coarse_axpy_kernel(int64_t n, float a, const float* __restrict__ x, float* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = fmaf(a, x[i], y[i]);
}

unsigned grid_1d(int64_t n, int threads) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 8)); }

template <typename TB>
int tdot(fkt_plan_s* P, int R, int nb, const float* A, const TB* B, double* C, int ldc) {
    FKT_CUDA_TRY(cudaMemsetAsync(C, 0, sizeof(double) * (size_t)R * ldc, P->stream));
    const int tiles = ((R + 31) / 32) * ((nb + 31) / 32);
    int64_t splits = std::max<int64_t>(1, std::min<int64_t>((P->N + 1023) / 1024, (152 * 8 + tiles - 1) / tiles));
    int64_t chunk = ((P->N + splits - 1) / splits + 31) / 32 * 32;
    splits = (P->N + chunk - 1) / chunk;
    const dim3 grid((unsigned)((R + 31) / 32), (unsigned)((nb + 31) / 32), (unsigned)splits);
    coarse_tdot_kernel<TB><<<grid, 256, 0, P->stream>>>(P->N, R, nb, A, B, chunk, C, ldc);
    FKT_CUDA_TRY(cudaGetLastError());
    return FKT_OK;
}

int expand(fkt_plan_s* P, int R, int nb, const float* A, const float* Y, int ldy, float sgn, const double* base64,
           const float* base32, float* out) {
    const dim3 grid(grid_1d(P->N, 256), (unsigned)((nb + kExpNb - 1) / kExpNb));
    coarse_expand_kernel<<<grid, 256, 0, P->stream>>>(P->N, R, nb, A, Y, ldy, sgn, base64, base32, out);
    FKT_CUDA_TRY(cudaGetLastError());
    return FKT_OK;
}

int solve_small(fkt_plan_s* P, int R, int nb, const double* u, int ldu, const double* v, int ldv, float* y,
                int ldy) {
    const int n = R * nb;
    coarse_solve_kernel<<<(n + 127) / 128, 128, 0, P->stream>>>(R, nb, state(P)->Einv, u, ldu, v, ldv, y, ldy);
    FKT_CUDA_TRY(cudaGetLastError());
    return FKT_OK;
}

// Eigen-decomposition of a symmetric n x n matrix (row-major) by cyclic Jacobi rotations:
// A = V diag(lam) V^T, eigenvectors in the columns of V.
void sym_eig(std::vector<double> A, int n, std::vector<double>& lam, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    double total = 0.0;
    for (double v : A) total += v * v;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
        if (off <= 1e-30 * total) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (fabs(apq) <= 1e-300) continue;
                const double th = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    lam.resize(n);
    for (int i = 0; i < n; ++i) lam[i] = A[(size_t)i * n + i];
}

}  // namespace

int spectral_sample(const fkt_kernel& k, int d, int R, uint64_t seed, double* omega, double* phase) {
    std::mt19937_64 gen(seed);
    std::normal_distribution<double> normal(0.0, 1.0);
    std::uniform_real_distribution<double> unif(0.0, 6.283185307179586);
    const double ell = k.lengthscale;
    for (int c = 0; c < R; ++c) {
        // omega = g * rho with g ~ N(0, I_d); rho a scalar mixing variable per kernel
        double rho = 1.0 / ell;
        switch (k.kind) {
        case FKT_EXPONENTIAL:  // Matern nu: multivariate t with 2 nu degrees of freedom, scale 1/l
        case FKT_MATERN32:
        case FKT_MATERN52: {
            const double nu = k.kind == FKT_EXPONENTIAL ? 0.5 : k.kind == FKT_MATERN32 ? 1.5 : 2.5;
            std::chi_squared_distribution<double> chi2(2.0 * nu);
            rho = sqrt(2.0 * nu / chi2(gen)) / ell;
            break;
        }
        case FKT_CAUCHY: {  // (1 + r^2/l^2)^-1 = E_tau exp(-tau r^2 / l^2), tau ~ Exp(1)
            std::exponential_distribution<double> ex(1.0);
            rho = sqrt(2.0 * ex(gen)) / ell;
            break;
        }
        case FKT_RATQUAD: {  // Gaussian scale mixture, tau ~ Gamma(shape a, rate a)
            std::gamma_distribution<double> gam(k.alpha, 1.0 / k.alpha);
            rho = sqrt(gam(gen)) / ell;
            break;
        }
        default:  // Gaussian; Laplace 1/r has no normalisable spectral density: Gaussian features at l
            break;
        }
        for (int a = 0; a < d; ++a) omega[(size_t)c * d + a] = normal(gen) * rho;
        phase[c] = unif(gen);
    }
    return FKT_OK;
}

void free_coarse(fkt_plan_s* P) {
    CoarseState* C = state(P);
    if (!C) return;
    release(C);
    delete C;
    P->coarse = nullptr;
}

int coarse_setup(fkt_plan_s* P, double sigma2) {
    const int R = P->coarse_rank;
    if (R <= 0) return FKT_OK;
    if (P->nprob) return FKT_ERR_UNSUPPORTED;
    if (R > kMaxCoarse || 4 * (int64_t)R > P->N) return FKT_ERR_INVALID_ARG;
    if (!P->coarse) P->coarse = new CoarseState();
    CoarseState* C = state(P);
    if (C->R == R && C->seed == P->coarse_seed && C->sigma2 == sigma2) return FKT_OK;
    release(C);
    const int64_t N = P->N;
    cudaStream_t st = P->stream;
    FKT_CUDA_TRY(cudaMalloc(&C->feat, sizeof(float) * 5 * R));
    FKT_CUDA_TRY(cudaMalloc(&C->Q, sizeof(float) * R * N));
    FKT_CUDA_TRY(cudaMalloc(&C->W, sizeof(float) * R * N));
    FKT_CUDA_TRY(cudaMalloc(&C->Y, sizeof(float) * R * kMaxCoarse));
    FKT_CUDA_TRY(cudaMalloc(&C->G, sizeof(double) * R * kMaxCoarse));
    FKT_CUDA_TRY(cudaMalloc(&C->G2, sizeof(double) * R * kMaxRhs));
    FKT_CUDA_TRY(cudaMalloc(&C->Einv, sizeof(double) * R * R));
    // features -> W (as scratch)
    std::vector<double> om((size_t)R * P->d), ph(R);
    spectral_sample(P->kernel, P->d, R, P->coarse_seed, om.data(), ph.data());
    std::vector<float> f((size_t)5 * R, 0.f);
    for (int c = 0; c < R; ++c) {
        for (int a = 0; a < P->d; ++a) f[5 * c + a] = (float)om[(size_t)c * P->d + a];
        f[5 * c + 4] = (float)ph[c];
    }
    FKT_CUDA_TRY(cudaMemcpyAsync(C->feat, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice, st));
    coarse_features_kernel<<<grid_1d(N, 256), 256, 0, st>>>(N, R, P->xs, P->perm, C->feat, C->W);
    FKT_CUDA_TRY(cudaGetLastError());
    // Gram matrix G = Z^T Z of the features; Q = Z V_k diag(lam_k)^-1/2 over the eigenpairs of G
    // above 1e-5 lam_max: features that are (numerically) dependent on these points are dropped,
    // so the coarse space has Re <= R orthonormal columns.
    int rc = tdot<float>(P, R, R, C->W, C->W, C->G, kMaxCoarse);
    if (rc) return rc;
    std::vector<double> g((size_t)R * kMaxCoarse), A((size_t)R * R), lam, V;
    FKT_CUDA_TRY(cudaMemcpyAsync(g.data(), C->G, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, st));
    FKT_CUDA_TRY(cudaStreamSynchronize(st));
    auto sym = [&](int n) {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                A[(size_t)i * n + j] = 0.5 * (g[(size_t)i * kMaxCoarse + j] + g[(size_t)j * kMaxCoarse + i]);
    };
    sym(R);
    sym_eig(A, R, lam, V);
    const double gmax = *std::max_element(lam.begin(), lam.end());
    std::vector<int> keep;
    for (int i = 0; i < R; ++i)
        if (lam[i] > 1e-5 * gmax) keep.push_back(i);
    const int Re = (int)keep.size();
    if (Re == 0) return FKT_ERR_INVALID_ARG;
    std::vector<float> y((size_t)R * kMaxCoarse, 0.f);
    for (int c = 0; c < R; ++c)
        for (int e = 0; e < Re; ++e)
            y[(size_t)c * kMaxCoarse + e] = (float)(V[(size_t)c * R + keep[e]] / sqrt(lam[keep[e]]));
    FKT_CUDA_TRY(cudaMemcpyAsync(C->Y, y.data(), sizeof(float) * y.size(), cudaMemcpyHostToDevice, st));
    if ((rc = expand(P, R, Re, C->W, C->Y, kMaxCoarse, 1.f, nullptr, nullptr, C->Q))) return rc;
    // W = (Ktilde + sigma2 I) Q with the plan's own product
    for (int g0 = 0; g0 < Re; g0 += kMaxRhs) {
        const int nr = std::min(kMaxRhs, Re - g0);
        if ((rc = launch_mvm(P, C->Q + (size_t)g0 * N, C->W + (size_t)g0 * N, nr))) return rc;
    }
    coarse_axpy_kernel<<<grid_1d((int64_t)Re * N, 256), 256, 0, st>>>((int64_t)Re * N, (float)sigma2, C->Q, C->W);
    FKT_CUDA_TRY(cudaGetLastError());
    // E = Q^T W, symmetrised; E^+ over its eigenvalues above max(sigma2 / 2, 1e-6 lam_max).  With
    // Ktilde + sigma2 I positive definite every eigenvalue is >= sigma2; smaller ones are
    // directions where the approximate operator is not, and are left to the first level.
    if ((rc = tdot<float>(P, Re, Re, C->Q, C->W, C->G, kMaxCoarse))) return rc;
    FKT_CUDA_TRY(cudaMemcpyAsync(g.data(), C->G, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, st));
    FKT_CUDA_TRY(cudaStreamSynchronize(st));
    sym(Re);
    sym_eig(std::vector<double>(A.begin(), A.begin() + (size_t)Re * Re), Re, lam, V);
    const double emax = *std::max_element(lam.begin(), lam.end());
    const double tau = std::max(0.5 * sigma2, 1e-6 * emax);
    std::vector<double> Ei((size_t)Re * Re, 0.0);
    int dropped = 0;
    for (int e = 0; e < Re; ++e) {
        if (!(lam[e] > tau)) {
            ++dropped;
            continue;
        }
        const double inv = 1.0 / lam[e];
        for (int i = 0; i < Re; ++i)
            for (int j = 0; j < Re; ++j) Ei[(size_t)i * Re + j] += V[(size_t)i * Re + e] * inv * V[(size_t)j * Re + e];
    }
    if (dropped == Re) return FKT_ERR_INVALID_ARG;
    FKT_CUDA_TRY(cudaMemcpyAsync(C->Einv, Ei.data(), sizeof(double) * Ei.size(), cudaMemcpyHostToDevice, st));
    FKT_CUDA_TRY(cudaStreamSynchronize(st));
    C->Re = Re;
    C->dropped = dropped;
    P->stats.coarse_columns = Re;
    P->stats.coarse_dropped = dropped;
    C->R = R;
    C->seed = P->coarse_seed;
    C->sigma2 = sigma2;
    return FKT_OK;
}

int coarse_apply(fkt_plan_s* P, const double* r64, float* z, int nrhs) {
    CoarseState* C = state(P);
    if (!C || C->Re <= 0) return FKT_ERR_INTERNAL;
    const int R = C->Re;
    const int64_t N = P->N;
    if (C->tcap < nrhs) {
        cudaFree(C->t);
        C->t = nullptr;
        C->tcap = 0;
        FKT_CUDA_TRY(cudaMalloc(&C->t, sizeof(float) * (size_t)nrhs * N));
        C->tcap = nrhs;
    }
    int rc;
    // c = Q^T r (kept in G), t = r - W E^-1 c
    if ((rc = tdot<double>(P, R, nrhs, C->Q, r64, C->G, kMaxCoarse))) return rc;
    if ((rc = solve_small(P, R, nrhs, C->G, kMaxCoarse, nullptr, 0, C->Y, kMaxCoarse))) return rc;
    if ((rc = expand(P, R, nrhs, C->W, C->Y, kMaxCoarse, -1.f, r64, nullptr, C->t))) return rc;
    // m = M t (into z)
    if ((rc = precond_apply(P, C->t, nullptr, z, nrhs))) return rc;
    // z = m + Q E^-1 (c - W^T m)
    if ((rc = tdot<float>(P, R, nrhs, C->W, z, C->G2, kMaxRhs))) return rc;
    if ((rc = solve_small(P, R, nrhs, C->G, kMaxCoarse, C->G2, kMaxRhs, C->Y, kMaxCoarse))) return rc;
    return expand(P, R, nrhs, C->Q, C->Y, kMaxCoarse, 1.f, nullptr, z, z);
}

}  // namespace fkt

extern "C" int fkt_spectral_sample(fkt_kernel kernel, int d, int R, uint64_t seed, double* omega, double* phase) {
    if (!omega || !phase || d < 1 || d > 8 || R < 1 || R > (1 << 24)) return FKT_ERR_INVALID_ARG;
    if (kernel.kind < FKT_GAUSSIAN || kernel.kind > FKT_LAPLACE || !(kernel.lengthscale > 0.0) ||
        !std::isfinite(kernel.lengthscale) || (kernel.kind == FKT_RATQUAD && !(kernel.alpha > 0.0 && std::isfinite(kernel.alpha))))
        return FKT_ERR_INVALID_ARG;
    return fkt::spectral_sample(kernel, d, R, seed, omega, phase);
}
