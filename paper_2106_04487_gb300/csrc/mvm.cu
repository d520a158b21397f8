// Host orchestration of one FKT matrix-vector product (Algorithm 1) on the GPU:
//   permute w -> [s2m -> s2m_reduce] (second stream)  ||  near field (plan stream)
//   -> far field + combine + scatter to the caller's order.
// Right-hand sides are processed in groups of 8 (or 1 for a single right-hand side).
#include <algorithm>

#include "mvm_kernels.cuh"
#include "far_dispatch.cuh"

namespace fkt {

#define FKT_DECL_RANGE(D, A, B)                                         \
    int launch_s2m_d##D##_p##A##_##B(int p, int nrb, const FarLaunch& L); \
    int launch_far_d##D##_p##A##_##B(int p, int nrb, const FarLaunch& L);
FKT_DECL_RANGE(3, 0, 4)
FKT_DECL_RANGE(3, 5, 6)
FKT_DECL_RANGE(3, 7, 8)
FKT_DECL_RANGE(3, 9, 10)
FKT_DECL_RANGE(4, 0, 4)
FKT_DECL_RANGE(4, 5, 6)
FKT_DECL_RANGE(4, 7, 8)
#undef FKT_DECL_RANGE

static int launch_s2m_any(int d, int p, int nrb, const FarLaunch& L) {
    if (d == 3) {
        if (p <= 4) return launch_s2m_d3_p0_4(p, nrb, L);
        if (p <= 6) return launch_s2m_d3_p5_6(p, nrb, L);
        if (p <= 8) return launch_s2m_d3_p7_8(p, nrb, L);
        return launch_s2m_d3_p9_10(p, nrb, L);
    }
    if (p <= 4) return launch_s2m_d4_p0_4(p, nrb, L);
    if (p <= 6) return launch_s2m_d4_p5_6(p, nrb, L);
    return launch_s2m_d4_p7_8(p, nrb, L);
}

static int launch_far_any(int d, int p, int nrb, const FarLaunch& L) {
    if (d == 3) {
        if (p <= 4) return launch_far_d3_p0_4(p, nrb, L);
        if (p <= 6) return launch_far_d3_p5_6(p, nrb, L);
        if (p <= 8) return launch_far_d3_p7_8(p, nrb, L);
        return launch_far_d3_p9_10(p, nrb, L);
    }
    if (p <= 4) return launch_far_d4_p0_4(p, nrb, L);
    if (p <= 6) return launch_far_d4_p5_6(p, nrb, L);
    return launch_far_d4_p7_8(p, nrb, L);
}

namespace {

template <int D, int NR>
void launch_near_t(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp) {
    switch (kind) {
    case FKT_GAUSSIAN: near_kernel<D, FKT_GAUSSIAN, NR><<<grid, kTB, 0, st>>>(a, kp); break;
    case FKT_EXPONENTIAL: near_kernel<D, FKT_EXPONENTIAL, NR><<<grid, kTB, 0, st>>>(a, kp); break;
    case FKT_MATERN32: near_kernel<D, FKT_MATERN32, NR><<<grid, kTB, 0, st>>>(a, kp); break;
    case FKT_MATERN52: near_kernel<D, FKT_MATERN52, NR><<<grid, kTB, 0, st>>>(a, kp); break;
    case FKT_CAUCHY: near_kernel<D, FKT_CAUCHY, NR><<<grid, kTB, 0, st>>>(a, kp); break;
    case FKT_RATQUAD: near_kernel<D, FKT_RATQUAD, NR><<<grid, kTB, 0, st>>>(a, kp); break;
    default: near_kernel<D, FKT_LAPLACE, NR><<<grid, kTB, 0, st>>>(a, kp); break;
    }
}

template <int D, int NR>
void launch_dense_t(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp) {
    switch (kind) {
    case FKT_GAUSSIAN: dense_kernel<D, FKT_GAUSSIAN, NR><<<grid, kTB, 0, st>>>(a, kp); break;
    case FKT_EXPONENTIAL: dense_kernel<D, FKT_EXPONENTIAL, NR><<<grid, kTB, 0, st>>>(a, kp); break;
    case FKT_MATERN32: dense_kernel<D, FKT_MATERN32, NR><<<grid, kTB, 0, st>>>(a, kp); break;
    case FKT_MATERN52: dense_kernel<D, FKT_MATERN52, NR><<<grid, kTB, 0, st>>>(a, kp); break;
    case FKT_CAUCHY: dense_kernel<D, FKT_CAUCHY, NR><<<grid, kTB, 0, st>>>(a, kp); break;
    case FKT_RATQUAD: dense_kernel<D, FKT_RATQUAD, NR><<<grid, kTB, 0, st>>>(a, kp); break;
    default: dense_kernel<D, FKT_LAPLACE, NR><<<grid, kTB, 0, st>>>(a, kp); break;
    }
}

void launch_near(int d, int nrb, int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp) {
    if (d == 3) nrb == 1 ? launch_near_t<3, 1>(kind, grid, st, a, kp) : launch_near_t<3, 8>(kind, grid, st, a, kp);
    else nrb == 1 ? launch_near_t<4, 1>(kind, grid, st, a, kp) : launch_near_t<4, 8>(kind, grid, st, a, kp);
}

void launch_dense(int d, int nrb, int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp) {
    if (d == 3) nrb == 1 ? launch_dense_t<3, 1>(kind, grid, st, a, kp) : launch_dense_t<3, 8>(kind, grid, st, a, kp);
    else nrb == 1 ? launch_dense_t<4, 1>(kind, grid, st, a, kp) : launch_dense_t<4, 8>(kind, grid, st, a, kp);
}

MvmArgs base_args(fkt_plan_s* P) {
    MvmArgs a{};
    a.N = P->N;
    a.xs = P->xs;
    a.perm = P->perm;
    a.blk = P->blk_range;
    a.far_off = P->far_off;
    a.far_ent = P->far_ent;
    a.near_off = P->near_off;
    a.near_ent = P->near_ent;
    a.masks = P->masks;
    a.nd_begin = P->nd_begin;
    a.nd_end = P->nd_end;
    a.nd_cf = P->nd_cf;
    a.nd_scale = P->nd_scale;
    a.s2m_items = P->s2m_items;
    a.s2m_item_off = P->s2m_item_off;
    a.nnodes = P->nnodes;
    return a;
}

}  // namespace

int ensure_rhs_capacity(fkt_plan_s* P, int nrhs) {
    const int groups = nrhs == 1 ? 1 : (nrhs + 7) / 8;
    const int cap = nrhs == 1 ? 1 : groups * 8;
    if (cap <= P->cap_rhs) return FKT_OK;
    cudaFree(P->ws);
    cudaFree(P->ynear);
    cudaFree(P->mult);
    cudaFree(P->s2m_part);
    P->ws = P->ynear = P->mult = P->s2m_part = nullptr;
    P->cap_rhs = 0;
    const size_t NT = (size_t)P->nterms;
    FKT_CUDA_TRY(cudaMalloc(&P->ws, sizeof(float) * cap * P->N));
    FKT_CUDA_TRY(cudaMalloc(&P->ynear, sizeof(float) * cap * P->N));
    FKT_CUDA_TRY(cudaMalloc(&P->mult, sizeof(float) * cap * NT * std::max<int64_t>(P->nnodes, 1)));
    FKT_CUDA_TRY(cudaMalloc(&P->s2m_part, sizeof(float) * cap * NT * std::max<int64_t>(P->n_s2m_items, 1)));
    P->cap_rhs = cap;
    return FKT_OK;
}

int launch_mvm(fkt_plan_s* P, const float* w, float* y, int nrhs) {
    int rc = ensure_rhs_capacity(P, nrhs);
    if (rc) return rc;
    const int nrb = nrhs == 1 ? 1 : 8;
    const int groups = (nrhs + nrb - 1) / nrb;
    cudaStream_t st = P->stream, st2 = P->stream2;
    const int64_t N = P->N;
    const size_t NT = (size_t)P->nterms;
    if (P->timing) FKT_CUDA_TRY(cudaEventRecord(P->ev[0], st));
    for (int g = 0; g < groups; ++g) {
        const int nr = std::min(nrb, nrhs - g * nrb);
        MvmArgs a = base_args(P);
        a.ws = P->ws + (size_t)g * nrb * N;
        a.ynear = P->ynear + (size_t)g * nrb * N;
        a.mult = P->mult + (size_t)g * nrb * NT * P->nnodes;
        a.part = P->s2m_part + (size_t)g * nrb * NT * P->n_s2m_items;
        a.y = y + (size_t)g * nrb * N;
        a.nr = nr;
        const float* wg = w + (size_t)g * nrb * N;
        unsigned pg = (unsigned)((N + 255) / 256);
        if (nrb == 1) permute_kernel<1><<<pg, 256, 0, st>>>(N, P->perm, wg, nr, const_cast<float*>(a.ws));
        else permute_kernel<8><<<pg, 256, 0, st>>>(N, P->perm, wg, nr, const_cast<float*>(a.ws));
        FKT_CUDA_TRY(cudaGetLastError());
        // fork: s2m on the second stream while the near field runs on the plan stream
        FKT_CUDA_TRY(cudaEventRecord(P->ev[1], st));
        FKT_CUDA_TRY(cudaStreamWaitEvent(st2, P->ev[1], 0));
        FarLaunch L{&a, &P->kp, &P->tabs, P->nblocks, P->n_s2m_items, P->nnodes, st, st2};
        if (P->timing) FKT_CUDA_TRY(cudaEventRecord(P->ev[2], st2));
        rc = launch_s2m_any(P->d, P->p, nrb, L);
        if (rc) return rc;
        if (P->timing) FKT_CUDA_TRY(cudaEventRecord(P->ev[3], st2));
        FKT_CUDA_TRY(cudaEventRecord(P->ev[4], st2));
        if (P->timing) FKT_CUDA_TRY(cudaEventRecord(P->ev[5], st));
        launch_near(P->d, nrb, P->kernel.kind, (unsigned)P->nblocks, st, a, P->kp);
        FKT_CUDA_TRY(cudaGetLastError());
        if (P->timing) FKT_CUDA_TRY(cudaEventRecord(P->ev[6], st));
        FKT_CUDA_TRY(cudaStreamWaitEvent(st, P->ev[4], 0));  // join
        rc = launch_far_any(P->d, P->p, nrb, L);
        if (rc) return rc;
    }
    if (P->timing) {
        FKT_CUDA_TRY(cudaEventRecord(P->ev[7], st));
        FKT_CUDA_TRY(cudaEventSynchronize(P->ev[7]));
        float t_tot = 0, t_s2m = 0, t_near = 0, t_far = 0;
        cudaEventElapsedTime(&t_tot, P->ev[0], P->ev[7]);
        cudaEventElapsedTime(&t_s2m, P->ev[2], P->ev[3]);
        cudaEventElapsedTime(&t_near, P->ev[5], P->ev[6]);
        cudaEventElapsedTime(&t_far, P->ev[6], P->ev[7]);  // includes the wait for s2m, if any
        P->stats.last_total_ms = t_tot;
        P->stats.last_s2m_ms = t_s2m;
        P->stats.last_near_ms = t_near;
        P->stats.last_far_ms = t_far;
    }
    return FKT_OK;
}

int launch_dense(fkt_plan_s* P, const float* w, float* y, int nrhs) {
    int rc = ensure_rhs_capacity(P, nrhs);
    if (rc) return rc;
    const int nrb = nrhs == 1 ? 1 : 8;
    const int groups = (nrhs + nrb - 1) / nrb;
    const int64_t N = P->N;
    cudaStream_t st = P->stream;
    for (int g = 0; g < groups; ++g) {
        const int nr = std::min(nrb, nrhs - g * nrb);
        MvmArgs a = base_args(P);
        a.ws = P->ws + (size_t)g * nrb * N;
        a.y = y + (size_t)g * nrb * N;
        a.nr = nr;
        const float* wg = w + (size_t)g * nrb * N;
        unsigned pg = (unsigned)((N + 255) / 256);
        if (nrb == 1) permute_kernel<1><<<pg, 256, 0, st>>>(N, P->perm, wg, nr, const_cast<float*>(a.ws));
        else permute_kernel<8><<<pg, 256, 0, st>>>(N, P->perm, wg, nr, const_cast<float*>(a.ws));
        launch_dense(P->d, nrb, P->kernel.kind, (unsigned)((N + kTB - 1) / kTB), st, a, P->kp);
        FKT_CUDA_TRY(cudaGetLastError());
    }
    return FKT_OK;
}

}  // namespace fkt

// Entry points into the stage launchers above for other translation units.
namespace fkt {

int mvm_launch_s2m(int d, int p, int nrb, const FarLaunch& L) { return launch_s2m_any(d, p, nrb, L); }
int mvm_launch_far(int d, int p, int nrb, const FarLaunch& L) { return launch_far_any(d, p, nrb, L); }
void mvm_launch_near(int d, int nrb, int kind, unsigned grid, cudaStream_t st, const MvmArgs& a,
                     const KernelParams& kp) {
    launch_near(d, nrb, kind, grid, st, a, kp);
}
MvmArgs mvm_base_args(fkt_plan_s* P) { return base_args(P); }

}  // namespace fkt
