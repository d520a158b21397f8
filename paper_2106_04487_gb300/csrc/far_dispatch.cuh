// Launchers of the order-templated s2m and far kernels for one dimension.
#pragma once

#include "mvm_kernels.cuh"

namespace fkt {

struct FarLaunch {
    const MvmArgs* a;
    const KernelParams* kp;
    const FarTables* T;
    int64_t nblocks, nitems, nnodes;
    cudaStream_t s_far, s_s2m;
};

template <int D, int P, int NR>
int launch_s2m_t(const FarLaunch& L) {
    using Sh = S2MShape<D, P, NR>;
    constexpr int NT = Layout<D, P>::nterms;
    if (L.nitems == 0) return FKT_OK;
    const size_t smem = Sh::smem_bytes();
    static bool attr = false;  // per instantiation, set once
    if (!attr) {
        FKT_CUDA_TRY(cudaFuncSetAttribute(s2m_kernel<D, P, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    s2m_kernel<D, P, NR><<<(unsigned)L.nitems, Sh::WARPS * 32, smem, L.s_s2m>>>(*L.a, *L.T);
    FKT_CUDA_TRY(cudaGetLastError());
    s2m_reduce_kernel<><<<(unsigned)L.nnodes, 128, 0, L.s_s2m>>>(L.nnodes, L.a->s2m_item_off, NT * NR, L.a->part,
                                                                 L.a->mult);
    FKT_CUDA_TRY(cudaGetLastError());
    return FKT_OK;
}

template <int D, int P, int NR>
int launch_far_t(const FarLaunch& L) {
    if constexpr (NR == 1) {
        using Sh = FarShape<D, P, 1>;
        const size_t smem = Sh::smem_bytes();
        static bool attr = false;
        if (!attr) {
            FKT_CUDA_TRY(cudaFuncSetAttribute(far_kernel<D, P, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr = true;
        }
        far_kernel<D, P, 1><<<(unsigned)L.nblocks, kTB, smem, L.s_far>>>(*L.a, *L.kp, *L.T);
    } else {
        using Sh = FarMrShape<D, P>;
        if constexpr (!Sh::supported) {
            return FKT_ERR_UNSUPPORTED;
        } else {
            const size_t smem = Sh::smem_bytes();
            static bool attr = false;
            if (!attr) {
                FKT_CUDA_TRY(cudaFuncSetAttribute(far_mr_kernel<D, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                attr = true;
            }
            far_mr_kernel<D, P><<<(unsigned)L.nblocks, kTB, smem, L.s_far>>>(*L.a, *L.kp, *L.T);
        }
    }
    FKT_CUDA_TRY(cudaGetLastError());
    return FKT_OK;
}

// Orders PLO..PHI of one dimension, both right-hand-side widths.
template <int D, int PLO, int PHI>
int launch_s2m_range(int p, int nrb, const FarLaunch& L) {
    if (p == PHI) return nrb == 1 ? launch_s2m_t<D, PHI, 1>(L) : launch_s2m_t<D, PHI, 8>(L);
    if constexpr (PHI > PLO) return launch_s2m_range<D, PLO, PHI - 1>(p, nrb, L);
    return FKT_ERR_INVALID_ARG;
}

template <int D, int PLO, int PHI>
int launch_far_range(int p, int nrb, const FarLaunch& L) {
    if (p == PHI) return nrb == 1 ? launch_far_t<D, PHI, 1>(L) : launch_far_t<D, PHI, 8>(L);
    if constexpr (PHI > PLO) return launch_far_range<D, PLO, PHI - 1>(p, nrb, L);
    return FKT_ERR_INVALID_ARG;
}

}  // namespace fkt
