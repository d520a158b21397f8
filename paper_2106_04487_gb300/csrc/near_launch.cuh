// Launcher of the near-field kernel for one dimension: kernel kind x right-hand sides per pass
// (1, 4, 8, 16, 32) x targets per thread.  Instantiated in one translation unit per dimension.
#pragma once

#include "mvm_kernels.cuh"

namespace fkt {

template <int D, int NR, int T>
void launch_near_t(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp) {
    constexpr int TH = NearShape<D, NR, T>::THREADS;
    switch (kind) {
    case FKT_GAUSSIAN: near_kernel<D, FKT_GAUSSIAN, NR, T><<<grid, TH, 0, st>>>(a, kp); break;
    case FKT_EXPONENTIAL: near_kernel<D, FKT_EXPONENTIAL, NR, T><<<grid, TH, 0, st>>>(a, kp); break;
    case FKT_MATERN32: near_kernel<D, FKT_MATERN32, NR, T><<<grid, TH, 0, st>>>(a, kp); break;
    case FKT_MATERN52: near_kernel<D, FKT_MATERN52, NR, T><<<grid, TH, 0, st>>>(a, kp); break;
    case FKT_CAUCHY: near_kernel<D, FKT_CAUCHY, NR, T><<<grid, TH, 0, st>>>(a, kp); break;
    case FKT_RATQUAD: near_kernel<D, FKT_RATQUAD, NR, T><<<grid, TH, 0, st>>>(a, kp); break;
    default: near_kernel<D, FKT_LAPLACE, NR, T><<<grid, TH, 0, st>>>(a, kp); break;
    }
}

template <int D, int NR>
void launch_near_wide_t(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp) {
    const unsigned g = grid * NearWideShape<D, NR>::SPLIT;
    switch (kind) {
    case FKT_GAUSSIAN: near_wide_kernel<D, FKT_GAUSSIAN, NR><<<g, 32, 0, st>>>(a, kp); break;
    case FKT_EXPONENTIAL: near_wide_kernel<D, FKT_EXPONENTIAL, NR><<<g, 32, 0, st>>>(a, kp); break;
    case FKT_MATERN32: near_wide_kernel<D, FKT_MATERN32, NR><<<g, 32, 0, st>>>(a, kp); break;
    case FKT_MATERN52: near_wide_kernel<D, FKT_MATERN52, NR><<<g, 32, 0, st>>>(a, kp); break;
    case FKT_CAUCHY: near_wide_kernel<D, FKT_CAUCHY, NR><<<g, 32, 0, st>>>(a, kp); break;
    case FKT_RATQUAD: near_wide_kernel<D, FKT_RATQUAD, NR><<<g, 32, 0, st>>>(a, kp); break;
    default: near_wide_kernel<D, FKT_LAPLACE, NR><<<g, 32, 0, st>>>(a, kp); break;
    }
}

template <int D, int NR>
void launch_near_tile_t(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp) {
    const unsigned g = grid * NearTileShape<D, NR>::SPLIT;
    switch (kind) {
    case FKT_GAUSSIAN: near_tile_kernel<D, FKT_GAUSSIAN, NR><<<g, 32, 0, st>>>(a, kp); break;
    case FKT_EXPONENTIAL: near_tile_kernel<D, FKT_EXPONENTIAL, NR><<<g, 32, 0, st>>>(a, kp); break;
    case FKT_MATERN32: near_tile_kernel<D, FKT_MATERN32, NR><<<g, 32, 0, st>>>(a, kp); break;
    case FKT_MATERN52: near_tile_kernel<D, FKT_MATERN52, NR><<<g, 32, 0, st>>>(a, kp); break;
    case FKT_CAUCHY: near_tile_kernel<D, FKT_CAUCHY, NR><<<g, 32, 0, st>>>(a, kp); break;
    case FKT_RATQUAD: near_tile_kernel<D, FKT_RATQUAD, NR><<<g, 32, 0, st>>>(a, kp); break;
    default: near_tile_kernel<D, FKT_LAPLACE, NR><<<g, 32, 0, st>>>(a, kp); break;
    }
}

// nw = right-hand sides of the pass (1, 4, 8, 16 or 32); grid = target blocks to cover; tpt =
// targets per thread of the single-RHS kernel (2 or 4).  Multi-RHS passes use the one-warp
// near_wide_kernel (two CTAs per target block).
template <int D>
void launch_near_dim(int nw, int tpt, int kind, unsigned grid, cudaStream_t st, const MvmArgs& a,
                     const KernelParams& kp) {
    switch (nw) {
    case 1:
        if (tpt == 4) launch_near_t<D, 1, 4>(kind, grid, st, a, kp);
        else launch_near_t<D, 1, 2>(kind, grid, st, a, kp);
        break;
    case 4: launch_near_wide_t<D, 4>(kind, grid, st, a, kp); break;
    case 8: launch_near_wide_t<D, 8>(kind, grid, st, a, kp); break;
    case 16: launch_near_tile_t<D, 16>(kind, grid, st, a, kp); break;
    default: launch_near_tile_t<D, 32>(kind, grid, st, a, kp); break;
    }
}

}  // namespace fkt
