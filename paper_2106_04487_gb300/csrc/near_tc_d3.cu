#include <algorithm>

// Tensor-core near-field kernel instantiations for d = 3 (one translation unit per dimension).
#include "near_tc2.cuh"

namespace fkt {

void launch_near_tc_d3(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp) {
    launch_near_tc_dim<3>(kind, grid, st, a, kp);
}

void launch_near_tc2_d3(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp,
                         unsigned* wmax) {
    cudaMemsetAsync(wmax, 0, sizeof(unsigned) * 32, st);
    const unsigned g = (unsigned)std::min<int64_t>((a.N + 255) / 256, 152 * 4);
    near_wscale_kernel<3><<<g, 256, 0, st>>>(a.N, a.rec, a.rec_f4, 4, a.nr, wmax);
    launch_near_tc2_dim<3>(kind, grid, st, a, kp, wmax);
}

}  // namespace fkt
