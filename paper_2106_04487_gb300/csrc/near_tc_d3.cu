// Tensor-core near-field kernel instantiations for d = 3 (one translation unit per dimension).
#include "near_tc.cuh"

namespace fkt {

void launch_near_tc_d3(int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp) {
    launch_near_tc_dim<3>(kind, grid, st, a, kp);
}

}  // namespace fkt
