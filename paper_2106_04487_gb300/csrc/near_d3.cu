// Near-field kernel instantiations for d = 3 (one translation unit per dimension so the
// library builds in parallel).
#include "near_launch.cuh"

namespace fkt {

void launch_near_d3(int nw, int tpt, int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp) {
    launch_near_dim<3>(nw, tpt, kind, grid, st, a, kp);
}

}  // namespace fkt
