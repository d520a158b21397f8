// Near-field kernel instantiations for d = 4 (one translation unit per dimension so the
// library builds in parallel).
#include "near_launch.cuh"

namespace fkt {

void launch_near_d4(int nw, int tpt, int kind, unsigned grid, cudaStream_t st, const MvmArgs& a, const KernelParams& kp) {
    launch_near_dim<4>(nw, tpt, kind, grid, st, a, kp);
}

}  // namespace fkt
