// Instantiations of the s2m and float32 far kernels for the compressed d = 3 layout (j = k terms
// only, the Laplace kernel), orders 6..10.
#include "far_dispatch.cuh"

namespace fkt {

int launch_s2m_diag_p6_10(int p, int nrb, const FarLaunch& L) { return launch_s2m_range<kDiag3, 6, 10>(p, nrb, L); }
int launch_far_diag_p6_10(int p, int nrb, const FarLaunch& L) { return launch_far_range<kDiag3, 6, 10>(p, nrb, L); }

}  // namespace fkt
