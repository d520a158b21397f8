// Instantiations of the s2m and far kernels for d = 2 (circular harmonics), orders 0..10.
#include "far_dispatch.cuh"

namespace fkt {

int launch_s2m_d2_p0_10(int p, int nrb, const FarLaunch& L) { return launch_s2m_range<2, 0, 10>(p, nrb, L); }
int launch_far_d2_p0_10(int p, int nrb, const FarLaunch& L) { return launch_far_range<2, 0, 10>(p, nrb, L); }

}  // namespace fkt
