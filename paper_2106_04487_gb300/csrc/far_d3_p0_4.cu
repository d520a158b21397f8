// Instantiations of the s2m and far kernels for d = 3, orders 0..4 (one translation
// unit per order range so the library builds in parallel).
#include "far_dispatch.cuh"

namespace fkt {

int launch_s2m_d3_p0_4(int p, int nrb, const FarLaunch& L) { return launch_s2m_range<3, 0, 4>(p, nrb, L); }
int launch_far_d3_p0_4(int p, int nrb, const FarLaunch& L) { return launch_far_range<3, 0, 4>(p, nrb, L); }

}  // namespace fkt
