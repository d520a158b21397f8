// Instantiations of the s2m and far kernels for d = 3, orders 7..8 (one translation
// unit per order range so the library builds in parallel).
#include "far_dispatch.cuh"

namespace fkt {

int launch_s2m_d3_p7_8(int p, int nrb, const FarLaunch& L) { return launch_s2m_range<3, 7, 8>(p, nrb, L); }
int launch_far_d3_p7_8(int p, int nrb, const FarLaunch& L) { return launch_far_range<3, 7, 8>(p, nrb, L); }

}  // namespace fkt
