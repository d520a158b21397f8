// Instantiations of the s2m and far kernels for d = 3, orders 9..10 (one translation
// unit per order range so the library builds in parallel).
#include "far_dispatch.cuh"

namespace fkt {

int launch_s2m_d3_p9_10(int p, int nrb, const FarLaunch& L) { return launch_s2m_range<3, 9, 10>(p, nrb, L); }
int launch_far_d3_p9_10(int p, int nrb, const FarLaunch& L) { return launch_far_range<3, 9, 10>(p, nrb, L); }

}  // namespace fkt
