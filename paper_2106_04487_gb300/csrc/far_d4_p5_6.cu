// Instantiations of the s2m and far kernels for d = 4, orders 5..6 (one translation
// unit per order range so the library builds in parallel).
#include "far_dispatch.cuh"

namespace fkt {

int launch_s2m_d4_p5_6(int p, int nrb, const FarLaunch& L) { return launch_s2m_range<4, 5, 6>(p, nrb, L); }
int launch_far_d4_p5_6(int p, int nrb, const FarLaunch& L) { return launch_far_range<4, 5, 6>(p, nrb, L); }

}  // namespace fkt
