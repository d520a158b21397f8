// Instantiations of the tensor-core far field for the compressed d = 3 layout (j = k terms only,
// the Laplace kernel), orders 0..6.
#include "far_tc.cuh"

namespace fkt {

int launch_tc_diag_p0_6(int p, int prec, bool far, const TcLaunch& L) { return launch_tc_range<kDiag3, 0, 6>(p, prec, far, L); }

}  // namespace fkt
