// Instantiations of the tensor-core far field for d = 3, orders 0..6.
#include "far_tc.cuh"

namespace fkt {

int launch_tc_d3_p0_6(int p, int prec, bool far, const TcLaunch& L) { return launch_tc_range<3, 0, 6>(p, prec, far, L); }

}  // namespace fkt
