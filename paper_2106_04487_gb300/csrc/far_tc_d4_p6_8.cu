// Instantiations of the tensor-core far field for d = 4, orders 6..8.
#include "far_tc.cuh"

namespace fkt {

int launch_tc_d4_p6_8(int p, int prec, bool far, const TcLaunch& L) { return launch_tc_range<4, 6, 8>(p, prec, far, L); }

}  // namespace fkt
