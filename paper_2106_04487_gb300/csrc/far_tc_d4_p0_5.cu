// Instantiations of the tensor-core far field for d = 4, orders 0..5.
#include "far_tc.cuh"

namespace fkt {

int launch_tc_d4_p0_5(int p, int prec, bool far, const TcLaunch& L) { return launch_tc_range<4, 0, 5>(p, prec, far, L); }

}  // namespace fkt
