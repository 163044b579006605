// Discrete adjoint (paper Sec. 2.3, Eq. dR_u, Eq. main_grad, Algorithm adjoint_ad).
#include "handle.h"

namespace hfe {

struct AdjointWork {};

hfe_status adjoint_run(hfe_handle* h, int, const double*, const double*, double, double*, double*, hfe_stats*) {
  return fail(h, HFE_EINVAL, "adjoint: not available in this build");
}

void adjoint_free(AdjointWork* w) { delete w; }

}  // namespace hfe
