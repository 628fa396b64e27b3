// Entry points whose kernels are not built yet report FFC_EUNSUPPORTED.
#include "ffc_internal.h"

namespace ffc {
int launch_adjoint(const LaunchArgs&, const double*, double*) { return FFC_EUNSUPPORTED; }
}  // namespace ffc
