// Entry points whose kernels are not built yet report FFC_EUNSUPPORTED.
#include "ffc_internal.h"

namespace ffc {
}  // namespace ffc
