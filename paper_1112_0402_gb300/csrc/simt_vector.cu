// CUDA-core kernels: vector forms on tetrahedra (convection P1..P2, elasticity P1..P3).
#include <type_traits>

#include "simt_dispatch.cuh"

namespace ffc {
int launch_simt_vector(const LaunchArgs& a, int precision, bool assemble) {
  if (a.f->d != 3) return FFC_EUNSUPPORTED;
  if (a.f->kind == FFC_NS_CONVECTION) return simt_by_precision<3, FFC_NS_CONVECTION, 2>(a, precision, assemble);
  if (a.f->kind == FFC_ELASTICITY) return simt_by_precision<3, FFC_ELASTICITY, 3>(a, precision, assemble);
  return FFC_EUNSUPPORTED;
}
}  // namespace ffc
