// CUDA-core kernels: mass on tetrahedra, P1..P4.
#include <type_traits>

#include "simt_dispatch.cuh"

namespace ffc {
int launch_simt_tet_mass(const LaunchArgs& a, int precision, bool assemble) {
  if (a.f->d != 3 || a.f->kind != FFC_MASS) return FFC_EUNSUPPORTED;
  return simt_by_precision<3, FFC_MASS, 4>(a, precision, assemble);
}
}  // namespace ffc
