// CUDA-core kernels: mass and Poisson on triangles, P1..P4.
#include <type_traits>

#include "simt_dispatch.cuh"

namespace ffc {
int launch_simt_tri(const LaunchArgs& a, int precision, bool assemble) {
  if (a.f->d != 2) return FFC_EUNSUPPORTED;
  if (a.f->kind == FFC_MASS) return simt_by_precision<2, FFC_MASS, 4>(a, precision, assemble);
  if (a.f->kind == FFC_POISSON) return simt_by_precision<2, FFC_POISSON, 4>(a, precision, assemble);
  return FFC_EUNSUPPORTED;
}
}  // namespace ffc
