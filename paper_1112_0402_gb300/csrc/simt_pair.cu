// CUDA-core kernel of the mass + Poisson pair: the two matrices of one Lagrange space in
// one launch (Algorithm 2 of Section 2.2 for two forms sharing the dof map and the CSR
// pattern). Each cell's geometry is computed once, each slot is loaded once and feeds an
// atomic add into each matrix; the contributions are the single-form kernels' own.
#include "simt_dispatch.cuh"

namespace ffc {
namespace {

template <int D, int Q>
int pair_run(const LaunchArgs& a, const DeviceTensors* tm, const DeviceTensors* tp, double* val_mass,
             double* val_poisson) {
  SimtParams p{};
  p.cells = a.cells;
  p.vertices = a.vertices;
  p.n_vert = a.n_vert;
  p.slot = a.slot;
  p.csr_val = val_mass;
  p.csr_val2 = val_poisson;
  p.nnz = a.nnz;
  p.n_elem = a.n_elem;
  p.status = a.status;
  p.a0b = tp->a0_f32;
  return launch_simt_one<D, FFC_PAIR_MASS_POISSON, Q, float, true>(p, tm->a0_f32, nullptr,
                                                                    static_cast<cudaStream_t>(a.stream));
}

template <int D>
int pair_by_degree(const LaunchArgs& a, const DeviceTensors* tm, const DeviceTensors* tp, double* vm, double* vp) {
  switch (a.f->q) {
    case 1: return pair_run<D, 1>(a, tm, tp, vm, vp);
    case 2: return pair_run<D, 2>(a, tm, tp, vm, vp);
    case 3: return pair_run<D, 3>(a, tm, tp, vm, vp);
    case 4: return pair_run<D, 4>(a, tm, tp, vm, vp);
  }
  return FFC_EUNSUPPORTED;
}

}  // namespace

int launch_simt_pair(const LaunchArgs& a, const DeviceTensors* t_mass, const DeviceTensors* t_poisson,
                     double* val_mass, double* val_poisson) {
  if (a.f->d == 3) return pair_by_degree<3>(a, t_mass, t_poisson, val_mass, val_poisson);
  if (a.f->d == 2) return pair_by_degree<2>(a, t_mass, t_poisson, val_mass, val_poisson);
  return FFC_EUNSUPPORTED;
}

}  // namespace ffc
