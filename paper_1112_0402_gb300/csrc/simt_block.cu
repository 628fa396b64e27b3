// Launchers of the structured contraction of the vector forms (kernels in simt_block.cuh).
#include "simt_block.cuh"

namespace ffc {
namespace {

template <int D, int FORM, int Q, typename T, bool ASSEMBLE>
int run(const LaunchArgs& a) {
  using C = BlockCfg<D, FORM, Q, T>;
  constexpr size_t SMEM = C::SMEM + BlockStaging<C, T, ASSEMBLE>::BYTES;
  auto kern = simt_block_kernel<D, FORM, Q, T, ASSEMBLE>;
  // elasticity: the whole unified L1 / shared array as shared memory, so the nine
  // geometry blocks of several resident CTAs fit (measured faster; the convection
  // kernel and the batched kernel, which lean on L1 for their streamed loads, keep the
  // default split)
  int sms = 0, per_sm = 1;
  if (launch_config(reinterpret_cast<const void*>(kern), C::NT, SMEM, FORM == FFC_ELASTICITY ? 100 : -1, &sms,
                    &per_sm) != FFC_OK)
    return FFC_ECUDA;
  SimtParams p{};
  p.cells = a.cells;
  p.vertices = a.vertices;
  p.n_vert = a.n_vert;
  p.coeffs = a.coeffs;
  p.a0 = std::is_same<T, double>::value ? (const void*)a.t->r_f64 : (const void*)a.t->r_f32;
  p.out = a.out;
  p.slot = a.slot;
  p.csr_val = a.csr_val;
  p.nnz = a.nnz;
  p.n_elem = a.n_elem;
  p.mu = a.f->mu;
  p.lambda = a.f->lambda;
  p.status = a.status;
  const long long n_tiles = (a.n_elem + C::E - 1) / C::E;
  long long grid = (long long)sms * per_sm;
  if (grid > n_tiles) grid = n_tiles;
  kern<<<unsigned(grid), C::NT, SMEM, static_cast<cudaStream_t>(a.stream)>>>(p);
  return cudaPeekAtLastError() == cudaSuccess ? FFC_OK : FFC_ECUDA;
}

template <int D, int FORM, int Q>
int by_prec(const LaunchArgs& a, int precision, bool assemble) {
  if (precision == FFC_FP64) return assemble ? run<D, FORM, Q, double, true>(a) : run<D, FORM, Q, double, false>(a);
  if (precision == FFC_FP32) return assemble ? run<D, FORM, Q, float, true>(a) : run<D, FORM, Q, float, false>(a);
  return FFC_EUNSUPPORTED;
}

}  // namespace

int launch_simt_block(const LaunchArgs& a, int precision, bool assemble) {
  const ffc_form* f = a.f;
  if (f->d != 3 || f->kr == 0 || !a.t->r_f64) return FFC_EUNSUPPORTED;
  if (f->kind == FFC_NS_CONVECTION) {
    if (f->q == 1) return by_prec<3, FFC_NS_CONVECTION, 1>(a, precision, assemble);
    if (f->q == 2) return by_prec<3, FFC_NS_CONVECTION, 2>(a, precision, assemble);
  } else if (f->kind == FFC_ELASTICITY) {
    if (f->q == 1) return by_prec<3, FFC_ELASTICITY, 1>(a, precision, assemble);
    if (f->q == 2) return by_prec<3, FFC_ELASTICITY, 2>(a, precision, assemble);
    if (f->q == 3) return by_prec<3, FFC_ELASTICITY, 3>(a, precision, assemble);
  }
  return FFC_EUNSUPPORTED;
}

}  // namespace ffc
