// Runtime -> compile-time dispatch for the CUDA-core kernels. Each translation
// unit that includes this header instantiates one family of (dimension, form).
#pragma once

#include "ffc_internal.h"
#include "simt_kernels.cuh"

namespace ffc {

template <int D, int FORM, int Q, typename T>
int simt_run(const LaunchArgs& a, bool assemble) {
  SimtParams p{};
  p.cells = a.cells;
  p.vertices = a.vertices;
  p.n_vert = a.n_vert;
  p.coeffs = a.coeffs;
  p.out = a.out;
  p.slot = a.slot;
  p.csr_val = a.csr_val;
  p.nnz = a.nnz;
  p.n_elem = a.n_elem;
  p.mu = a.f->mu;
  p.lambda = a.f->lambda;
  p.status = a.status;
  const void* rows = std::is_same<T, double>::value ? (const void*)a.t->a0_f64 : (const void*)a.t->a0_f32;
  const void* cols = std::is_same<T, double>::value ? (const void*)a.t->a0t_f64 : (const void*)a.t->a0t_f32;
  cudaStream_t s = static_cast<cudaStream_t>(a.stream);
  return assemble ? launch_simt_one<D, FORM, Q, T, true>(p, rows, cols, s)
                  : launch_simt_one<D, FORM, Q, T, false>(p, rows, cols, s);
}

template <int D, int FORM, int QMAX, typename T>
int simt_by_degree(const LaunchArgs& a, bool assemble) {
  switch (a.f->q) {
    case 1: return simt_run<D, FORM, 1, T>(a, assemble);
    case 2: if constexpr (QMAX >= 2) return simt_run<D, FORM, 2, T>(a, assemble); break;
    case 3: if constexpr (QMAX >= 3) return simt_run<D, FORM, 3, T>(a, assemble); break;
    case 4: if constexpr (QMAX >= 4) return simt_run<D, FORM, 4, T>(a, assemble); break;
  }
  return FFC_EUNSUPPORTED;
}

template <int D, int FORM, int QMAX>
int simt_by_precision(const LaunchArgs& a, int precision, bool assemble) {
  if (precision == FFC_FP64) return simt_by_degree<D, FORM, QMAX, double>(a, assemble);
  if (precision == FFC_FP32) return simt_by_degree<D, FORM, QMAX, float>(a, assemble);
  return FFC_EUNSUPPORTED;
}

}  // namespace ffc
