// Internal: the compiled quadrature form shared by the quadrature kernels (CUDA-core and
// tensor-core contractions in quadrature.cu, the digit-split FP64 contraction in
// quadrature_ozaki.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <vector>

struct ffc_qform {
  int kind = 0, d = 0, q = 0, g = 0, p = 0;
  int n = 0;     // local dofs
  int ngeo = 0;  // geometry nodes per cell
  int nq = 0;    // quadrature points
  int ng = 0;    // geometry entries per point
  int K = 0;     // contraction length nq * ng
  std::vector<double> X, W;  // rule: points [nq][d], weights [nq]
  std::vector<double> At;    // A~0 [n*n][K], j = k * ng + g
  std::vector<double> dgeo;  // geometry basis gradients [nq][ngeo][d]
  struct Dev {
    double* at_f64 = nullptr;  // [K][ne64], entries i1 <= i2, padded to an even count
    float* at_f32 = nullptr;   // [K][ne32], all entries, padded to a multiple of 4
    double* dgeo = nullptr;
    uint16_t* epair = nullptr;  // [n(n+1)/2]: i1 << 8 | i2
    void* tc_part[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};  // TF32 / BF16 parts
    float* tq_table = nullptr;  // the tensor-core producers' geometry table (FP32)
    void* oz_a = nullptr;       // digit planes of A~0 (BF16), per 16-column K piece
    double* oz_table = nullptr; // the digit-split kernel's geometry table (FP64) and row exponents
  };
  std::mutex lock;
  std::map<int, Dev> dev;
};

namespace ffc {
// Where a tensor-core quadrature kernel puts A_K: stored into `out` ([n_elem][n*n], float or
// double by precision), or, when `slot` is set, added into csr_val[slot[e][i]] with FP64
// atomics (Algorithm 2; a slot outside [0, nnz) sets FFC_FLAG_BOUNDS and is skipped).
struct QOut {
  void* out = nullptr;
  const int32_t* slot = nullptr;
  double* csr_val = nullptr;
  long long nnz = 0;
};
// The digit-split FP64 contraction (precision FFC_FP64_OZAKI) for n_elem cells; dv is the
// form's device state.
int run_ozaki(ffc_qform* f, ffc_qform::Dev* dv, long long n_elem, const int32_t* cells, const double* nodes,
              long long n_nodes, const QOut& o, unsigned* status, cudaStream_t s);
// FFC_EUNSUPPORTED (with the reason set) when the form is outside the kernel's range.
int ozaki_supported(const ffc_qform* f);
}  // namespace ffc
