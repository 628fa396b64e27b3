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
namespace quad {

// Column of the symmetric pair {a, b} (either order) in the Poisson geometry entries:
// diagonal pairs first, then (0,1) [, (0,2), (1,2)].
template <int D>
__host__ __device__ constexpr int qpair(int a, int b) {
  return a == b ? a : (D == 2 ? 2 : ((a == 0 || b == 0) ? ((a == 1 || b == 1) ? 3 : 4) : 5));
}

// Determinant of J and its adjugate A (J A = det I).
template <int D, typename T>
__host__ __device__ __forceinline__ T det_adj(const T (&J)[D][D], T (&A)[D][D]) {
  if constexpr (D == 2) {
    A[0][0] = J[1][1];
    A[0][1] = -J[0][1];
    A[1][0] = -J[1][0];
    A[1][1] = J[0][0];
    return J[0][0] * J[1][1] - J[0][1] * J[1][0];
  } else {
    A[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    A[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    A[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    A[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    A[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    A[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    A[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    A[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    A[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    return J[0][0] * A[0][0] + J[0][1] * A[1][0] + J[0][2] * A[2][0];
  }
}

// The tensor-core producers' geometry table of a form (FP64): gradients of the geometry
// basis at X = 0 [n_geometry][d], its second derivatives [n_geometry][d(d+1)/2] (geometry
// degree 2 only; differences of the gradients at X = e_c and X = 0, exact for a quadratic
// basis), then the rule's points [nq][d]. F'(X) of the cell is then affine in X:
// F'(X)[a][b] = J0[a][b] + sum_c H[a][{b,c}] X_c with J0 and H these tables contracted with
// the cell's geometry nodes.
std::vector<double> geometry_table(const ffc_qform* f);

}  // namespace quad

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
