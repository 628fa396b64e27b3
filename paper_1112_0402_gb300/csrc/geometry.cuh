// Per-cell geometry on the device: affine Jacobian J = [x_1 - x_0, ..., x_d - x_0],
// |det J|, K = J^{-1} (all FP64), and the geometry tensor G_K of each form
// (Section 3.2: G = c det F' prod dX/dx; Section 3.3 gives G for each test case).
#pragma once

#include <cstdint>

#include "../../include/ffc_gb300.h"

namespace ffc {

constexpr int nscalar(int d, int q) { return d == 2 ? (q + 1) * (q + 2) / 2 : (q + 1) * (q + 2) * (q + 3) / 6; }
constexpr int nlocal(int form, int d, int q) {
  return (form == FFC_NS_CONVECTION || form == FFC_ELASTICITY) ? d * nscalar(d, q) : nscalar(d, q);
}
constexpr int nalpha(int form, int d, int q) {
  return form == FFC_MASS ? 1
       : form == FFC_SOURCE ? nscalar(d, q)
       : form == FFC_POISSON ? d * d
       : form == FFC_NS_CONVECTION ? nlocal(form, d, q) * d
       : d * d * d * d;
}

// Column layout of the CUDA-core kernels' reference tensor: the Poisson G_K is
// symmetric, so it is kept once per pair a1 <= a2 (Section 3.5: symmetry means fewer
// operations), d(d+1)/2 columns: diagonal pairs first, then (0,1) [, (0,2), (1,2)].
// Internal form code of the fused mass + Poisson pair (one launch, two matrices): its
// kernel columns are the mass column followed by the d(d+1)/2 symmetric Poisson columns.
constexpr int FFC_PAIR_MASS_POISSON = 100;
constexpr int nalpha_k(int form, int d, int q) {
  return form == FFC_POISSON ? d * (d + 1) / 2
       : form == FFC_PAIR_MASS_POISSON ? 1 + d * (d + 1) / 2
       : nalpha(form, d, q);
}
template <int D>
__host__ __device__ constexpr int sym_pair_index(int a, int b) {
  return a == b ? a : (D == 2 ? 2 : (a == 0 ? (b == 1 ? 3 : 4) : 5));
}

// Gathers the cell's vertex coordinates; an out-of-range vertex id is reported and
// replaced by vertex 0 (never read out of bounds).
template <int D>
__device__ __forceinline__ void gather_vertices(const int32_t* __restrict__ cells, const double* __restrict__ vertices,
                                                int64_t n_vert, int64_t e, double x[D + 1][D], bool& bad_index) {
  int id[D + 1];
  if constexpr (D == 3) {
    const int4 c = __ldg(reinterpret_cast<const int4*>(cells) + e);
    id[0] = c.x;
    id[1] = c.y;
    id[2] = c.z;
    id[3] = c.w;
  } else {
#pragma unroll
    for (int j = 0; j < 3; ++j) id[j] = __ldg(cells + e * 3 + j);
  }
  bad_index = false;
#pragma unroll
  for (int j = 0; j <= D; ++j) {
    if (id[j] < 0 || id[j] >= n_vert) {
      bad_index = true;
      id[j] = 0;
    }
    // 16-byte loads where the vertex's coordinates allow them: in 2D a vertex is one
    // 16-byte pair when its address is 16-byte aligned; in 3D its 24 bytes are a pair and
    // a single value, in the order its address's alignment gives
    const double* v = vertices + int64_t(id[j]) * D;
    const bool odd = (reinterpret_cast<uintptr_t>(v) >> 3) & 1;
    if constexpr (D == 2) {
      if (!odd) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(v));
        x[j][0] = a.x;
        x[j][1] = a.y;
      } else {
        x[j][0] = __ldg(v);
        x[j][1] = __ldg(v + 1);
      }
    } else {
      if (!odd) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(v));
        x[j][0] = a.x;
        x[j][1] = a.y;
        x[j][2] = __ldg(v + 2);
      } else {
        x[j][0] = __ldg(v);
        const double2 a = __ldg(reinterpret_cast<const double2*>(v + 1));
        x[j][1] = a.x;
        x[j][2] = a.y;
      }
    }
  }
}

// The degeneracy test |det J| <= 1e-14 h_max^d (h_max the longest edge), evaluated as
// det^2 <= 1e-28 h_max^{2d}: no square root, no division. The edges are J's columns
// (x_j - x_0) and their differences (x_j - x_i); their squared lengths are formed in
// FP32 from J, since a threshold needs no more (on GB300 every FP64 instruction is
// scarce), and the comparison is made in FP64 against the FP64 determinant.
template <int D>
__device__ __forceinline__ bool degenerate_test(const double J[D][D], double det) {
  float Jf[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) Jf[r][c] = float(J[r][c]);
  float h2 = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    float s = 0.f;
#pragma unroll
    for (int r = 0; r < D; ++r) s = fmaf(Jf[r][i], Jf[r][i], s);
    h2 = fmaxf(h2, s);
#pragma unroll
    for (int j = i + 1; j < D; ++j) {
      float t = 0.f;
#pragma unroll
      for (int r = 0; r < D; ++r) {
        const float dd = Jf[r][j] - Jf[r][i];
        t = fmaf(dd, dd, t);
      }
      h2 = fmaxf(h2, t);
    }
  }
  const double h2_64 = double(h2);
  double h2d = h2_64;
#pragma unroll
  for (int r = 1; r < D; ++r) h2d *= h2_64;
  return !(det * det > 1e-28 * h2d);
}

// Gathers the cell's vertices and computes K = J^{-1} and |det J|.
template <int D>
__device__ __forceinline__ void cell_geometry(const int32_t* __restrict__ cells, const double* __restrict__ vertices,
                                              int64_t n_vert, int64_t e, double K[D][D], double& det_abs,
                                              bool& degenerate, bool& bad_index) {
  double x[D + 1][D];
  gather_vertices<D>(cells, vertices, n_vert, e, x, bad_index);
  double J[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) J[r][c] = x[c + 1][r] - x[0][r];
  double det;
  if constexpr (D == 3) {
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    const double inv = 1.0 / det;
    // K = adj(J) / det; adj(J)[a][b] = cofactor(b, a)
    K[0][0] = c00 * inv;
    K[1][0] = c01 * inv;
    K[2][0] = c02 * inv;
    K[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * inv;
    K[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * inv;
    K[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * inv;
    K[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * inv;
    K[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * inv;
    K[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * inv;
  } else {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double inv = 1.0 / det;
    K[0][0] = J[1][1] * inv;
    K[0][1] = -J[0][1] * inv;
    K[1][0] = -J[1][0] * inv;
    K[1][1] = J[0][0] * inv;
  }
  det_abs = fabs(det);
  degenerate = degenerate_test<D>(J, det);
}

// Geometry for an FP32 contraction: J, its cofactors (adjugate) and det J in FP64,
// which is where the cancellation of a near-degenerate cell happens, then
// K = J^{-1} = adj(J) / det J formed in FP32 from them (a well-conditioned step once adj
// and det are exact to FP64). About 40% fewer FP64 instructions than cell_geometry
// followed by FP64 products; cells whose |det J| lies outside [1e-30, 1e30] take the
// all-FP64 route so the FP32 reciprocal never under- or overflows.
template <int D>
__device__ __forceinline__ void cell_geometry_f32(const int32_t* __restrict__ cells,
                                                  const double* __restrict__ vertices, int64_t n_vert, int64_t e,
                                                  float K[D][D], float& det_abs, bool& degenerate, bool& bad_index) {
  double x[D + 1][D];
  gather_vertices<D>(cells, vertices, n_vert, e, x, bad_index);
  double J[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) J[r][c] = x[c + 1][r] - x[0][r];
  double adj[D][D], det;
  if constexpr (D == 3) {
    adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
  } else {
    adj[0][0] = J[1][1];
    adj[0][1] = -J[0][1];
    adj[1][0] = -J[1][0];
    adj[1][1] = J[0][0];
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  }
  degenerate = degenerate_test<D>(J, det);
  const double ad = fabs(det);
  if (ad >= 1e-30 && ad <= 1e30) {
    const float inv = 1.0f / float(det);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) K[a][b] = float(adj[a][b]) * inv;
  } else {
    const double inv = 1.0 / det;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) K[a][b] = float(adj[a][b] * inv);
  }
  det_abs = float(ad);
}

// |det J| alone (forms whose geometry tensor needs no J^{-1}: mass and source), with the
// same degeneracy test as cell_geometry.
template <int D>
__device__ __forceinline__ void cell_det(const int32_t* __restrict__ cells, const double* __restrict__ vertices,
                                         int64_t n_vert, int64_t e, double& det_abs, bool& degenerate,
                                         bool& bad_index) {
  double x[D + 1][D];
  gather_vertices<D>(cells, vertices, n_vert, e, x, bad_index);
  double J[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) J[r][c] = x[c + 1][r] - x[0][r];
  double det;
  if constexpr (D == 3) {
    det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) + J[0][1] * (J[1][2] * J[2][0] - J[1][0] * J[2][2]) +
          J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  } else {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  }
  det_abs = fabs(det);
  degenerate = degenerate_test<D>(J, det);
}

// Geometry tensor of the form, written as G[alpha] (alpha layouts documented in
// form_compiler.cpp). `w` is the cell's coefficient vector (convection only).
template <int D, int FORM, int Q, typename Store>
__device__ __forceinline__ void geometry_tensor(const double K[D][D], double det, const double* w, double mu,
                                                double lambda, Store&& store) {
  if constexpr (FORM == FFC_MASS) {
    store(0, det);
  } else if constexpr (FORM == FFC_POISSON) {
#pragma unroll
    for (int a1 = 0; a1 < D; ++a1)
#pragma unroll
      for (int a2 = 0; a2 < D; ++a2) {
        double s = 0.0;
#pragma unroll
        for (int b = 0; b < D; ++b) s += K[a1][b] * K[a2][b];
        store(a1 * D + a2, det * s);
      }
  } else if constexpr (FORM == FFC_NS_CONVECTION) {
    constexpr int NS = nscalar(D, Q);
#pragma unroll
    for (int ct = 0; ct < D; ++ct)
#pragma unroll
      for (int st = 0; st < NS; ++st) {
        const int t = ct * NS + st;
        const double dw = det * w[t];
#pragma unroll
        for (int a = 0; a < D; ++a) store(t * D + a, dw * K[a][ct]);
      }
  } else {  // elasticity
    double KK[D][D];
#pragma unroll
    for (int a1 = 0; a1 < D; ++a1)
#pragma unroll
      for (int a2 = 0; a2 < D; ++a2) {
        double s = 0.0;
#pragma unroll
        for (int b = 0; b < D; ++b) s += K[a1][b] * K[a2][b];
        KK[a1][a2] = s;
      }
#pragma unroll
    for (int b1 = 0; b1 < D; ++b1)
#pragma unroll
      for (int b2 = 0; b2 < D; ++b2)
#pragma unroll
        for (int a1 = 0; a1 < D; ++a1)
#pragma unroll
          for (int a2 = 0; a2 < D; ++a2) {
            double g = mu * K[a1][b2] * K[a2][b1] + lambda * K[a1][b1] * K[a2][b2];
            if (b1 == b2) g += mu * KK[a1][a2];
            store(((b1 * D + b2) * D + a1) * D + a2, det * g);
          }
  }
}

}  // namespace ffc

namespace ffc {

// G_K in the CUDA-core kernels' layout (nalpha_k entries): the symmetric Poisson G once
// per pair a1 <= a2, every other form as geometry_tensor.
template <int D, int FORM, int Q, typename Store>
__device__ __forceinline__ void geometry_tensor_k(const double K[D][D], double det, const double* w, double mu,
                                                  double lambda, Store&& store) {
  if constexpr (FORM == FFC_POISSON) {
#pragma unroll
    for (int a1 = 0; a1 < D; ++a1)
#pragma unroll
      for (int a2 = a1; a2 < D; ++a2) {
        double s = 0.0;
#pragma unroll
        for (int b = 0; b < D; ++b) s += K[a1][b] * K[a2][b];
        store(sym_pair_index<D>(a1, a2), det * s);
      }
  } else {
    geometry_tensor<D, FORM, Q>(K, det, w, mu, lambda, store);
  }
}

// G_K in FP32 from the FP32 inverse of cell_geometry_f32 (K, |det J|), for the FP32
// CUDA-core and the tensor-core contractions, which round G_K to FP32 (or to its operand
// parts) anyway. SYM: the Poisson G in the CUDA-core kernels' symmetric layout.
// `w` (convection only) is the cell's coefficient vector.
template <int D, int FORM, int Q, bool SYM>
__device__ __forceinline__ void geometry_tensor_f32(const float K[D][D], float det, const double* w, double mu,
                                                    double lambda, float* g) {
  if constexpr (FORM == FFC_MASS || FORM == FFC_SOURCE) {
    g[0] = det;
  } else if constexpr (FORM == FFC_POISSON) {
#pragma unroll
    for (int a1 = 0; a1 < D; ++a1)
#pragma unroll
      for (int a2 = SYM ? a1 : 0; a2 < D; ++a2) {
        float s = 0.f;
#pragma unroll
        for (int b = 0; b < D; ++b) s = fmaf(K[a1][b], K[a2][b], s);
        g[SYM ? sym_pair_index<D>(a1, a2) : a1 * D + a2] = det * s;
      }
  } else if constexpr (FORM == FFC_NS_CONVECTION) {
    constexpr int NS = nscalar(D, Q);
#pragma unroll
    for (int ct = 0; ct < D; ++ct)
#pragma unroll
      for (int st = 0; st < NS; ++st) {
        const int t = ct * NS + st;
        const float dw = det * float(w[t]);
#pragma unroll
        for (int a = 0; a < D; ++a) g[t * D + a] = dw * K[a][ct];
      }
  } else {
    float KK[D][D];
#pragma unroll
    for (int a1 = 0; a1 < D; ++a1)
#pragma unroll
      for (int a2 = 0; a2 < D; ++a2) {
        float s = 0.f;
#pragma unroll
        for (int b = 0; b < D; ++b) s = fmaf(K[a1][b], K[a2][b], s);
        KK[a1][a2] = s;
      }
    const float muf = float(mu), lf = float(lambda);
#pragma unroll
    for (int b1 = 0; b1 < D; ++b1)
#pragma unroll
      for (int b2 = 0; b2 < D; ++b2)
#pragma unroll
        for (int a1 = 0; a1 < D; ++a1)
#pragma unroll
          for (int a2 = 0; a2 < D; ++a2) {
            float v = muf * K[a1][b2] * K[a2][b1] + lf * K[a1][b1] * K[a2][b2];
            if (b1 == b2) v += muf * KK[a1][a2];
            g[((b1 * D + b2) * D + a1) * D + a2] = det * v;
          }
  }
}

}  // namespace ffc
