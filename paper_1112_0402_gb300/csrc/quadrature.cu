// Quadrature as a tensor contraction (Section 3.4, "Curvilinear elements").
//
// On a cell whose map F_K from the reference simplex is not affine, the Jacobian varies
// inside the cell and cannot be taken out of the integral. Summing over the points X_k of
// a quadrature rule instead keeps the element tensor a contraction, now with one more
// index: A^K[i] ~= sum_j A~0[i][j] G~_K[j], j = (point k, geometry entry g), where A~0
// holds the weighted reference basis products at the points (computed once, on the host)
// and G~_K the per-point Jacobian factors of the cell (computed here, per cell and point):
//   mass     G~_K[k]       = |det F'(X_k)|
//   Poisson  G~_K[(k, g)]  = |det F'(X_k)| (F'^-1 F'^-T)[a][b](X_k), g = (a <= b)
// The map is the geometry interpolant F_K(X) = sum_n x_n Psi_n(X) of degree 1 or 2 over the
// cell's geometry nodes, so F'(X_k) = sum_n x_n grad Psi_n(X_k)^T with the gradients of
// the geometry basis at the points tabulated on the host.
//
// Kernel: tiles of 16 cells per CTA (persistent). Phase 1 loads the tile's node
// coordinates; phase 2 computes G~ for every (cell, point) in FP64 (F', its determinant
// and adjugate) into shared memory, rounded to the contraction's type; phase 3 contracts:
// a thread item is one element-tensor entry for 8 cells, streaming the entry's row of
// A~0 (stored transposed, [K][entries], so a warp's loads are consecutive) against the 8
// cells' G~ (shared-memory broadcasts). The FP64 kernels compute the entries i1 <= i2 of
// these symmetric forms and store both (i1, i2) and (i2, i1); the FP32 ones all entries.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ffc_internal.h"

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
    double* at_f64 = nullptr;  // [K][n(n+1)/2], entries i1 <= i2
    float* at_f32 = nullptr;   // [K][n*n]
    double* dgeo = nullptr;
    uint16_t* epair = nullptr;  // [n(n+1)/2]: i1 << 8 | i2
  };
  std::mutex lock;
  std::map<int, Dev> dev;
};

namespace ffc {
namespace {

constexpr int QT_CELLS = 16;  // cells of one tile
constexpr int QT_GROUP = 8;   // cells of one thread item
constexpr int QT_THREADS = 256;

int cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return FFC_ECUDA;
}

int compile_qform(ffc_qform* f) {
  const int d = f->d;
  reference_rule(d, f->p, f->X, f->W);
  f->nq = int(f->W.size());
  std::vector<double> psi, dpsi, gpsi;
  reference_basis(d, f->q, f->X, psi, dpsi);
  reference_basis(d, f->g, f->X, gpsi, f->dgeo);
  f->n = n_scalar_local(d, f->q);
  f->ngeo = n_scalar_local(d, f->g);
  f->ng = f->kind == FFC_MASS ? 1 : d * (d + 1) / 2;
  f->K = f->nq * f->ng;
  const int n = f->n, nq = f->nq, ng = f->ng, K = f->K;
  f->At.assign(size_t(n) * n * K, 0.0);
  for (int i1 = 0; i1 < n; ++i1)
    for (int i2 = 0; i2 < n; ++i2) {
      double* row = f->At.data() + (size_t(i1) * n + i2) * K;
      for (int k = 0; k < nq; ++k) {
        const double w = f->W[k];
        if (f->kind == FFC_MASS) {
          row[k] = w * psi[size_t(k) * n + i1] * psi[size_t(k) * n + i2];
        } else {
          const double* g1 = dpsi.data() + (size_t(k) * n + i1) * d;
          const double* g2 = dpsi.data() + (size_t(k) * n + i2) * d;
          for (int a = 0; a < d; ++a)
            for (int b = a; b < d; ++b) {
              const double v = g1[a] * g2[b] + (a != b ? g1[b] * g2[a] : 0.0);
              row[k * ng + sym_pair(d, a, b)] = w * v;
            }
        }
      }
    }
  return FFC_OK;
}

int ensure_qdev(ffc_qform* f, ffc_qform::Dev** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "ffc_qform");
  std::lock_guard<std::mutex> g(f->lock);
  ffc_qform::Dev& D = f->dev[dev];
  if (!D.at_f64) {
    const int n = f->n, K = f->K, nn = n * n, ns = n * (n + 1) / 2;
    std::vector<double> a64(size_t(K) * ns);
    std::vector<float> a32(size_t(K) * nn);
    std::vector<uint16_t> ep(ns);
    int u = 0;
    for (int i1 = 0; i1 < n; ++i1)
      for (int i2 = i1; i2 < n; ++i2, ++u) {
        ep[u] = uint16_t((i1 << 8) | i2);
        for (int j = 0; j < K; ++j) a64[size_t(j) * ns + u] = f->At[(size_t(i1) * n + i2) * K + j];
      }
    for (int i = 0; i < nn; ++i)
      for (int j = 0; j < K; ++j) a32[size_t(j) * nn + i] = float(f->At[size_t(i) * K + j]);
    ffc_qform::Dev t;
    if ((e = cudaMalloc(&t.at_f64, a64.size() * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&t.at_f32, a32.size() * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&t.dgeo, f->dgeo.size() * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&t.epair, ep.size() * sizeof(uint16_t))) != cudaSuccess ||
        (e = cudaMemcpy(t.at_f64, a64.data(), a64.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(t.at_f32, a32.data(), a32.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(t.dgeo, f->dgeo.data(), f->dgeo.size() * sizeof(double), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(t.epair, ep.data(), ep.size() * sizeof(uint16_t), cudaMemcpyHostToDevice)) != cudaSuccess) {
      cudaFree(t.at_f64);
      cudaFree(t.at_f32);
      cudaFree(t.dgeo);
      cudaFree(t.epair);
      return cuda_fail(e, "ffc_qform device copy");
    }
    D = t;
  }
  *out = &D;
  return FFC_OK;
}

struct QParams {
  int n, nn, ne, ngeo, nq, K;
  long long n_elem, n_nodes, nnz;
  const int32_t* cells;
  const double* nodes;
  const void* At;  // [K][ne]
  const double* dgeo;
  const uint16_t* epair;
  void* out;  // A_K (T) or CSR values (double)
  const int32_t* slot;
  unsigned* status;
};

template <int D>
__device__ __forceinline__ double det_adj(const double (&J)[D][D], double (&A)[D][D]) {
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

// column of the pair (a <= b): diagonal pairs first, then (0,1) [, (0,2), (1,2)]
template <int D>
__device__ __forceinline__ int qsym(int a, int b) {
  return a == b ? a : (D == 2 ? 2 : (a == 0 ? (b == 1 ? 3 : 4) : 5));
}

template <int D, int FORM, typename T, bool ASM, bool SYMM>
__global__ void __launch_bounds__(QT_THREADS) quad_kernel(QParams p) {
  constexpr int NG = FORM == FFC_MASS ? 1 : D * (D + 1) / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  double* dg = reinterpret_cast<double*>(smem);           // [nq][ngeo][D]
  double* xs = dg + size_t(p.nq) * p.ngeo * D;            // [QT_CELLS][ngeo][D]
  T* gt = reinterpret_cast<T*>(xs + QT_CELLS * p.ngeo * D);  // [QT_CELLS][K]
  const int t = threadIdx.x, K = p.K, ngeo = p.ngeo;
  for (int i = t; i < p.nq * ngeo * D; i += QT_THREADS) dg[i] = p.dgeo[i];
  const long long n_tiles = (p.n_elem + QT_CELLS - 1) / QT_CELLS;
  bool bad_node = false, degenerate = false;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long long c0 = tile * QT_CELLS;
    const int cells_here = int(min((long long)QT_CELLS, p.n_elem - c0));
    __syncthreads();  // the previous tile's G~ and nodes are no longer read
    for (int idx = t; idx < QT_CELLS * ngeo; idx += QT_THREADS) {
      const int e = idx / ngeo, nd = idx - e * ngeo;
      long long id = 0;
      if (e < cells_here) {
        id = p.cells[(c0 + e) * ngeo + nd];
        if (id < 0 || id >= p.n_nodes) {
          bad_node = true;
          id = 0;
        }
      }
#pragma unroll
      for (int a = 0; a < D; ++a) xs[idx * D + a] = p.nodes[id * D + a];
    }
    __syncthreads();
    for (int idx = t; idx < QT_CELLS * p.nq; idx += QT_THREADS) {
      const int e = idx / p.nq, k = idx - e * p.nq;
      T* gout = gt + size_t(e) * K + k * NG;
      if (e >= cells_here) {
#pragma unroll
        for (int g = 0; g < NG; ++g) gout[g] = T(0);
        continue;
      }
      const double* xe = xs + e * ngeo * D;
      const double* dk = dg + size_t(k) * ngeo * D;
      double J[D][D];
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) J[a][b] = 0.0;
      for (int nd = 0; nd < ngeo; ++nd)
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b) J[a][b] = fma(xe[nd * D + a], dk[nd * D + b], J[a][b]);
      double A[D][D];
      const double det = det_adj<D>(J, A);
      // cell size: the largest distance from vertex node 0 to the other vertex nodes
      double h2 = 0.0;
      for (int v = 1; v <= D; ++v) {
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const double dx = xe[v * D + a] - xe[a];
          s = fma(dx, dx, s);
        }
        h2 = fmax(h2, s);
      }
      const double hd = D == 2 ? h2 : h2 * sqrt(h2);
      if (!(fabs(det) > 1e-14 * hd)) degenerate = true;
      const double ad = fabs(det);
      if constexpr (FORM == FFC_MASS) {
        gout[0] = T(ad);
      } else {
        // |det| (F'^-1 F'^-T)[a][b] = (adj adj^T)[a][b] / |det|
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = a; b < D; ++b) {
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < D; ++c) s = fma(A[a][c], A[b][c], s);
            gout[qsym<D>(a, b)] = T(s / ad);
          }
      }
    }
    __syncthreads();
    const T* At = static_cast<const T*>(p.At);
    for (int item = t; item < p.ne * (QT_CELLS / QT_GROUP); item += QT_THREADS) {
      const int u = item % p.ne, cg = item / p.ne;
      if (cg * QT_GROUP >= cells_here) continue;
      T acc[QT_GROUP];
#pragma unroll
      for (int c = 0; c < QT_GROUP; ++c) acc[c] = T(0);
      const T* a = At + u;
      const T* g = gt + size_t(cg) * QT_GROUP * K;
      for (int j = 0; j < K; ++j) {
        const T av = __ldg(a + size_t(j) * p.ne);
#pragma unroll
        for (int c = 0; c < QT_GROUP; ++c) acc[c] = fma(av, g[c * K + j], acc[c]);
      }
      int i1, i2;
      if constexpr (SYMM) {
        const unsigned ep = p.epair[u];
        i1 = int(ep >> 8);
        i2 = int(ep & 255u);
      } else {
        i1 = u / p.n;
        i2 = u - i1 * p.n;
      }
#pragma unroll
      for (int c = 0; c < QT_GROUP; ++c) {
        const int e = cg * QT_GROUP + c;
        if (e >= cells_here) break;
        const long long cell = c0 + e;
        if constexpr (ASM) {
          double* csr = static_cast<double*>(p.out);
          const long long s1 = p.slot[cell * p.nn + i1 * p.n + i2];
          if (s1 >= 0 && s1 < p.nnz) atomicAdd(csr + s1, double(acc[c]));
          else bad_node = true;
          if (SYMM && i1 != i2) {
            const long long s2 = p.slot[cell * p.nn + i2 * p.n + i1];
            if (s2 >= 0 && s2 < p.nnz) atomicAdd(csr + s2, double(acc[c]));
            else bad_node = true;
          }
        } else {
          T* o = static_cast<T*>(p.out) + cell * p.nn;
          o[i1 * p.n + i2] = acc[c];
          if (SYMM && i1 != i2) o[i2 * p.n + i1] = acc[c];
        }
      }
    }
  }
  if (bad_node) atomicOr(p.status, FFC_FLAG_BOUNDS);
  if (degenerate) atomicOr(p.status, FFC_FLAG_DEGENERATE);
}

template <int D, int FORM, typename T, bool ASM, bool SYMM>
int launch_quad(const QParams& prm, cudaStream_t s) {
  const size_t smem = size_t(prm.nq) * prm.ngeo * D * sizeof(double) + size_t(QT_CELLS) * prm.ngeo * D * sizeof(double) +
                      size_t(QT_CELLS) * prm.K * sizeof(T);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > size_t(optin)) {
    set_error("ffc_tabulate_quadrature: the rule is too large for one tile in shared memory (" +
              std::to_string(smem) + " bytes)");
    return FFC_EINVAL;
  }
  auto kern = quad_kernel<D, FORM, T, ASM, SYMM>;
  int sms = 0, per_sm = 1;
  if (launch_config(reinterpret_cast<const void*>(kern), QT_THREADS, smem, -1, &sms, &per_sm) != FFC_OK)
    return FFC_ECUDA;
  const long long tiles = (prm.n_elem + QT_CELLS - 1) / QT_CELLS;
  long long blocks = std::min<long long>(tiles, (long long)sms * std::max(per_sm, 1));
  kern<<<unsigned(std::max<long long>(blocks, 1)), QT_THREADS, smem, s>>>(prm);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FFC_OK : cuda_fail(e, "quad_kernel launch");
}

template <int D, int FORM>
int launch_quad_prec(const QParams& prm, int precision, bool assemble, cudaStream_t s) {
  if (precision == FFC_FP64)
    return assemble ? launch_quad<D, FORM, double, true, true>(prm, s) : launch_quad<D, FORM, double, false, true>(prm, s);
  return assemble ? launch_quad<D, FORM, float, true, false>(prm, s) : launch_quad<D, FORM, float, false, false>(prm, s);
}

int run_quadrature(const ffc_qform* f, int64_t n_elem, const int32_t* cells, const double* nodes, int64_t n_nodes,
                   void* out, const int32_t* slot, int64_t nnz, int precision, void* stream, const char* who) {
  ffc_qform::Dev* dv = nullptr;
  int rc = ensure_qdev(const_cast<ffc_qform*>(f), &dv);
  if (rc != FFC_OK) return rc;
  unsigned* st = status_word();
  if (!st) {
    set_error(std::string(who) + ": status word allocation failed");
    return FFC_ECUDA;
  }
  const bool fp64 = precision == FFC_FP64;
  QParams prm{f->n,          f->n * f->n, fp64 ? f->n * (f->n + 1) / 2 : f->n * f->n,
              f->ngeo,       f->nq,       f->K,
              n_elem,        n_nodes,     nnz,
              cells,
              nodes,         fp64 ? static_cast<const void*>(dv->at_f64) : static_cast<const void*>(dv->at_f32),
              dv->dgeo,      dv->epair,   out,
              slot,          st};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool asm_ = slot != nullptr;
  if (f->d == 2)
    return f->kind == FFC_MASS ? launch_quad_prec<2, FFC_MASS>(prm, precision, asm_, s)
                               : launch_quad_prec<2, FFC_POISSON>(prm, precision, asm_, s);
  return f->kind == FFC_MASS ? launch_quad_prec<3, FFC_MASS>(prm, precision, asm_, s)
                             : launch_quad_prec<3, FFC_POISSON>(prm, precision, asm_, s);
}

int check_args(const ffc_qform* f, int64_t n_elem, const int32_t* cells, const double* nodes, int64_t n_nodes,
               int precision, const char* who) {
  if (!f || n_elem < 0 || n_nodes < 0 || (precision != FFC_FP64 && precision != FFC_FP32)) {
    set_error(std::string(who) + ": invalid argument (precision must be FFC_FP64 or FFC_FP32)");
    return FFC_EINVAL;
  }
  if (n_elem > 0 && (!cells || !nodes || n_nodes == 0 || (reinterpret_cast<uintptr_t>(nodes) & 7))) {
    set_error(std::string(who) + ": null or misaligned cells / nodes");
    return FFC_EINVAL;
  }
  return FFC_OK;
}

}  // namespace
}  // namespace ffc

using namespace ffc;

extern "C" int ffc_qform_create(int form, int cell, int degree, int geometry_degree, int quad_degree,
                                ffc_qform** out) {
  if (!out || (form != FFC_MASS && form != FFC_POISSON) || (cell != FFC_TRIANGLE && cell != FFC_TETRAHEDRON) ||
      degree < 1 || degree > 4 || geometry_degree < 1 || geometry_degree > 2 || quad_degree < 0 || quad_degree > 20) {
    set_error("ffc_qform_create: form MASS or POISSON, cell TRIANGLE or TETRAHEDRON, degree 1..4, geometry degree "
              "1..2, quadrature degree 0..20");
    return FFC_EINVAL;
  }
  auto* f = new ffc_qform;
  f->kind = form;
  f->d = cell == FFC_TRIANGLE ? 2 : 3;
  f->q = degree;
  f->g = geometry_degree;
  f->p = quad_degree;
  const int rc = compile_qform(f);
  if (rc != FFC_OK) {
    delete f;
    return rc;
  }
  *out = f;
  return FFC_OK;
}

extern "C" int ffc_qform_info(const ffc_qform* f, int* n_local, int* n_geometry, int* n_points, int* k_contract) {
  if (!f) return FFC_EINVAL;
  if (n_local) *n_local = f->n;
  if (n_geometry) *n_geometry = f->ngeo;
  if (n_points) *n_points = f->nq;
  if (k_contract) *k_contract = f->K;
  return FFC_OK;
}

extern "C" int ffc_qform_reference_tensor(const ffc_qform* f, double* out) {
  if (!f || !out) return FFC_EINVAL;
  std::copy(f->At.begin(), f->At.end(), out);
  return FFC_OK;
}

extern "C" int ffc_qform_rule(const ffc_qform* f, double* points, double* weights) {
  if (!f) return FFC_EINVAL;
  if (points) std::copy(f->X.begin(), f->X.end(), points);
  if (weights) std::copy(f->W.begin(), f->W.end(), weights);
  return FFC_OK;
}

extern "C" void ffc_qform_destroy(ffc_qform* f) {
  if (!f) return;
  for (auto& kv : f->dev) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(kv.first);
    cudaFree(kv.second.at_f64);
    cudaFree(kv.second.at_f32);
    cudaFree(kv.second.dgeo);
    cudaFree(kv.second.epair);
    cudaSetDevice(prev);
  }
  delete f;
}

extern "C" int ffc_tabulate_quadrature(const ffc_qform* f, int64_t n_elem, const int32_t* cells, const double* nodes,
                                       int64_t n_nodes, void* A_K, int precision, void* stream) {
  int rc = check_args(f, n_elem, cells, nodes, n_nodes, precision, "ffc_tabulate_quadrature");
  if (rc != FFC_OK || n_elem == 0) return rc;
  if (!A_K || (reinterpret_cast<uintptr_t>(A_K) & 15)) {
    set_error("ffc_tabulate_quadrature: A_K null or not 16-byte aligned");
    return FFC_EINVAL;
  }
  return run_quadrature(f, n_elem, cells, nodes, n_nodes, A_K, nullptr, 0, precision, stream,
                        "ffc_tabulate_quadrature");
}

extern "C" int ffc_assemble_quadrature(const ffc_qform* f, int64_t n_elem, const int32_t* cells, const double* nodes,
                                       int64_t n_nodes, const int32_t* slot, double* csr_val, int64_t nnz,
                                       int precision, void* stream) {
  int rc = check_args(f, n_elem, cells, nodes, n_nodes, precision, "ffc_assemble_quadrature");
  if (rc != FFC_OK || n_elem == 0) return rc;
  if (!slot || !csr_val || nnz <= 0) {
    set_error("ffc_assemble_quadrature: slot / csr_val");
    return FFC_EINVAL;
  }
  return run_quadrature(f, n_elem, cells, nodes, n_nodes, csr_val, slot, nnz, precision, stream,
                        "ffc_assemble_quadrature");
}
