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
// Kernel: a register-tiled GEMM, C[cell][entry] = sum_j G~[cell][j] A~0[j][entry], over
// tiles of MC cells per CTA (persistent; 32 cells for FP32, 16 for FP64). Per tile: the
// cells' geometry nodes relative to each cell's node 0 (differences in FP64, then rounded
// to the contraction's type, so F' keeps that type's relative precision); G~ for every
// (cell, point) in the contraction's type (F', its determinant and adjugate, one
// reciprocal), stored K-major ([j][cell]); then, for each block of 128 entries (FP64: 64),
// the K dimension in chunks of 32 rows of A~0 (stored transposed, [K][entries padded to
// 16 bytes]) staged by cp.async into a double buffer. Warp w owns cells 4w..4w+3 (FP64: 2w, 2w+1) and lane l entries 4l..4l+3
// of the block (FP64: 2l, 2l+1): each K step is one 16-byte shared load of G~ (a broadcast
// within the warp), one of A~0 and 16 (4) FMAs into registers. The FP64 kernels compute the
// entries i1 <= i2 of these symmetric forms and store both (i1, i2) and (i2, i1); the
// FP32 ones all entries, four consecutive per 16-byte store where the row allows it.
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
    double* at_f64 = nullptr;  // [K][ne64], entries i1 <= i2, padded to an even count
    float* at_f32 = nullptr;   // [K][ne32], all entries, padded to a multiple of 4
    double* dgeo = nullptr;
    uint16_t* epair = nullptr;  // [n(n+1)/2]: i1 << 8 | i2
  };
  std::mutex lock;
  std::map<int, Dev> dev;
};

namespace ffc {
namespace {

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
    const int ns_pad = (ns + 1) / 2 * 2, nn_pad = (nn + 3) / 4 * 4;
    std::vector<double> a64(size_t(K) * ns_pad, 0.0);
    std::vector<float> a32(size_t(K) * nn_pad, 0.0f);
    std::vector<uint16_t> ep(ns);
    int u = 0;
    for (int i1 = 0; i1 < n; ++i1)
      for (int i2 = i1; i2 < n; ++i2, ++u) {
        ep[u] = uint16_t((i1 << 8) | i2);
        for (int j = 0; j < K; ++j) a64[size_t(j) * ns_pad + u] = f->At[(size_t(i1) * n + i2) * K + j];
      }
    for (int i = 0; i < nn; ++i)
      for (int j = 0; j < K; ++j) a32[size_t(j) * nn_pad + i] = float(f->At[size_t(i) * K + j]);
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
  int n, nn, ne, ne_pad, ngeo, nq, K;
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

template <int D, typename T>
__device__ __forceinline__ T det_adj(const T (&J)[D][D], T (&A)[D][D]) {
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

__device__ __forceinline__ void q_cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void q_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void q_cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void q_cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename T>
struct QTile {
  static constexpr int TM = sizeof(T) == 4 ? 4 : 2;  // cells of a thread (one warp's cells)
  static constexpr int TN = sizeof(T) == 4 ? 4 : 2;  // entries of a thread (FP64: short symmetric
                                                     // rows keep the lanes busy)
  static constexpr int MC = 8 * TM;                 // cells of a tile (8 warps)
  static constexpr int NB = 32 * TN;                // entries of a block (32 lanes)
  static constexpr int KC = 32;                     // rows of A~0 per staged chunk
};

// shared memory of one CTA: geometry gradients, node coordinates, G~ [K][MC] and the
// double-buffered A~0 chunk [2][KC][NB]
// shared memory of one CTA: geometry gradients [nq][ngeo][D] (T), node coordinates
// relative to node 0 [MC][ngeo][D] (T), the cells' h^D [MC] (double), G~ [K][MC] (T) and the
// double-buffered A~0 chunk [2][KC][NB] (T), each part 16-byte aligned
template <int D, typename T>
__host__ __device__ inline size_t quad_smem_bytes(int nq, int ngeo, int K) {
  using Q = QTile<T>;
  auto al = [](size_t b) { return (b + 15) / 16 * 16; };
  return al(size_t(nq) * ngeo * D * sizeof(T)) + al(size_t(Q::MC) * ngeo * D * sizeof(T)) + al(size_t(Q::MC) * 8) +
         al(size_t(K) * Q::MC * sizeof(T)) + size_t(2) * Q::KC * Q::NB * sizeof(T);
}

template <int D, int FORM, typename T, bool ASM, bool SYMM>
__global__ void __launch_bounds__(QT_THREADS) quad_kernel(QParams p) {
  using Q = QTile<T>;
  constexpr int NG = FORM == FFC_MASS ? 1 : D * (D + 1) / 2;
  constexpr int TM = Q::TM, TN = Q::TN, MC = Q::MC, NB = Q::NB, KC = Q::KC;
  extern __shared__ __align__(16) unsigned char smem[];
  auto al = [](size_t x) { return (x + 15) / 16 * 16; };
  T* dg = reinterpret_cast<T*>(smem);                                                      // [nq][ngeo][D]
  T* xs = reinterpret_cast<T*>(smem + al(size_t(p.nq) * p.ngeo * D * sizeof(T)));          // [MC][ngeo][D]
  double* hd = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(xs) + al(size_t(MC) * p.ngeo * D * sizeof(T)));
  T* gt = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(hd) + al(size_t(MC) * 8));  // [K][MC]
  T* ab = gt + size_t(p.K) * MC;                                                           // [2][KC][NB]
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, K = p.K, ngeo = p.ngeo;
  for (int i = t; i < p.nq * ngeo * D; i += QT_THREADS) dg[i] = T(p.dgeo[i]);
  const T* At = static_cast<const T*>(p.At);
  const long long n_tiles = (p.n_elem + MC - 1) / MC;
  const int n_kc = (K + KC - 1) / KC;
  bool bad_node = false, degenerate = false;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long long c0 = tile * MC;
    const int cells_here = int(min((long long)MC, p.n_elem - c0));
    __syncthreads();  // the previous tile's G~ and nodes are no longer read
    // node coordinates relative to the cell's node 0, in FP64 then rounded to T (the
    // differences are of the cell's size, so F' keeps T's relative precision), and the
    // cell's h^D (h the largest distance from node 0 to the other vertices) in FP64
    for (int e = w; e < MC; e += QT_THREADS / 32) {
      long long id0 = 0;
      if (e < cells_here) {
        id0 = p.cells[(c0 + e) * ngeo];
        if (id0 < 0 || id0 >= p.n_nodes) {
          bad_node = true;
          id0 = 0;
        }
      }
      double h2 = 0.0;
      for (int nd = lane; nd < ngeo; nd += 32) {
        long long id = id0;
        if (e < cells_here) {
          id = p.cells[(c0 + e) * ngeo + nd];
          if (id < 0 || id >= p.n_nodes) {
            bad_node = true;
            id = id0;
          }
        }
        double sq = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const double dx = p.nodes[id * D + a] - p.nodes[id0 * D + a];
          xs[(e * ngeo + nd) * D + a] = T(dx);
          sq = fma(dx, dx, sq);
        }
        if (nd >= 1 && nd <= D) h2 = fmax(h2, sq);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) h2 = fmax(h2, __shfl_xor_sync(0xffffffffu, h2, o));
      if (lane == 0) hd[e] = D == 2 ? h2 : h2 * sqrt(h2);
    }
    __syncthreads();
    for (int idx = t; idx < MC * p.nq; idx += QT_THREADS) {
      const int k = idx / MC, e = idx - k * MC;
      T* gout = gt + size_t(k) * NG * MC + e;  // G~[(k, g)][e]
      if (e >= cells_here) {
#pragma unroll
        for (int g = 0; g < NG; ++g) gout[g * MC] = T(0);
        continue;
      }
      const T* xe = xs + e * ngeo * D;
      const T* dk = dg + size_t(k) * ngeo * D;
      T J[D][D];
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) J[a][b] = T(0);
      for (int nd = 1; nd < ngeo; ++nd)  // node 0 is the origin of the relative coordinates
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b) J[a][b] = fma(xe[nd * D + a], dk[nd * D + b], J[a][b]);
      T A[D][D];
      const T det = det_adj<D, T>(J, A);
      if (!(fabs(double(det)) > 1e-14 * hd[e])) degenerate = true;
      const T ad = fabs(det);
      if constexpr (FORM == FFC_MASS) {
        gout[0] = ad;
      } else {
        // |det| (F'^-1 F'^-T)[a][b] = (adj adj^T)[a][b] / |det|
        const T r = T(1) / ad;
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = a; b < D; ++b) {
            T sq = T(0);
#pragma unroll
            for (int c = 0; c < D; ++c) sq = fma(A[a][c], A[b][c], sq);
            gout[qsym<D>(a, b) * MC] = sq * r;
          }
      }
    }
    // entry blocks of NB: lane l takes entries nb + 4l .. nb + 4l + 3, warp w cells TM w ..
    for (int nb = 0; nb < p.ne; nb += NB) {
      const int nbw = min(NB, p.ne_pad - nb);  // staged width (a multiple of 16 bytes)
      auto stage = [&](int kc, int buf) {
        const int rows = min(KC, K - kc * KC);
        constexpr int V = 16 / int(sizeof(T));  // values of one 16-byte copy
        const int per_row = nbw / V;
        T* dst = ab + size_t(buf) * KC * NB;
        for (int c = t; c < rows * per_row; c += QT_THREADS) {
          const int r = c / per_row, x = (c - r * per_row) * V;
          q_cp_async16(dst + r * NB + x, At + size_t(kc * KC + r) * p.ne_pad + nb + x);
        }
        q_cp_commit();
      };
      T acc[TM][TN];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
      __syncthreads();  // G~ written; the A~0 buffers free
      stage(0, 0);
      for (int kc = 0; kc < n_kc; ++kc) {
        if (kc + 1 < n_kc) {
          stage(kc + 1, (kc + 1) & 1);
          q_cp_wait1();
        } else {
          q_cp_wait0();
        }
        __syncthreads();
        const T* a = ab + size_t(kc & 1) * KC * NB + TN * lane;
        const T* g = gt + size_t(kc) * KC * MC + TM * w;
        const int rows = min(KC, K - kc * KC);
        for (int r = 0; r < rows; ++r) {
          T av[TN], gv[TM];
          if constexpr (sizeof(T) == 4) {
            const float4 x = *reinterpret_cast<const float4*>(a + r * NB);
            av[0] = x.x, av[1] = x.y, av[2] = x.z, av[3] = x.w;
            const float4 y = *reinterpret_cast<const float4*>(g + r * MC);
            gv[0] = y.x, gv[1] = y.y, gv[2] = y.z, gv[3] = y.w;
          } else {
            const double2 x0 = *reinterpret_cast<const double2*>(a + r * NB);
            av[0] = x0.x, av[1] = x0.y;
            const double2 y = *reinterpret_cast<const double2*>(g + r * MC);
            gv[0] = y.x, gv[1] = y.y;
          }
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = fma(gv[i], av[j], acc[i][j]);
        }
        __syncthreads();  // this buffer is staged again two chunks later
      }
      // results: cells c0 + TM w + i, entries nb + TN lane + j
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int e = TM * w + i;
        if (e >= cells_here) break;
        const long long cell = c0 + e;
        const int u0 = nb + TN * lane;
        if constexpr (!ASM && !SYMM) {
          T* o = static_cast<T*>(p.out) + cell * p.nn;
          if (u0 + TN <= p.ne && (p.nn % 4) == 0) {
            *reinterpret_cast<float4*>(o + u0) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            continue;
          }
        }
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          const int u = u0 + j;
          if (u >= p.ne) break;
          int i1, i2;
          if constexpr (SYMM) {
            const unsigned ep = p.epair[u];
            i1 = int(ep >> 8);
            i2 = int(ep & 255u);
          } else {
            i1 = u / p.n;
            i2 = u - i1 * p.n;
          }
          if constexpr (ASM) {
            double* csr = static_cast<double*>(p.out);
            const long long s1 = p.slot[cell * p.nn + i1 * p.n + i2];
            if (s1 >= 0 && s1 < p.nnz) atomicAdd(csr + s1, double(acc[i][j]));
            else bad_node = true;
            if (SYMM && i1 != i2) {
              const long long s2 = p.slot[cell * p.nn + i2 * p.n + i1];
              if (s2 >= 0 && s2 < p.nnz) atomicAdd(csr + s2, double(acc[i][j]));
              else bad_node = true;
            }
          } else {
            T* o = static_cast<T*>(p.out) + cell * p.nn;
            o[i1 * p.n + i2] = acc[i][j];
            if (SYMM && i1 != i2) o[i2 * p.n + i1] = acc[i][j];
          }
        }
      }
    }
  }
  if (bad_node) atomicOr(p.status, FFC_FLAG_BOUNDS);
  if (degenerate) atomicOr(p.status, FFC_FLAG_DEGENERATE);
}

template <int D, int FORM, typename T, bool ASM, bool SYMM>
int launch_quad(const QParams& prm, cudaStream_t s) {
  const size_t smem = quad_smem_bytes<D, T>(prm.nq, prm.ngeo, prm.K);
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
  const long long tiles = (prm.n_elem + QTile<T>::MC - 1) / QTile<T>::MC;
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
  const int ne = fp64 ? f->n * (f->n + 1) / 2 : f->n * f->n;
  QParams prm{f->n,          f->n * f->n, ne, fp64 ? (ne + 1) / 2 * 2 : (ne + 3) / 4 * 4,
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
