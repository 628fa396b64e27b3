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
#include "quadrature.h"
#include "tc_common.cuh"


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

using quad::det_adj;

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
            gout[quad::qpair<D>(a, b) * MC] = sq * r;
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

// ------------------------------------------------------------------ tensor cores
// The same contraction on tcgen05 for forms whose element tensor fits one M-tile (at most
// 128 entries: P1 and P2), D[i][e] = sum_j A~0[i][j] G~[e][j] with M = entries, N = 128
// cells, K = points x geometry entries, in K chunks of 48 columns (8 points of the 3D
// Poisson form): both operands are streamed per chunk. A~0 is split on the host into
// TF32 or BF16 parts and laid out per chunk in the K-major core-matrix layout, one 1-D
// bulk copy per part; G~ is produced per chunk by four warps (one cell per thread: F'
// at the chunk's points in FP32 from FP64 node differences, its determinant and adjugate,
// split into the same parts) into a second ring. One thread issues the split products
// (the correction products into their own TMEM accumulator), four warps drain TMEM to
// A_K. Warps: 0-3 producers, 4-7 drainers, 8 MMA, 9 TMA; 2 A stages, 2 B stages, two TMEM
// accumulators (cell tiles alternate). Every mbarrier wait is bounded.
namespace tq {
using namespace ffc::tc;

// The same contraction on the tensor cores (FFC_TF32 / FFC_TF32X3 / FFC_BF16X3): D[i][c] =
// sum_j A~0[i][j] (G~_c[j] - G~_c(centroid)) with M = 128 element-tensor entries per M tile
// (up to four), N = 128 cells, K = points x n_g in 48-column chunks; the operands split
// into TF32 or BF16 parts as for the tensor representation, A~0 on the host, G~ on the
// device. The drainers add the centroid term (sum_j A~0[i][j]) : G~_c in FP32, so the
// tensor cores' FP32 accumulation only carries the deviations from the centroid value.
// Warp roles: 0-7 produce the G~ chunks (two lanes per cell, each half of a chunk's
// columns), 8-11 drain TMEM into A_K (or add into CSR values), 12 issues the MMAs, 13
// streams the A~0 chunks, 14-15 gather the cells' nodes and form the per-cell Jacobian
// coefficients one tile ahead.
constexpr int QKCH = 48;  // K columns per chunk (a multiple of both MMA K steps)
constexpr int TQ_PRODUCER_WARPS = 8;
constexpr int TQ_DRAIN_WARP0 = 8, TQ_MMA_WARP = 12, TQ_TMA_WARP = 13, TQ_GEO_WARP0 = 14;
constexpr int TQ_THREADS = 512;
constexpr int TQ_GEO_THREADS = TQ_THREADS - 32 * TQ_GEO_WARP0;

template <int D, int FORM, int G, int MODE>
struct TqCfg {
  using S = Split<MODE>;
  static constexpr int NG = FORM == FFC_MASS ? 1 : D * (D + 1) / 2;
  static constexpr int PPC = QKCH / NG;                // points per chunk
  static constexpr int PPH = PPC / 2;                  // points per producer lane and chunk
  static constexpr int NGEO = G == 1 ? D + 1 : (D + 1) * (D + 2) / 2;
  // the map's Jacobian is affine in X for geometry degree 2:
  //   F'(X)[a][b] = J0[a][b] + sum_c H[a][(b,c)] X_c
  // J0 = sum_n x_n (dPsi_n/dX_b)(0), H[a][(b,c)] = sum_n x_n[a] d2Psi_n/dX_b dX_c
  static constexpr int NH = G == 2 ? D * (D + 1) / 2 : 0;
  static constexpr int NJ = D * D + D * NH;            // per-cell coefficients
  static constexpr int KCC = QKCH / S::EPC;            // core-matrix columns per chunk
  static constexpr uint32_t CH_BYTES = M_TILE * QKCH * S::ESIZE;  // one part of one chunk (A or B)
  static constexpr uint32_t STAGE_BYTES = S::PARTS * CH_BYTES;
  static constexpr int ACC_COLS = S::NPROD > 1 ? 2 * N_CELLS : N_CELLS;
  static constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;
  static_assert(QKCH % NG == 0 && QKCH % S::KSTEP == 0, "chunk width");
  static_assert(PPC % 2 == 0 && (QKCH / 2) % S::EPC == 0, "a chunk splits into two lanes' halves");
  // shared memory: A stages, B stages, the geometry table, the per-cell slot, barriers
  static constexpr size_t table_floats(int nq) { return size_t(NGEO) * D + size_t(NGEO) * NH + size_t(nq) * D; }
  static constexpr size_t off_table() { return 4 * size_t(STAGE_BYTES); }
  static constexpr size_t off_cell(int nq) { return off_table() + (table_floats(nq) * 4 + 15) / 16 * 16; }
  static constexpr size_t off_gbar(int nq) { return off_cell(nq) + size_t(NJ + 1) * N_CELLS * 4; }
  static constexpr size_t off_bars(int nq) { return off_gbar(nq) + size_t(2) * NG * N_CELLS * 4; }
  static constexpr size_t smem_bytes(int nq) { return off_bars(nq) + NBARS * 8 + 16; }
  static constexpr int NBARS = 20;
};

struct TqParams {
  const int32_t* cells;
  const double* nodes;
  long long n_nodes, n_elem;
  const float* table;       // [NGEO][D] dPsi(0), [NGEO][NH] second derivatives, [nq][D] points
  const float* a0sum;       // [nn][NG]: A~0 summed over the points (the centroid term)
  const void* a_part[3];    // [NCH][MT][128 x QKCH] per part: chunk c of M tile m at block c * MT + m
  float* out;               // A_K [n_elem][nn], or (slot set) CSR values csr_val[slot] += A_K
  const int32_t* slot;
  double* csr_val;
  long long nnz;
  int nn, nq, nch;
  int mt;                   // 128-entry M tiles (1..4)
  unsigned* status;
};

// every lane of the warp waits; the warp goes on only when all of them saw the phase
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t phase, volatile int* abort_flag) {
  const bool ok = mbar_wait_or_abort(bar, phase, abort_flag);
  return __all_sync(0xffffffffu, ok);
}

template <int D, int FORM, int G, int MODE, bool MULTI>
__global__ void __launch_bounds__(TQ_THREADS, 1) tq_kernel(TqParams p) {
  using C = TqCfg<D, FORM, G, MODE>;
  using S = Split<MODE>;
  constexpr int NG = C::NG, NGEO = C::NGEO, NH = C::NH, NJ = C::NJ;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* As = smem;                          // 2 x STAGE_BYTES
  unsigned char* Bs = smem + 2 * C::STAGE_BYTES;     // 2 x STAGE_BYTES
  float* tab = reinterpret_cast<float*>(smem + C::off_table());
  const float* g0 = tab;                             // [NGEO][D]
  const float* hs = tab + NGEO * D;                  // [NGEO][NH]
  const float* xq = hs + NGEO * NH;                  // [nq][D]
  float* cellj = reinterpret_cast<float*>(smem + C::off_cell(p.nq));  // [NJ][128], then thr [128]
  float* thr_s = cellj + NJ * N_CELLS;
  float* gbar = reinterpret_cast<float*>(smem + C::off_gbar(p.nq));  // [2][NG][128]: G~ at the centroid
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::off_bars(p.nq));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + C::NBARS);
  __shared__ int abort_flag;
  constexpr int A_FULL = 0, A_EMPTY = 2, B_FULL = 4, B_EMPTY = 6, ACC_FULL = 8, ACC_EMPTY = 10, GEO_FULL = 12,
                GEO_EMPTY = 13, GBAR_FULL = 14, GBAR_EMPTY = 16;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  auto bar = [&](int k) { return smem_u32(&bars[k]); };
  for (int i = t; i < int(C::table_floats(p.nq)); i += TQ_THREADS) tab[i] = p.table[i];
  if (t == 0) {
    for (int k = 0; k < 2; ++k) {
      mbar_init(bar(A_FULL + k), 1);
      mbar_init(bar(A_EMPTY + k), 1);
      mbar_init(bar(B_FULL + k), TQ_PRODUCER_WARPS);
      mbar_init(bar(B_EMPTY + k), 1);
      mbar_init(bar(ACC_FULL + k), 1);
      mbar_init(bar(ACC_EMPTY + k), 4);
    }
    mbar_init(bar(GEO_FULL), TQ_GEO_THREADS / 32);
    mbar_init(bar(GEO_EMPTY), TQ_PRODUCER_WARPS);
    for (int k = 0; k < 2; ++k) {
      mbar_init(bar(GBAR_FULL + k), TQ_PRODUCER_WARPS);
      mbar_init(bar(GBAR_EMPTY + k), 4);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // one M tile (MULTI false): two accumulator buffers (main and correction products apart,
  // the drain of a tile overlapping the next tile's MMAs); two to four M tiles (MULTI
  // true): one 128-column accumulator per M tile holding all the products, single-buffered
  constexpr uint32_t tmem_cols = MULTI ? 512u : C::TMEM_COLS;
  constexpr int nbuf = MULTI ? 1 : 2;
  const int mt = MULTI ? p.mt : 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const long long n_tiles = (p.n_elem + N_CELLS - 1) / N_CELLS;
  const long long my_tiles = blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int nblk = p.nch * mt;                     // A~0 blocks per cell tile
  const long long total = my_tiles * nblk;         // A~0 blocks this CTA consumes
  if (warp == TQ_TMA_WARP) {
    // ---------------------------------------------------------------- TMA: A~0 chunks
    if (lane == 0) {
      bool ok = true;
      for (long long g = 0; g < total && ok; ++g) {
        const int s = int(g & 1);
        if (g >= 2) ok = mbar_wait_or_abort(bar(A_EMPTY + s), uint32_t((g - 2) >> 1) & 1u, &abort_flag);
        if (!ok) break;
        const long long c = g % nblk;
        mbar_expect_tx(bar(A_FULL + s), C::STAGE_BYTES);
#pragma unroll
        for (int q = 0; q < S::PARTS; ++q)
          bulk_g2s(smem_u32(As + s * C::STAGE_BYTES + q * C::CH_BYTES),
                   static_cast<const unsigned char*>(p.a_part[q]) + size_t(c) * C::CH_BYTES, C::CH_BYTES,
                   bar(A_FULL + s));
      }
      if (!ok) {
        atomicOr(p.status, FFC_FLAG_TIMEOUT);
        abort_flag = 1;
      }
    }
  } else if (warp == TQ_MMA_WARP) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      constexpr uint32_t IDESC = S::idesc(M_TILE, N_CELLS);
      constexpr uint32_t SBO = C::KCC * 128;
      constexpr int KS = QKCH / S::KSTEP;
      bool ok = true;
      long long ga = 0, gb = 0;  // A~0 blocks and G~ chunks consumed
      for (long long ct = 0; ct < my_tiles && ok; ++ct) {
        const int acc = int(ct % nbuf);
        const long long use = ct / nbuf;
        if (ct >= nbuf) ok = mbar_wait_or_abort(bar(ACC_EMPTY + acc), uint32_t(use - 1) & 1u, &abort_flag);
        if (!ok) break;
        for (int c = 0; c < p.nch && ok; ++c, ++gb) {
          const int sb = int(gb & 1);
          ok = mbar_wait_or_abort(bar(B_FULL + sb), uint32_t(gb >> 1) & 1u, &abort_flag);
          for (int m = 0; m < mt && ok; ++m, ++ga) {
            const int sa = int(ga & 1);
            ok = mbar_wait_or_abort(bar(A_FULL + sa), uint32_t(ga >> 1) & 1u, &abort_flag);
            if (!ok) break;
            fence_after();
            const uint32_t d_main = tmem + uint32_t(nbuf > 1 ? acc * C::ACC_COLS : m * N_CELLS);
            const uint32_t d_corr = d_main + uint32_t(N_CELLS);
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
#pragma unroll
              for (int k = 0; k < S::NPROD; ++k) {
                const uint64_t da =
                    smem_desc(smem_u32(As + sa * C::STAGE_BYTES + S::pa(k) * C::CH_BYTES) + ks * 256, 128, SBO);
                const uint64_t db =
                    smem_desc(smem_u32(Bs + sb * C::STAGE_BYTES + S::pb(k) * C::CH_BYTES) + ks * 256, 128, SBO);
                const bool first = c == 0 && ks == 0;
                if constexpr (MULTI) mma<S::BF16>(d_main, da, db, IDESC, (first && k == 0) ? 0u : 1u);
                else if (k == S::NPROD - 1) mma<S::BF16>(d_main, da, db, IDESC, first ? 0u : 1u);
                else mma<S::BF16>(d_corr, da, db, IDESC, (first && k == 0) ? 0u : 1u);
              }
            }
            mma_commit(bar(A_EMPTY + sa));
          }
          if (ok) mma_commit(bar(B_EMPTY + sb));
        }
        if (ok) mma_commit(bar(ACC_FULL + acc));
      }
      if (!ok) {
        atomicOr(p.status, FFC_FLAG_TIMEOUT);
        abort_flag = 1;
      }
      if (ga > 0) mbar_wait(bar(A_EMPTY + int((ga - 1) & 1)), uint32_t((ga - 1) >> 1) & 1u);  // last chain done
    }
  } else if (warp >= TQ_GEO_WARP0) {
    // ---------------------------------------------------------------- per-cell geometry, one tile ahead
    const int gt = t - 32 * TQ_GEO_WARP0;
    bool ok = true;
    for (long long ct = 0; ct < my_tiles && ok; ++ct) {
#pragma unroll 1
      for (int half = 0; half < N_CELLS / TQ_GEO_THREADS; ++half) {
        const int c = gt + half * TQ_GEO_THREADS;
        const long long e = (blockIdx.x + ct * gridDim.x) * N_CELLS + c;
        const bool live = e < p.n_elem;
        // node coordinates relative to node 0: FP64 differences rounded to FP32
        float xr[NGEO][D];
        float h2 = 0.f;
        long long id0 = live ? p.cells[e * NGEO] : 0;
        if (id0 < 0 || id0 >= p.n_nodes) {
          atomicOr(p.status, FFC_FLAG_BOUNDS);
          id0 = 0;
        }
        double x0[D];
#pragma unroll
        for (int a = 0; a < D; ++a) x0[a] = p.nodes[id0 * D + a];
#pragma unroll
        for (int nd = 1; nd < NGEO; ++nd) {
          long long id = live ? p.cells[e * NGEO + nd] : id0;
          if (id < 0 || id >= p.n_nodes) {
            atomicOr(p.status, FFC_FLAG_BOUNDS);
            id = id0;
          }
          float sq = 0.f;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            xr[nd][a] = float(p.nodes[id * D + a] - x0[a]);
            sq = fmaf(xr[nd][a], xr[nd][a], sq);
          }
          if (nd <= D) h2 = fmaxf(h2, sq);
        }
        float cj[NJ];
#pragma unroll
        for (int a = 0; a < D; ++a) {
#pragma unroll
          for (int b = 0; b < D; ++b) {
            float s = 0.f;
#pragma unroll
            for (int nd = 1; nd < NGEO; ++nd) s = fmaf(xr[nd][a], g0[nd * D + b], s);
            cj[a * D + b] = s;
          }
#pragma unroll
          for (int h = 0; h < NH; ++h) {
            float s = 0.f;
#pragma unroll
            for (int nd = 1; nd < NGEO; ++nd) s = fmaf(xr[nd][a], hs[nd * NH + h], s);
            cj[D * D + a * NH + h] = s;
          }
        }
        const float thr = 1e-14f * (D == 2 ? h2 : h2 * sqrtf(h2));
        if (half == 0 && ct >= 1) ok = warp_wait(bar(GEO_EMPTY), uint32_t(ct - 1) & 1u, &abort_flag);
        if (!ok) break;
#pragma unroll
        for (int j = 0; j < NJ; ++j) cellj[j * N_CELLS + c] = cj[j];
        thr_s[c] = thr;
      }
      if (!ok) break;
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(GEO_FULL));
    }
    if (!ok) {
      if (lane == 0) atomicOr(p.status, FFC_FLAG_TIMEOUT);
      abort_flag = 1;
    }
  } else if (warp < TQ_PRODUCER_WARPS) {
    // ---------------------------------------------------------------- producers: G~ chunks
    // lanes 0-7 and 8-15 take cells 0-7 of the warp's 16 (first and second half of the
    // columns), lanes 16-31 cells 8-15: each 8-lane phase of a 16-byte store writes eight
    // different rows of a core matrix, one bank group each
    const int c = warp * 16 + (lane & 7) + ((lane >> 4) << 3), hlf = (lane >> 3) & 1;
    bool ok = true;
    long long g = 0;
    for (long long ct = 0; ct < my_tiles && ok; ++ct) {
      ok = warp_wait(bar(GEO_FULL), uint32_t(ct) & 1u, &abort_flag);
      if (!ok) break;
      float cj[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) cj[j] = cellj[j * N_CELLS + c];
      const float thr = thr_s[c];
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(GEO_EMPTY));
      const long long e = (blockIdx.x + ct * gridDim.x) * N_CELLS + c;
      const bool live = e < p.n_elem;
      bool degenerate = false;
      // G~ at one point from the Jacobian there
      auto point_geometry = [&](const float (&J)[D][D], float* out) {
        float A[D][D];
        const float det = det_adj<D, float>(J, A);
        if (!(fabsf(det) > thr)) degenerate = true;
        const float ad = fabsf(det);
        if constexpr (FORM == FFC_MASS) {
          out[0] = ad;
        } else {
          const float r = __frcp_rn(ad);
#pragma unroll
          for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b) {
              float sq = 0.f;
#pragma unroll
              for (int cc = 0; cc < D; ++cc) sq = fmaf(A[a][cc], A[b][cc], sq);
              out[quad::qpair<D>(a, b)] = sq * r;
            }
        }
      };
      // G~ at the reference centroid: the drainers add (sum_k A~0(k)) : G~c in FP32 and
      // the tensor cores accumulate only the deviations G~(X_k) - G~c (exactly zero on
      // affine cells), so their FP32 accumulation error scales with the deviations
      float gc[NG];
      {
        float J[D][D];
        constexpr float xc = 1.f / (D + 1);
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b) {
            float v = cj[a * D + b];
#pragma unroll
            for (int cc = 0; cc < D; ++cc)
              if constexpr (NH > 0) v = fmaf(cj[D * D + a * NH + quad::qpair<D>(b, cc)], xc, v);
            J[a][b] = v;
          }
        float A[D][D];
        const float det = det_adj<D, float>(J, A);
        const float ad = fabsf(det);
        if constexpr (FORM == FFC_MASS) {
          gc[0] = ad;
        } else {
          const float r = __frcp_rn(ad);
#pragma unroll
          for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b) {
              float sq = 0.f;
#pragma unroll
              for (int cc = 0; cc < D; ++cc) sq = fmaf(A[a][cc], A[b][cc], sq);
              gc[quad::qpair<D>(a, b)] = sq * r;
            }
        }
        if (G == 1 && !(ad > thr)) degenerate = true;
        if (!live) {
#pragma unroll
          for (int gg = 0; gg < NG; ++gg) gc[gg] = 0.f;
        }
      }
      if (ct >= 2) ok = warp_wait(bar(GBAR_EMPTY + int(ct & 1)), uint32_t((ct - 2) >> 1) & 1u, &abort_flag);
      if (!ok) break;
      if (hlf == 0) {
#pragma unroll
        for (int gg = 0; gg < NG; ++gg) gbar[(int(ct & 1) * NG + gg) * N_CELLS + c] = gc[gg];
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(GBAR_FULL + int(ct & 1)));
      for (int ch = 0; ch < p.nch && ok; ++ch, ++g) {
        const int s = int(g & 1);
        if (g >= 2) ok = warp_wait(bar(B_EMPTY + s), uint32_t((g - 2) >> 1) & 1u, &abort_flag);
        if (!ok) break;
        float col[QKCH / 2];
#pragma unroll
        for (int pp = 0; pp < C::PPH; ++pp) {
          const int k = ch * C::PPC + hlf * C::PPH + pp;
          if (!live || k >= p.nq) {
#pragma unroll
            for (int gg = 0; gg < NG; ++gg) col[pp * NG + gg] = 0.f;
            continue;
          }
          if constexpr (G == 1) {
#pragma unroll
            for (int gg = 0; gg < NG; ++gg) col[pp * NG + gg] = 0.f;
          } else {
            float X[D];
#pragma unroll
            for (int a = 0; a < D; ++a) X[a] = xq[k * D + a];
            float J[D][D];
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
              for (int b = 0; b < D; ++b) {
                float v = cj[a * D + b];
#pragma unroll
                for (int cc = 0; cc < D; ++cc) v = fmaf(cj[D * D + a * NH + quad::qpair<D>(b, cc)], X[cc], v);
                J[a][b] = v;
              }
            point_geometry(J, col + pp * NG);
#pragma unroll
            for (int gg = 0; gg < NG; ++gg) col[pp * NG + gg] -= gc[gg];
          }
        }
        // split into the parts and write this lane's half of the cell's chunk row, 16 bytes at a time
        unsigned char* bs = Bs + s * C::STAGE_BYTES;
#pragma unroll
        for (int kc = 0; kc < C::KCC / 2; ++kc) {
          uint32_t w[S::PARTS][4];
#pragma unroll
          for (int j = 0; j < S::EPC; ++j) {
            typename S::Store parts[3];
            split_f32<MODE>(col[kc * S::EPC + j], parts);
#pragma unroll
            for (int qq = 0; qq < S::PARTS; ++qq) {
              if constexpr (S::BF16) {
                if (j & 1) w[qq][j >> 1] |= uint32_t(parts[qq]) << 16;
                else w[qq][j >> 1] = uint32_t(parts[qq]);
              } else {
                w[qq][j] = uint32_t(parts[qq]);
              }
            }
          }
          const uint32_t o = core_offset(c, (hlf * (C::KCC / 2) + kc) * S::EPC, C::KCC, S::EPC) * S::ESIZE;
#pragma unroll
          for (int qq = 0; qq < S::PARTS; ++qq)
            *reinterpret_cast<uint4*>(bs + qq * C::CH_BYTES + o) = make_uint4(w[qq][0], w[qq][1], w[qq][2], w[qq][3]);
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_FULL + s));
      }
      if (live && degenerate) atomicOr(p.status, FFC_FLAG_DEGENERATE);
    }
    if (!ok) {
      if (lane == 0) atomicOr(p.status, FFC_FLAG_TIMEOUT);
      abort_flag = 1;
    }
  } else {
    // ---------------------------------------------------------------- drainers: TMEM -> A_K
    bool ok = true;
    const int q4 = warp - TQ_DRAIN_WARP0;  // TMEM lanes 32 q4 .. 32 q4 + 31 (warp % 4)
    float a0s1[NG];  // one M tile: the entry's centroid-term row, loaded once
#pragma unroll
    for (int gg = 0; gg < NG; ++gg) a0s1[gg] = (!MULTI && q4 * 32 + lane < p.nn) ? p.a0sum[(q4 * 32 + lane) * NG + gg] : 0.f;
    for (long long ct = 0; ct < my_tiles && ok; ++ct) {
      const int acc = int(ct % nbuf), gsl = int(ct & 1);
      ok = warp_wait(bar(ACC_FULL + acc), uint32_t(ct / nbuf) & 1u, &abort_flag) &&
           warp_wait(bar(GBAR_FULL + gsl), uint32_t(ct >> 1) & 1u, &abort_flag);
      if (!ok) break;
      fence_after();
      const float* gb = gbar + gsl * NG * N_CELLS;
      const long long e0 = (blockIdx.x + ct * gridDim.x) * N_CELLS;
#pragma unroll 1
      for (int m = 0; m < mt; ++m) {
      const int i = m * M_TILE + q4 * 32 + lane;  // element-tensor entry (TMEM lane of M tile m)
      float a0s[NG];
#pragma unroll
      for (int gg = 0; gg < NG; ++gg) a0s[gg] = MULTI ? (i < p.nn ? p.a0sum[i * NG + gg] : 0.f) : a0s1[gg];
      const uint32_t taddr = tmem + (uint32_t(q4 * 32) << 16) + uint32_t(nbuf > 1 ? acc * C::ACC_COLS : m * N_CELLS);
#pragma unroll 1
      for (int c = 0; c < N_CELLS / 16; ++c) {
        uint32_t rv[16];
        float v[16];
        tmem_ld16_issue(taddr + c * 16, rv);
        if constexpr (S::NPROD > 1 && !MULTI) {
          uint32_t rw[16];
          tmem_ld16_issue(taddr + N_CELLS + c * 16, rw);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(rv[j]) + __uint_as_float(rw[j]);
        } else {
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(rv[j]);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float m = 0.f;
#pragma unroll
          for (int gg = 0; gg < NG; ++gg) m = fmaf(a0s[gg], gb[gg * N_CELLS + c * 16 + j], m);
          v[j] += m;
        }
        if (i < p.nn) {
          const long long ec = e0 + c * 16;
          if (p.slot) {  // Algorithm 2: FP64 atomic adds into the CSR values
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (ec + j < p.n_elem) {
                const int sl = __ldg(p.slot + (ec + j) * p.nn + i);
                if (sl >= 0 && sl < p.nnz) atomicAdd(p.csr_val + sl, double(v[j]));
                else atomicOr(p.status, FFC_FLAG_BOUNDS);
              }
          } else {
            float* dst = p.out + ec * p.nn + i;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (ec + j < p.n_elem) __stcs(dst + j * p.nn, v[j]);
          }
        }
      }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(bar(ACC_EMPTY + acc));
        mbar_arrive(bar(GBAR_EMPTY + gsl));
      }
    }
    if (!ok) {
      if (lane == 0) atomicOr(p.status, FFC_FLAG_TIMEOUT);
      abort_flag = 1;
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
  }
}

// The producers' table in FP32: the geometry table, then A~0 summed over the points
// [n*n][n_g] (FP64 sums rounded once), the drainers' centroid term.
std::vector<float> tq_table(const ffc_qform* f) {
  const std::vector<double> g = quad::geometry_table(f);
  std::vector<float> t(g.begin(), g.end());
  for (int i = 0; i < f->n * f->n; ++i)
    for (int gg = 0; gg < f->ng; ++gg) {
      double sum = 0.0;
      for (int k = 0; k < f->nq; ++k) sum += f->At[size_t(i) * f->K + size_t(k) * f->ng + gg];
      t.push_back(float(sum));
    }
  return t;
}

template <int MODE>
int upload_tq(ffc_qform* f, ffc_qform::Dev* dv, int nch) {
  using S = Split<MODE>;
  const int fam = S::BF16 ? 1 : 0;
  std::lock_guard<std::mutex> g(f->lock);
  if (dv->tc_part[fam][S::PARTS - 1] && dv->tq_table) return FFC_OK;
  const int nn = f->n * f->n, K = f->K, mt = (nn + M_TILE - 1) / M_TILE;
  const size_t per = size_t(nch) * mt * M_TILE * QKCH;  // elements per part
  const int nparts = S::BF16 ? 3 : 2;  // a family uploads all its parts once
  std::vector<std::vector<typename S::Store>> parts(nparts, std::vector<typename S::Store>(per, 0));
  for (int i = 0; i < nn; ++i)
    for (int j = 0; j < K; ++j) {
      double r = f->At[size_t(i) * K + j];
      const size_t o = (size_t(j / QKCH) * mt + i / M_TILE) * (M_TILE * QKCH) +
                       core_offset(i % M_TILE, j % QKCH, QKCH / S::EPC, S::EPC);
      for (int q = 0; q < nparts; ++q) {
        if constexpr (S::BF16) {
          const uint16_t b = host_bf16_bits(r);
          parts[q][o] = b;
          r -= host_value(uint32_t(b) << 16);
        } else {
          const uint32_t b = host_tf32_bits(r);
          parts[q][o] = b;
          r -= host_value(b);
        }
      }
    }
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < nparts && e == cudaSuccess; ++q) {
    cudaFree(dv->tc_part[fam][q]);
    dv->tc_part[fam][q] = nullptr;
    if ((e = cudaMalloc(&dv->tc_part[fam][q], per * sizeof(typename S::Store))) == cudaSuccess)
      e = cudaMemcpy(dv->tc_part[fam][q], parts[q].data(), per * sizeof(typename S::Store), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && !dv->tq_table) {
    const std::vector<float> t = tq_table(f);
    if ((e = cudaMalloc(&dv->tq_table, t.size() * sizeof(float))) == cudaSuccess)
      e = cudaMemcpy(dv->tq_table, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice);
  }
  return e == cudaSuccess ? FFC_OK : cuda_fail(e, "ffc_tabulate_quadrature: tensor-core operands");
}

template <int D, int FORM, int G, int MODE>
int launch_tq(ffc_qform* f, ffc_qform::Dev* dv, long long n_elem, const int32_t* cells, const double* nodes,
              long long n_nodes, const QOut& o, unsigned* status, cudaStream_t s) {
  using C = TqCfg<D, FORM, G, MODE>;
  using S = Split<MODE>;
  const int nch = (f->K + QKCH - 1) / QKCH;
  const size_t smem = C::smem_bytes(f->nq);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > size_t(optin)) {
    set_error("ffc_tabulate_quadrature: the rule's points do not fit next to the operand stages");
    return FFC_EINVAL;
  }
  int rc = upload_tq<MODE>(f, dv, nch);
  if (rc != FFC_OK) return rc;
  TqParams p{};
  p.cells = cells;
  p.nodes = nodes;
  p.n_nodes = n_nodes;
  p.n_elem = n_elem;
  p.table = dv->tq_table;
  p.a0sum = dv->tq_table + C::table_floats(f->nq);
  for (int q = 0; q < 3; ++q) p.a_part[q] = dv->tc_part[S::BF16 ? 1 : 0][q];
  p.out = static_cast<float*>(o.out);
  p.slot = o.slot;
  p.csr_val = o.csr_val;
  p.nnz = o.nnz;
  p.nn = f->n * f->n;
  p.nq = f->nq;
  p.nch = nch;
  p.mt = (p.nn + M_TILE - 1) / M_TILE;
  p.status = status;
  auto kern = p.mt > 1 ? tq_kernel<D, FORM, G, MODE, true> : tq_kernel<D, FORM, G, MODE, false>;
  int sms = 0;
  if (launch_config(reinterpret_cast<const void*>(kern), TQ_THREADS, smem, -1, &sms, nullptr) != FFC_OK)
    return FFC_ECUDA;
  const long long n_tiles = (n_elem + N_CELLS - 1) / N_CELLS;
  const long long grid = std::min<long long>(sms, n_tiles);
  kern<<<unsigned(std::max<long long>(grid, 1)), TQ_THREADS, smem, s>>>(p);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FFC_OK : cuda_fail(e, "tq_kernel launch");
}

template <int D, int FORM, int G>
int launch_tq_mode(ffc_qform* f, ffc_qform::Dev* dv, int precision, long long n_elem, const int32_t* cells,
                   const double* nodes, long long n_nodes, const QOut& out, unsigned* status, cudaStream_t s) {
  switch (precision) {
    case FFC_TF32: return launch_tq<D, FORM, G, MODE_TF32>(f, dv, n_elem, cells, nodes, n_nodes, out, status, s);
    case FFC_TF32X3: return launch_tq<D, FORM, G, MODE_TF32X3>(f, dv, n_elem, cells, nodes, n_nodes, out, status, s);
    default: return launch_tq<D, FORM, G, MODE_BF16X3>(f, dv, n_elem, cells, nodes, n_nodes, out, status, s);
  }
}

int run_tq(ffc_qform* f, ffc_qform::Dev* dv, int precision, long long n_elem, const int32_t* cells,
           const double* nodes, long long n_nodes, const QOut& out, unsigned* status, cudaStream_t s) {
  const bool mass = f->kind == FFC_MASS;
  if (f->d == 2) {
    if (f->g == 1)
      return mass ? launch_tq_mode<2, FFC_MASS, 1>(f, dv, precision, n_elem, cells, nodes, n_nodes, out, status, s)
                  : launch_tq_mode<2, FFC_POISSON, 1>(f, dv, precision, n_elem, cells, nodes, n_nodes, out, status, s);
    return mass ? launch_tq_mode<2, FFC_MASS, 2>(f, dv, precision, n_elem, cells, nodes, n_nodes, out, status, s)
                : launch_tq_mode<2, FFC_POISSON, 2>(f, dv, precision, n_elem, cells, nodes, n_nodes, out, status, s);
  }
  if (f->g == 1)
    return mass ? launch_tq_mode<3, FFC_MASS, 1>(f, dv, precision, n_elem, cells, nodes, n_nodes, out, status, s)
                : launch_tq_mode<3, FFC_POISSON, 1>(f, dv, precision, n_elem, cells, nodes, n_nodes, out, status, s);
  return mass ? launch_tq_mode<3, FFC_MASS, 2>(f, dv, precision, n_elem, cells, nodes, n_nodes, out, status, s)
              : launch_tq_mode<3, FFC_POISSON, 2>(f, dv, precision, n_elem, cells, nodes, n_nodes, out, status, s);
}

}  // namespace tq

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
               int precision, const char* who, bool tensor_cores = false) {
  const bool tc = precision == FFC_TF32 || precision == FFC_TF32X3 || precision == FFC_BF16X3;
  const bool oz = precision == FFC_FP64_OZAKI;
  if (!f || n_elem < 0 || n_nodes < 0 ||
      (precision != FFC_FP64 && precision != FFC_FP32 && !(tensor_cores && (tc || oz)))) {
    set_error(std::string(who) + (tensor_cores ? ": invalid argument (precision FFC_FP64, FFC_FP32, FFC_TF32, "
                                                 "FFC_TF32X3, FFC_BF16X3 or FFC_FP64_OZAKI)"
                                               : ": invalid argument (precision must be FFC_FP64 or FFC_FP32)"));
    return FFC_EINVAL;
  }
  if (tc && f->n * f->n > 4 * tc::M_TILE) {
    set_error(std::string(who) + ": the tensor-core precisions take element tensors of at most 512 entries");
    return FFC_EUNSUPPORTED;
  }
  if (oz) {
    const int rc = ozaki_supported(f);
    if (rc != FFC_OK) return rc;
  }
  if (n_elem > 0 && (!cells || !nodes || n_nodes == 0 || (reinterpret_cast<uintptr_t>(nodes) & 7))) {
    set_error(std::string(who) + ": null or misaligned cells / nodes");
    return FFC_EINVAL;
  }
  return FFC_OK;
}

}  // namespace
}  // namespace ffc

namespace ffc {
namespace quad {
std::vector<double> geometry_table(const ffc_qform* f) {
  const int d = f->d, ng = f->ngeo, nh = f->g == 2 ? d * (d + 1) / 2 : 0;
  std::vector<double> X(size_t(d + 1) * d, 0.0), psi, dpsi;
  for (int c = 0; c < d; ++c) X[size_t(c + 1) * d + c] = 1.0;
  reference_basis(d, f->g, X, psi, dpsi);  // [d+1][ng][d]
  std::vector<double> t;
  for (int nd = 0; nd < ng; ++nd)
    for (int b = 0; b < d; ++b) t.push_back(dpsi[size_t(nd) * d + b]);
  std::vector<double> h(size_t(ng) * std::max(nh, 1), 0.0);
  for (int nd = 0; nd < ng && nh; ++nd)
    for (int b = 0; b < d; ++b)
      for (int c = b; c < d; ++c)
        h[size_t(nd) * nh + sym_pair(d, b, c)] = dpsi[(size_t(c + 1) * ng + nd) * d + b] - dpsi[size_t(nd) * d + b];
  t.insert(t.end(), h.begin(), h.begin() + size_t(ng) * nh);
  t.insert(t.end(), f->X.begin(), f->X.end());
  return t;
}
}  // namespace quad
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
    cudaFree(kv.second.tq_table);
    cudaFree(kv.second.oz_a);
    cudaFree(kv.second.oz_table);
    for (auto& fam : kv.second.tc_part)
      for (void* q : fam) cudaFree(q);
    cudaSetDevice(prev);
  }
  delete f;
}

extern "C" int ffc_tabulate_quadrature(const ffc_qform* f, int64_t n_elem, const int32_t* cells, const double* nodes,
                                       int64_t n_nodes, void* A_K, int precision, void* stream) {
  int rc = check_args(f, n_elem, cells, nodes, n_nodes, precision, "ffc_tabulate_quadrature", true);
  if (rc != FFC_OK || n_elem == 0) return rc;
  if (!A_K || (reinterpret_cast<uintptr_t>(A_K) & 15)) {
    set_error("ffc_tabulate_quadrature: A_K null or not 16-byte aligned");
    return FFC_EINVAL;
  }
  if (precision != FFC_FP64 && precision != FFC_FP32) {
    ffc_qform::Dev* dv = nullptr;
    if ((rc = ensure_qdev(const_cast<ffc_qform*>(f), &dv)) != FFC_OK) return rc;
    unsigned* st = status_word();
    if (!st) {
      set_error("ffc_tabulate_quadrature: status word allocation failed");
      return FFC_ECUDA;
    }
    QOut o;
    o.out = A_K;
    if (precision == FFC_FP64_OZAKI)
      return run_ozaki(const_cast<ffc_qform*>(f), dv, n_elem, cells, nodes, n_nodes, o, st,
                       static_cast<cudaStream_t>(stream));
    return tq::run_tq(const_cast<ffc_qform*>(f), dv, precision, n_elem, cells, nodes, n_nodes, o, st,
                      static_cast<cudaStream_t>(stream));
  }
  return run_quadrature(f, n_elem, cells, nodes, n_nodes, A_K, nullptr, 0, precision, stream,
                        "ffc_tabulate_quadrature");
}

extern "C" int ffc_assemble_quadrature(const ffc_qform* f, int64_t n_elem, const int32_t* cells, const double* nodes,
                                       int64_t n_nodes, const int32_t* slot, double* csr_val, int64_t nnz,
                                       int precision, void* stream) {
  int rc = check_args(f, n_elem, cells, nodes, n_nodes, precision, "ffc_assemble_quadrature", true);
  if (rc != FFC_OK || n_elem == 0) return rc;
  if (!slot || !csr_val || nnz <= 0 || (reinterpret_cast<uintptr_t>(slot) & 3) ||
      (reinterpret_cast<uintptr_t>(csr_val) & 7)) {
    set_error("ffc_assemble_quadrature: slot / csr_val null, misaligned, or nnz <= 0");
    return FFC_EINVAL;
  }
  if (precision != FFC_FP64 && precision != FFC_FP32) {  // the tensor-core kernels, atomics in their drain
    ffc_qform::Dev* dv = nullptr;
    if ((rc = ensure_qdev(const_cast<ffc_qform*>(f), &dv)) != FFC_OK) return rc;
    unsigned* st = status_word();
    if (!st) {
      set_error("ffc_assemble_quadrature: status word allocation failed");
      return FFC_ECUDA;
    }
    QOut o;
    o.slot = slot;
    o.csr_val = csr_val;
    o.nnz = nnz;
    if (precision == FFC_FP64_OZAKI)
      return run_ozaki(const_cast<ffc_qform*>(f), dv, n_elem, cells, nodes, n_nodes, o, st,
                       static_cast<cudaStream_t>(stream));
    return tq::run_tq(const_cast<ffc_qform*>(f), dv, precision, n_elem, cells, nodes, n_nodes, o, st,
                      static_cast<cudaStream_t>(stream));
  }
  return run_quadrature(f, n_elem, cells, nodes, n_nodes, csr_val, slot, nnz, precision, stream,
                        "ffc_assemble_quadrature");
}
