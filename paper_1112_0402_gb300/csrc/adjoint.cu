// Reverse mode of the Poisson element tensors with respect to the vertex coordinates.
//
// Forward (Section 3.3, test case 2): A^K_i = sum_alpha A0[i][alpha] G[alpha] with
// G = s K K^T, s = |det J|, K = J^{-1}, J = [x_1 - x_0, ..., x_d - x_0].
// Given the upstream gradient dA[e][i] = dL/dA^K_i:
//   Gbar[alpha] = sum_i A0[i][alpha] dA[e][i]                      (transposed contraction)
//   c           = Gbar : (K K^T)
//   dL/dJ       = s (c K^T - K^T (Gbar + Gbar^T) K K^T)
// which follows from d s = s tr(K dJ) and dK = -K dJ K. Column c of J is
// x_{c+1} - x_0, so dL/dx_{c+1} += dL/dJ[:, c] and dL/dx_0 -= sum_c dL/dJ[:, c]; the
// vertex gradients are accumulated with FP64 atomic adds.
//
// A warp takes 32 cells: for each, the lanes stride over the n^2 entries (coalesced
// reads of dA) keeping |alpha| = d^2 partial sums against the transposed reference
// tensor held in shared memory, and reduce them with warp shuffles; lane k keeps cell
// k's Gbar. Then all 32 lanes run the geometry chain rule, one cell each. FP64.
#include <cuda_runtime.h>

#include "ffc_internal.h"
#include "geometry.cuh"

namespace ffc {
namespace {

constexpr int WARPS = 8;

template <int D, int Q>
__global__ void __launch_bounds__(WARPS * 32) poisson_adjoint_kernel(const int32_t* __restrict__ cells,
                                                                     const double* __restrict__ vertices,
                                                                     long long n_vert, const double* __restrict__ a0t,
                                                                     const double* __restrict__ dA, double* dvert,
                                                                     long long n_elem, unsigned* status) {
  constexpr int N = nscalar(D, Q);
  constexpr int NN = N * N;
  constexpr int NA = D * D;
  extern __shared__ double a0s[];  // [NA][NN]
  for (int k = threadIdx.x; k < NA * NN; k += blockDim.x) a0s[k] = a0t[k];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long warp_global = (long long)blockIdx.x * WARPS + (threadIdx.x >> 5);
  const long long n_warps = (long long)gridDim.x * WARPS;
  // each warp takes 32 consecutive cells: the lanes reduce Gbar for one cell at a
  // time (lane k keeps cell k's sums), then every lane runs the chain rule of its cell
  for (long long base = warp_global * 32; base < n_elem; base += n_warps * 32) {
    double mine[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) mine[a] = 0.0;
    const int count = (n_elem - base) < 32 ? int(n_elem - base) : 32;
#pragma unroll 1
    for (int k = 0; k < count; ++k) {
      double gb[NA];
#pragma unroll
      for (int a = 0; a < NA; ++a) gb[a] = 0.0;
      const double* row = dA + (base + k) * NN;
      for (int i = lane; i < NN; i += 32) {
        const double g = __ldg(row + i);
#pragma unroll
        for (int a = 0; a < NA; ++a) gb[a] = fma(a0s[a * NN + i], g, gb[a]);
      }
#pragma unroll
      for (int a = 0; a < NA; ++a) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) gb[a] += __shfl_xor_sync(0xffffffffu, gb[a], off);
        if (lane == k) mine[a] = gb[a];
      }
    }
    if (lane < count) {
      const long long e = base + lane;
      double gb[NA];
#pragma unroll
      for (int a = 0; a < NA; ++a) gb[a] = mine[a];
      double K[D][D], s;
      bool degenerate, bad_index;
      cell_geometry<D>(cells, vertices, n_vert, e, K, s, degenerate, bad_index);
      if (degenerate) atomicOr(status, FFC_FLAG_DEGENERATE);
      if (bad_index) atomicOr(status, FFC_FLAG_BOUNDS);
      double M[D][D];  // K K^T
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
          double t = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) t += K[a][k] * K[b][k];
          M[a][b] = t;
        }
      double c = 0.0, S[D][D];
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
          c += gb[a * D + b] * M[a][b];
          S[a][b] = gb[a * D + b] + gb[b * D + a];
        }
      // T = S M ; dJ = s (c K^T - K^T T)
      double T[D][D];
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
          double t = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) t += S[a][k] * M[k][b];
          T[a][b] = t;
        }
      double dJ[D][D];
#pragma unroll
      for (int r = 0; r < D; ++r)
#pragma unroll
        for (int col = 0; col < D; ++col) {
          double t = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) t += K[k][r] * T[k][col];
          dJ[r][col] = s * (c * K[col][r] - t);
        }
      int id[D + 1];
#pragma unroll
      for (int j = 0; j <= D; ++j) id[j] = __ldg(cells + e * (D + 1) + j);
#pragma unroll
      for (int r = 0; r < D && !bad_index; ++r) {
        double sum = 0.0;
#pragma unroll
        for (int col = 0; col < D; ++col) {
          atomicAdd(dvert + (long long)id[col + 1] * D + r, dJ[r][col]);
          sum += dJ[r][col];
        }
        atomicAdd(dvert + (long long)id[0] * D + r, -sum);
      }
    }
  }
}

template <int D, int Q>
int run(const LaunchArgs& a, const double* dA, double* dvert) {
  constexpr int N = nscalar(D, Q);
  constexpr size_t SMEM = size_t(D * D) * N * N * sizeof(double);
  auto kern = poisson_adjoint_kernel<D, Q>;
  static int sms = 0, per_sm = 1;
  if (sms == 0) {
    if (SMEM > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SMEM)) != cudaSuccess)
      return FFC_ECUDA;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, SMEM) != cudaSuccess)
      return FFC_ECUDA;
    if (per_sm < 1) per_sm = 1;
  }
  long long grid = (long long)sms * per_sm;
  const long long need = (a.n_elem + 32 * WARPS - 1) / (32 * WARPS);
  if (grid > need) grid = need;
  kern<<<unsigned(grid), WARPS * 32, SMEM, static_cast<cudaStream_t>(a.stream)>>>(
      a.cells, a.vertices, a.n_vert, a.t->a0t_f64, dA, dvert, a.n_elem, a.status);
  return cudaPeekAtLastError() == cudaSuccess ? FFC_OK : FFC_ECUDA;
}

}  // namespace

int launch_adjoint(const LaunchArgs& a, const double* dA, double* dvert) {
  if (a.f->kind != FFC_POISSON) return FFC_EUNSUPPORTED;
  if (a.f->d == 3) {
    switch (a.f->q) {
      case 1: return run<3, 1>(a, dA, dvert);
      case 2: return run<3, 2>(a, dA, dvert);
      case 3: return run<3, 3>(a, dA, dvert);
      case 4: return run<3, 4>(a, dA, dvert);
    }
  } else {
    switch (a.f->q) {
      case 1: return run<2, 1>(a, dA, dvert);
      case 2: return run<2, 2>(a, dA, dvert);
      case 3: return run<2, 3>(a, dA, dvert);
      case 4: return run<2, 4>(a, dA, dvert);
    }
  }
  return FFC_EUNSUPPORTED;
}

}  // namespace ffc
