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
// One thread per cell. Only the symmetric part of Gbar enters (c = Gbar : K K^T with
// K K^T symmetric, and Gbar + Gbar^T), so each thread accumulates the d(d+1)/2
// combinations against the reference tensor in the kernels' symmetric layout (columns
// (a,a) and (a,b) + (b,a)), held in shared memory and read as a broadcast (all lanes at
// the same entry i); no cross-lane reductions. Then it runs the geometry chain rule
// and scatters with atomics. FP64.
#include <cuda_runtime.h>

#include "ffc_internal.h"
#include "geometry.cuh"

namespace ffc {
namespace {

constexpr int THREADS = 256;

template <int D, int Q>
__global__ void __launch_bounds__(THREADS) poisson_adjoint_kernel(const int32_t* __restrict__ cells,
                                                                 const double* __restrict__ vertices,
                                                                 long long n_vert, const double* __restrict__ a0t,
                                                                 const double* __restrict__ dA, double* dvert,
                                                                 long long n_elem, unsigned* status) {
  constexpr int N = nscalar(D, Q);
  constexpr int NN = N * N;
  constexpr int NP = D * (D + 1) / 2;
  // the reference tensor in the symmetric layout, one row per entry i:
  // P[i][aa] = A0[i][(a,a)], P[i][ab] = A0[i][(a,b)] + A0[i][(b,a)] (a < b)
  extern __shared__ double a0s[];  // [NN][NP]
  for (int k = threadIdx.x; k < NN * NP; k += blockDim.x) {
    const int i = k / NP, pidx = k % NP;
    a0s[k] = a0t[pidx * NN + i];
  }
  __syncthreads();
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n_elem;
       e += (long long)gridDim.x * blockDim.x) {
    // gp[aa] = Gbar[a][a], gp[ab] = Gbar[a][b] + Gbar[b][a]
    double gp[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) gp[k] = 0.0;
    const double* row = dA + e * NN;
#pragma unroll 4
    for (int i = 0; i < NN; ++i) {
      const double g = __ldg(row + i);
#pragma unroll
      for (int k = 0; k < NP; ++k) gp[k] = fma(a0s[i * NP + k], g, gp[k]);
    }
    double K[D][D], s;
    bool degenerate, bad_index;
    cell_geometry<D>(cells, vertices, n_vert, e, K, s, degenerate, bad_index);
    if (degenerate) atomicOr(status, FFC_FLAG_DEGENERATE);
    if (bad_index) {
      atomicOr(status, FFC_FLAG_BOUNDS);
      continue;
    }
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
    // S = Gbar + Gbar^T, c = Gbar : M (M symmetric)
    double S[D][D], c = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) {
        const double v = gp[sym_pair_index<D>(a < b ? a : b, a < b ? b : a)];
        S[a][b] = (a == b) ? 2.0 * v : v;
        if (a <= b) c += v * M[a][b];
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
    for (int r = 0; r < D; ++r) {
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

template <int D, int Q>
int run(const LaunchArgs& a, const double* dA, double* dvert) {
  constexpr int N = nscalar(D, Q);
  constexpr size_t SMEM = size_t(D * (D + 1) / 2) * N * N * sizeof(double);
  auto kern = poisson_adjoint_kernel<D, Q>;
  int sms = 0, per_sm = 1;
  if (launch_config(reinterpret_cast<const void*>(kern), THREADS, SMEM, -1, &sms, &per_sm) != FFC_OK)
    return FFC_ECUDA;
  long long grid = (long long)sms * per_sm;
  const long long need = (a.n_elem + THREADS - 1) / THREADS;
  if (grid > need) grid = need;
  kern<<<unsigned(grid), THREADS, SMEM, static_cast<cudaStream_t>(a.stream)>>>(
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
