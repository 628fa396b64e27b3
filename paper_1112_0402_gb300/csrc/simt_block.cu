// Structured contraction of the vector forms on CUDA cores.
//
// For a component-blocked Cartesian vector basis (phi_i = psi_s e_c), the reference
// tensors of the convection and elasticity forms are block structured (Section 3.5
// proposes exploiting exactly this): the element tensor decomposes into n_s x n_s
// blocks indexed by the components (c1, c2),
//
//   A_K[(c1,s1),(c2,s2)] = sum_k R[(s1,s2)][k] * Gb_K[b(c1,c2)][k],
//
// with a reduced reference tensor R and nb reduced geometry blocks per cell:
//   convection  R[(s1,s2)][(t,a)] = int psi_s1 psi_t d_a psi_s2 (k = t*d + a, n_s*d values),
//               one block H[(t,a)] = |det J| sum_c K[a][c] w_{c,t}, used on the diagonal
//               blocks c1 = c2 (off-diagonal blocks are structurally zero);
//   elasticity  R = scalar stiffness int d_a1 psi_s1 d_a2 psi_s2 (k = a1*d + a2, d*d values),
//               nine blocks Gb[(c1,c2)][(a1,a2)] = |det J| (mu delta(c1,c2) (K K^T)[a1][a2]
//               + mu K[a1][c2] K[a2][c1] + lambda K[a1][c1] K[a2][c2]).
// This is the same value as the dense A0 : G_K contraction (identical sums), with
// 27x (convection) and 9x (elasticity) fewer multiply-adds and a reference tensor small
// enough for registers. Thread layout as in the dense SIMT kernel: thread t owns
// entries i = t mod NTI + r*NTI of the cells of its group, so stores are coalesced;
// structurally zero entries are stored as 0 (tabulate) or skipped (assembly).
#include <cuda_runtime.h>

#include <type_traits>

#include "ffc_internal.h"
#include "geometry.cuh"

namespace ffc {
namespace {

template <int D, int FORM, int Q, typename T>
struct BlockCfg {
  static constexpr int NS = nscalar(D, Q);
  static constexpr int N = D * NS;
  static constexpr int NN = N * N;
  static constexpr int KR = FORM == FFC_NS_CONVECTION ? NS * D : D * D;
  static constexpr int NB = FORM == FFC_NS_CONVECTION ? 1 : D * D;
  static constexpr int VEC = 16 / int(sizeof(T));
  static constexpr int KRP = (KR + VEC - 1) / VEC * VEC;
  static constexpr int R = (NN + 511) / 512;
  static constexpr int NTI = (NN + R - 1) / R;
  static constexpr int EG = NTI >= 256 ? 1 : 256 / NTI;
  static constexpr int NT = NTI * EG;
  static constexpr bool REG_R = R * KR * int(sizeof(T)) / 4 <= 96;
  static constexpr int KE = (128 + EG - 1) / EG;  // 128 cells per tile: 4 warps share the geometry
  static constexpr int E = EG * KE;
  static constexpr int NCOEF = FORM == FFC_NS_CONVECTION ? N : 0;
  static constexpr size_t G_BYTES = size_t(E) * NB * KRP * sizeof(T);
  static constexpr size_t R_BYTES = REG_R ? 0 : size_t(NS) * NS * KRP * sizeof(T);
  static constexpr size_t SMEM = G_BYTES + R_BYTES + size_t(E) * NCOEF * sizeof(double);
};

struct BlockParams {
  const int32_t* cells;
  const double* vertices;
  long long n_vert;
  const double* coeffs;
  const void* r;  // reduced reference tensor [ns*ns][kr]
  void* out;
  const int32_t* slot;
  double* csr_val;
  long long nnz;
  long long n_elem;
  double mu, lambda;
  unsigned* status;
};

template <int D, int FORM, int Q, typename T, bool ASSEMBLE>
__global__ void __launch_bounds__(BlockCfg<D, FORM, Q, T>::NT) simt_block_kernel(BlockParams p) {
  using C = BlockCfg<D, FORM, Q, T>;
  extern __shared__ __align__(16) unsigned char smem[];
  T* Gs = reinterpret_cast<T*>(smem);                                       // [E][NB][KRP]
  T* Rs = reinterpret_cast<T*>(smem + C::G_BYTES);                          // [NS*NS][KRP] (smem path)
  double* Ws = reinterpret_cast<double*>(smem + C::G_BYTES + C::R_BYTES);   // [E][NCOEF]
  const int t = threadIdx.x;
  const int ti = t % C::NTI;
  const int eg = t / C::NTI;
  const T* Rg = static_cast<const T*>(p.r);

  // per owned entry: reduced row index and block offset (-1: structurally zero)
  int row[C::R], boff[C::R];
#pragma unroll
  for (int r = 0; r < C::R; ++r) {
    const int i = ti + r * C::NTI;
    row[r] = 0;
    boff[r] = -1;
    if (i < C::NN) {
      const int i1 = i / C::N, i2 = i % C::N;
      const int c1 = i1 / C::NS, s1 = i1 % C::NS, c2 = i2 / C::NS, s2 = i2 % C::NS;
      row[r] = s1 * C::NS + s2;
      if constexpr (FORM == FFC_NS_CONVECTION) boff[r] = (c1 == c2) ? 0 : -1;
      else boff[r] = (c1 * D + c2) * C::KRP;
    }
  }
  T rr[C::REG_R ? C::R : 1][C::REG_R ? C::KR : 1];
  if constexpr (C::REG_R) {
#pragma unroll
    for (int r = 0; r < C::R; ++r)
#pragma unroll
      for (int k = 0; k < C::KR; ++k) rr[r][k] = Rg[size_t(row[r]) * C::KR + k];
  } else {
    for (int k = t; k < C::NS * C::NS * C::KRP; k += C::NT) {
      const int rw = k / C::KRP, kk = k % C::KRP;
      Rs[k] = kk < C::KR ? Rg[size_t(rw) * C::KR + kk] : T(0);
    }
  }
  const long long n_tiles = (p.n_elem + C::E - 1) / C::E;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long long e0 = tile * C::E;
    if constexpr (C::NCOEF > 0) {
      const long long lim = (p.n_elem - e0) * C::NCOEF;
      const double* src = p.coeffs + e0 * C::NCOEF;
      for (int k = t; k < C::E * C::NCOEF; k += C::NT) Ws[k] = (k < lim) ? __ldg(src + k) : 0.0;
    }
    __syncthreads();
    // ---- reduced geometry blocks of the tile's cells (FP64)
    for (int el = t; el < C::E; el += C::NT) {
      const long long e = e0 + el;
      T* g = Gs + size_t(el) * C::NB * C::KRP;
      double K[D][D] = {}, det = 0.0;
      bool live = e < p.n_elem;
      if (live) {
        bool degenerate, bad_index;
        cell_geometry<D>(p.cells, p.vertices, p.n_vert, e, K, det, degenerate, bad_index);
        if (degenerate) atomicOr(p.status, FFC_FLAG_DEGENERATE);
        if (bad_index) atomicOr(p.status, FFC_FLAG_BOUNDS);
      }
      if constexpr (FORM == FFC_NS_CONVECTION) {
        const double* w = Ws + el * C::NCOEF;
#pragma unroll
        for (int st = 0; st < C::NS; ++st)
#pragma unroll
          for (int a = 0; a < D; ++a) {
            double h = 0.0;
#pragma unroll
            for (int c = 0; c < D; ++c) h += K[a][c] * w[c * C::NS + st];
            g[st * D + a] = live ? T(det * h) : T(0);
          }
      } else {
        double KK[D][D];
#pragma unroll
        for (int a1 = 0; a1 < D; ++a1)
#pragma unroll
          for (int a2 = 0; a2 < D; ++a2) {
            double sum = 0.0;
#pragma unroll
            for (int b = 0; b < D; ++b) sum += K[a1][b] * K[a2][b];
            KK[a1][a2] = sum;
          }
#pragma unroll
        for (int c1 = 0; c1 < D; ++c1)
#pragma unroll
          for (int c2 = 0; c2 < D; ++c2)
#pragma unroll
            for (int a1 = 0; a1 < D; ++a1)
#pragma unroll
              for (int a2 = 0; a2 < D; ++a2) {
                double v = p.mu * K[a1][c2] * K[a2][c1] + p.lambda * K[a1][c1] * K[a2][c2];
                if (c1 == c2) v += p.mu * KK[a1][a2];
                g[(c1 * D + c2) * C::KRP + a1 * D + a2] = live ? T(det * v) : T(0);
              }
      }
#pragma unroll
      for (int b = 0; b < C::NB; ++b)
        for (int k = C::KR; k < C::KRP; ++k) g[b * C::KRP + k] = T(0);
    }
    __syncthreads();
    // ---- contraction per owned entry
#pragma unroll 1
    for (int kc = 0; kc < C::KE; ++kc) {
      const int el = eg + kc * C::EG;
      const long long e = e0 + el;
      if (e >= p.n_elem) break;
      const T* g = Gs + size_t(el) * C::NB * C::KRP;
#pragma unroll
      for (int r = 0; r < C::R; ++r) {
        const int i = ti + r * C::NTI;
        if (i >= C::NN) continue;
        T acc = T(0);
        if (boff[r] >= 0) {
          const T* gb = g + boff[r];
          if constexpr (C::REG_R) {
#pragma unroll
            for (int k = 0; k < C::KR; ++k) acc = fma(gb[k], rr[r][k], acc);
          } else {
            const T* rw = Rs + size_t(row[r]) * C::KRP;
#pragma unroll
            for (int k = 0; k < C::KR; ++k) acc = fma(gb[k], rw[k], acc);
          }
        }
        const long long o = e * C::NN + i;
        if constexpr (ASSEMBLE) {
          if (boff[r] >= 0) {  // structural zeros add nothing
            const int s = __ldg(p.slot + o);
            if (s >= 0 && s < p.nnz) atomicAdd(p.csr_val + s, double(acc));
            else atomicOr(p.status, FFC_FLAG_BOUNDS);
          }
        } else {
          __stcs(static_cast<T*>(p.out) + o, acc);
        }
      }
    }
    __syncthreads();
  }
}

template <int D, int FORM, int Q, typename T, bool ASSEMBLE>
int run(const LaunchArgs& a) {
  using C = BlockCfg<D, FORM, Q, T>;
  auto kern = simt_block_kernel<D, FORM, Q, T, ASSEMBLE>;
  static int sms = 0, per_sm = 1;
  if (sms == 0) {
    if (C::SMEM > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM)) != cudaSuccess)
      return FFC_ECUDA;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NT, C::SMEM) != cudaSuccess)
      return FFC_ECUDA;
    if (per_sm < 1) per_sm = 1;
  }
  BlockParams p{a.cells, a.vertices, a.n_vert, a.coeffs,
                std::is_same<T, double>::value ? (const void*)a.t->r_f64 : (const void*)a.t->r_f32,
                a.out, a.slot, a.csr_val, a.nnz, a.n_elem, a.f->mu, a.f->lambda, a.status};
  const long long n_tiles = (a.n_elem + C::E - 1) / C::E;
  long long grid = (long long)sms * per_sm;
  if (grid > n_tiles) grid = n_tiles;
  kern<<<unsigned(grid), C::NT, C::SMEM, static_cast<cudaStream_t>(a.stream)>>>(p);
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
