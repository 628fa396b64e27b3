// Structured contraction of the vector forms on CUDA cores (tile body and kernel).
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
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "ffc_internal.h"
#include "geometry.cuh"
#include "simt_kernels.cuh"

namespace ffc {

// BLOCK = 0: block size from n^2; BLOCK > 0: fixed block size shared with other forms
// (batched kernel). KE_T: cells per thread group and tile (0 = 128).
template <int D, int FORM, int Q, typename T, int BLOCK = 0, int KE_T = 0>
struct BlockCfg {
  static constexpr int NS = nscalar(D, Q);
  static constexpr int N = D * NS;
  static constexpr int NN = N * N;
  static constexpr int KR = FORM == FFC_NS_CONVECTION ? NS * D : D * D;
  static constexpr int NB = FORM == FFC_NS_CONVECTION ? 1 : D * D;
  static constexpr int VEC = 16 / int(sizeof(T));
  static constexpr int KRP = (KR + VEC - 1) / VEC * VEC;
  static constexpr int RMAX_THREADS = BLOCK > 0 ? BLOCK : 512;
  static constexpr int R = (NN + RMAX_THREADS - 1) / RMAX_THREADS;
  static constexpr int NTI = (NN + R - 1) / R;
  static constexpr int EG = BLOCK > 0 ? BLOCK / NTI : (NTI >= 256 ? 1 : 256 / NTI);
  static constexpr int NT = BLOCK > 0 ? BLOCK : NTI * EG;
  static constexpr bool REG_R = R * KR * int(sizeof(T)) / 4 <= (BLOCK > 0 ? (BLOCK >= 512 ? 80 : 32) : 96);
  static constexpr int KE = ((KE_T > 0 ? KE_T : 128) + EG - 1) / EG;  // 128 cells: 4 warps share the geometry
  static constexpr int E = EG * KE;
  static constexpr int NCOEF = FORM == FFC_NS_CONVECTION ? N : 0;
  static constexpr size_t G_BYTES = size_t(E) * NB * KRP * sizeof(T);
  static constexpr size_t R_BYTES = REG_R ? 0 : size_t(NS) * NS * KRP * sizeof(T);
  static constexpr size_t SMEM = G_BYTES + R_BYTES + size_t(E) * NCOEF * sizeof(double);
};

template <class C, typename T>
struct BlockRows {
  int row[C::R];   // reduced row (s1, s2) of each owned entry
  int boff[C::R];  // offset of its geometry block in a cell's blocks; -1: structurally zero
  T rr[C::REG_R ? C::R : 1][C::REG_R ? C::KR : 1];
};

// Per-thread entry decoding and the reduced reference tensor (registers, or shared memory
// behind the geometry blocks; the first barrier of block_tile orders those stores).
template <class C, int D, int FORM, typename T>
__device__ __forceinline__ void block_rows_init(const void* r, BlockRows<C, T>& b, unsigned char* smem) {
  const int t = threadIdx.x;
  const int ti = t % C::NTI;
  const T* Rg = static_cast<const T*>(r);
#pragma unroll
  for (int k = 0; k < C::R; ++k) {
    const int i = ti + k * C::NTI;
    b.row[k] = 0;
    b.boff[k] = -1;
    if (i < C::NN) {
      const int i1 = i / C::N, i2 = i % C::N;
      const int c1 = i1 / C::NS, s1 = i1 % C::NS, c2 = i2 / C::NS, s2 = i2 % C::NS;
      b.row[k] = s1 * C::NS + s2;
      if constexpr (FORM == FFC_NS_CONVECTION) b.boff[k] = (c1 == c2) ? 0 : -1;
      else b.boff[k] = (c1 * D + c2) * C::KRP;
    }
  }
  if constexpr (C::REG_R) {
#pragma unroll
    for (int k = 0; k < C::R; ++k)
#pragma unroll
      for (int j = 0; j < C::KR; ++j) b.rr[k][j] = Rg[size_t(b.row[k]) * C::KR + j];
  } else {
    T* Rs = reinterpret_cast<T*>(smem + C::G_BYTES);
    for (int k = t; k < C::NS * C::NS * C::KRP; k += C::NT) {
      const int rw = k / C::KRP, kk = k % C::KRP;
      Rs[k] = kk < C::KR ? Rg[size_t(rw) * C::KR + kk] : T(0);
    }
  }
}

// One tile of E cells: reduced geometry blocks (FP64) into shared memory, then each
// owned entry contracts its block with its reduced row. Contains block barriers.
template <class C, int D, int FORM, int Q, typename T, bool ASSEMBLE>
__device__ __forceinline__ void block_tile(const SimtParams& p, long long tile, unsigned char* smem,
                                           const BlockRows<C, T>& br) {
  T* Gs = reinterpret_cast<T*>(smem);                                       // [E][NB][KRP]
  const T* Rs = reinterpret_cast<const T*>(smem + C::G_BYTES);              // [NS*NS][KRP]
  double* Ws = reinterpret_cast<double*>(smem + C::G_BYTES + C::R_BYTES);   // [E][NCOEF]
  const int t = threadIdx.x;
  const int ti = t % C::NTI;
  const int eg = t / C::NTI;
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
  // ---- contraction per owned entry (thread groups beyond EG idle); in assembly the
  // slots of the next cell are loaded while this cell's atomics issue
  int slot_next[ASSEMBLE ? C::R : 1];
  if constexpr (ASSEMBLE) {
    const long long e = e0 + eg;
#pragma unroll
    for (int r = 0; r < C::R; ++r) {
      const int i = ti + r * C::NTI;
      slot_next[r] = (eg < C::EG && e < p.n_elem && i < C::NN && br.boff[r] >= 0) ? __ldg(p.slot + e * C::NN + i)
                                                                                  : -1;
    }
  }
#pragma unroll 1
  for (int kc = 0; kc < C::KE && eg < C::EG; ++kc) {
    const int el = eg + kc * C::EG;
    const long long e = e0 + el;
    if (e >= p.n_elem) break;
    int slot_cur[ASSEMBLE ? C::R : 1];
    if constexpr (ASSEMBLE) {
      const long long en = e + C::EG;
      const bool more = (kc + 1 < C::KE) && (en < p.n_elem);
#pragma unroll
      for (int r = 0; r < C::R; ++r) {
        const int i = ti + r * C::NTI;
        slot_cur[r] = slot_next[r];
        slot_next[r] = (more && i < C::NN && br.boff[r] >= 0) ? __ldg(p.slot + en * C::NN + i) : -1;
      }
    }
    const T* g = Gs + size_t(el) * C::NB * C::KRP;
#pragma unroll
    for (int r = 0; r < C::R; ++r) {
      const int i = ti + r * C::NTI;
      if (i >= C::NN) continue;
      T acc = T(0);
      if (br.boff[r] >= 0) {
        const T* gb = g + br.boff[r];
        if constexpr (C::REG_R) {
#pragma unroll
          for (int k = 0; k < C::KR; ++k) acc = fma(gb[k], br.rr[r][k], acc);
        } else {
          const T* rw = Rs + size_t(br.row[r]) * C::KRP;
#pragma unroll
          for (int k = 0; k < C::KR; ++k) acc = fma(gb[k], rw[k], acc);
        }
      }
      const long long o = e * C::NN + i;
      if constexpr (ASSEMBLE) {
        if (br.boff[r] >= 0) {  // structural zeros add nothing
          const int s = slot_cur[r];
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

template <int D, int FORM, int Q, typename T, bool ASSEMBLE>
__global__ void __launch_bounds__(BlockCfg<D, FORM, Q, T>::NT) simt_block_kernel(SimtParams p) {
  using C = BlockCfg<D, FORM, Q, T>;
  extern __shared__ __align__(16) unsigned char smem[];
  BlockRows<C, T> rows;
  block_rows_init<C, D, FORM, T>(p.a0, rows, smem);
  const long long n_tiles = (p.n_elem + C::E - 1) / C::E;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x)
    block_tile<C, D, FORM, Q, T, ASSEMBLE>(p, tile, smem, rows);
}

}  // namespace ffc
