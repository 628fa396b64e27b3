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
// enough for registers.
//
// Thread layouts. Elasticity, "row slots": a slot is (s1, c2, s2), numbered with s2
// fastest, then c2, then s1, so consecutive slots are consecutive entries of element
// tensor row (c1, s1) for every c1; the slot keeps R[(s1,s2)] in registers and per cell
// contracts it with the block (c1, c2) for each c1: a warp's store (or atomic) instruction
// covers a contiguous run of one row (one CSR row in assembly). Convection, "pair major":
// a slot is a pair (s1, s2); its one block is contracted once per cell and written to the
// d diagonal positions, zeros elsewhere (tabulate) or nothing (assembly); row slots would
// repeat that contraction d times. Earlier single layouts for both: "entry major" (each
// thread an entry of the row-major element tensor; convection P2 1.57 ms) and pair major
// for elasticity too (runs of n_s entries per store: elasticity P3 0.66 ms, batched 17.2
// ms, against 0.56 and 15.1 ms with row slots).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "ffc_internal.h"
#include "geometry.cuh"
#include "simt_kernels.cuh"

namespace ffc {

// BLOCK = 0: thread count from the number of pairs; BLOCK > 0: fixed block size shared
// with other forms (batched kernel). KE_T > 0: cells per thread group and tile (tiles
// are capped at 128 cells); 0 = 128 cells per tile.
template <int D, int FORM, int Q, typename T, int BLOCK = 0, int KE_T = 0>
struct BlockCfg {
  static constexpr int NS = nscalar(D, Q);
  static constexpr int N = D * NS;
  static constexpr int NN = N * N;
  static constexpr int KR = FORM == FFC_NS_CONVECTION ? NS * D : D * D;
  static constexpr int NB = FORM == FFC_NS_CONVECTION ? 1 : D * D;
  static constexpr int VEC = 16 / int(sizeof(T));
  static constexpr int KRP = (KR + VEC - 1) / VEC * VEC;
  static constexpr bool DIAG = FORM == FFC_NS_CONVECTION;  // one block, on the diagonal
  static constexpr int NP2 = NS * NS;                      // pairs (s1, s2): rows of R
  static constexpr int NSL = DIAG ? NP2 : D * NS * NS;     // slots: pairs, or row slots (s1, c2, s2)
  // about 256 threads: whole groups of NSL slots, or up to 512 threads with several
  // slots each, rounded up to whole warps
  // (FP32 with 512 or more slots: 416 threads, two resident CTAs; see MIN_BLOCKS)
  static constexpr int NT0 = NSL >= 256 ? (NSL < 512 ? NSL : (sizeof(T) == 4 ? 416 : 512)) : NSL * (256 / NSL);
  static constexpr int NT = BLOCK > 0 ? BLOCK : (NT0 + 31) / 32 * 32;
  static constexpr int GRP = NT >= NSL ? NT / NSL : 1;  // thread groups; a tile's cells are dealt to them
  static constexpr int PPT = (NSL + NT - 1) / NT;       // slots per thread
  static constexpr bool REG_R = PPT * KR * int(sizeof(T)) / 4 <= 64;
  static constexpr int E_DEF = (FORM == FFC_NS_CONVECTION && sizeof(T) == 8) ? 64 : 128;
  static constexpr int E = KE_T > 0 ? (KE_T * GRP < 128 ? KE_T * GRP : 128) : E_DEF;  // cells per tile
  static constexpr int NCOEF = FORM == FFC_NS_CONVECTION ? N : 0;
  static constexpr size_t G_BYTES = size_t(E) * NB * KRP * sizeof(T);
  static constexpr size_t R_BYTES = REG_R ? 0 : size_t(NP2) * KRP * sizeof(T);
  static constexpr size_t W_BYTES = size_t(E) * NCOEF * sizeof(double);
  static constexpr size_t SMEM = G_BYTES + R_BYTES + W_BYTES;
  // register budget of the single-form FP32 kernel: two resident CTAs of 257..511 threads
  // (up to 78 registers), three of up to 256; FP64 (bound by the FP64 pipe) keeps its
  // reduced rows in registers without spills
  static constexpr int MIN_BLOCKS = sizeof(T) == 8 ? 1 : (NT >= 512 ? 1 : (NT > 256 ? 2 : 3));
};

template <class C, typename T>
struct BlockRows {
  T rr[C::REG_R ? C::PPT : 1][C::REG_R ? C::KR : 1];  // reduced rows of the thread's slots
};

// Tabulate of the single-form FP32 convection kernel: the element tensors of CELLS cells
// at a time are put together in shared memory (the off-diagonal blocks, always zero, are
// written there once), then one thread writes them to A_K with a TMA bulk copy, two
// buffers deep, so A_K leaves the SM as whole contiguous lines instead of runs of n_s
// floats. Convection P2 on 384,000 cells: 0.362 ms with direct stores; 0.297 ms staged
// with 4-cell chunks and 128-cell tiles, against 0.31-0.34 ms for 2-, 6- or 8-cell chunks
// or 64-cell tiles. Elasticity, whose row-slot stores are already contiguous runs of a
// row, writes directly (staged in 2-cell chunks its P3 tabulate went 0.513 -> 0.608 ms).
template <class C, typename T, bool ASSEMBLE>
struct BlockStaging {
  static constexpr bool ON = !ASSEMBLE && C::DIAG && sizeof(T) == 4;
  static constexpr int CELLS = C::GRP > 4 ? C::GRP : 4;  // at least one cell per thread group
  static constexpr size_t BUF = size_t(CELLS) * C::NN * sizeof(T);  // a multiple of 16 bytes
  static constexpr size_t BYTES = ON ? 2 * BUF : 0;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
// shared -> global bulk copy (addresses 16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_s2g(void* gdst, const void* ssrc, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gdst), "r"(smem_u32(ssrc)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(PENDING) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// The thread's slots: slot j is q = t mod NSL (NT >= NSL, group t / NSL) or q = t + j*NT
// (NT < NSL, one group); -1: none. Slot q is (s1, c2, s2) with s2 fastest.
template <class C>
__device__ __forceinline__ int slot_of(int t, int j) {
  if constexpr (C::NT >= C::NSL) return (j == 0 && t < C::GRP * C::NSL) ? t % C::NSL : -1;
  else return (t + j * C::NT < C::NSL) ? t + j * C::NT : -1;
}
template <class C>
__device__ __forceinline__ int pair_of_slot(int q) {  // the row (s1, s2) of R a slot uses
  if constexpr (C::DIAG) return q;
  const int s2 = q % C::NS, s1 = q / (C::NS * (C::N / C::NS));
  return s1 * C::NS + s2;
}

// The reduced reference tensor rows (registers, or shared memory behind the geometry
// blocks; the first barrier of block_tile orders those stores).
template <class C, int D, int FORM, typename T>
__device__ __forceinline__ void block_rows_init(const void* r, BlockRows<C, T>& b, unsigned char* smem) {
  const int t = threadIdx.x;
  const T* Rg = static_cast<const T*>(r);
  if constexpr (C::REG_R) {
#pragma unroll
    for (int j = 0; j < C::PPT; ++j) {
      const int q = slot_of<C>(t, j);
      const int pp = q >= 0 ? pair_of_slot<C>(q) : 0;
#pragma unroll
      for (int k = 0; k < C::KR; ++k) b.rr[j][k] = q >= 0 ? Rg[size_t(pp) * C::KR + k] : T(0);
    }
  } else {
    T* Rs = reinterpret_cast<T*>(smem + C::G_BYTES);
    for (int k = t; k < C::NP2 * C::KRP; k += C::NT) {
      const int rw = k / C::KRP, kk = k % C::KRP;
      Rs[k] = kk < C::KR ? Rg[size_t(rw) * C::KR + kk] : T(0);
    }
  }
}

// One tile of E cells: reduced geometry blocks into shared memory, then each thread
// contracts its pairs with every block of the group's cells. Contains block barriers.
template <class C, int D, int FORM, int Q, typename T, bool ASSEMBLE>
__device__ __forceinline__ void block_tile(const SimtParams& p, long long tile, unsigned char* smem,
                                           const BlockRows<C, T>& br, int* staged_chunks = nullptr) {
  T* Gs = reinterpret_cast<T*>(smem);                                       // [E][NB][KRP]
  const T* Rs = reinterpret_cast<const T*>(smem + C::G_BYTES);              // [NP2][KRP]
  double* Ws = reinterpret_cast<double*>(smem + C::G_BYTES + C::R_BYTES);   // [E][NCOEF]
  const int t = threadIdx.x;
  const long long e0 = tile * C::E;
  if constexpr (C::NCOEF > 0) {
    const long long lim = (p.n_elem - e0) * C::NCOEF;
    const double* src = p.coeffs + e0 * C::NCOEF;
    for (int k = t; k < C::E * C::NCOEF; k += C::NT) Ws[k] = (k < lim) ? __ldg(src + k) : 0.0;
  }
  __syncthreads();
  // ---- reduced geometry blocks of the tile's cells
  for (int el = t; el < C::E; el += C::NT) {
    const long long e = e0 + el;
    T* g = Gs + size_t(el) * C::NB * C::KRP;
    // J^{-1} and det J in FP64 (measured: forming J^{-1} in FP32 from the FP64 adjugate,
    // as the dense kernels do, made this tile slower); the reduced geometry blocks, their
    // products with the coefficients, in the contraction's type (rounded to it anyway)
    double K[D][D] = {}, det = 0.0;
    bool live = e < p.n_elem;
    if (live) {
      bool degenerate, bad_index;
      cell_geometry<D>(p.cells, p.vertices, p.n_vert, e, K, det, degenerate, bad_index);
      if (degenerate) atomicOr(p.status, FFC_FLAG_DEGENERATE);
      if (bad_index) atomicOr(p.status, FFC_FLAG_BOUNDS);
    }
    using GT = T;
    GT Kt[D][D], dett = GT(det);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) Kt[a][b] = GT(K[a][b]);
    if constexpr (FORM == FFC_NS_CONVECTION) {
      const double* w = Ws + el * C::NCOEF;
#pragma unroll
      for (int st = 0; st < C::NS; ++st) {
        GT wc[D];
#pragma unroll
        for (int c = 0; c < D; ++c) wc[c] = GT(w[c * C::NS + st]);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          GT h = GT(0);
#pragma unroll
          for (int c = 0; c < D; ++c) h = fma(Kt[a][c], wc[c], h);
          g[st * D + a] = live ? dett * h : T(0);
        }
      }
    } else {
      GT KK[D][D];
#pragma unroll
      for (int a1 = 0; a1 < D; ++a1)
#pragma unroll
        for (int a2 = 0; a2 < D; ++a2) {
          GT sum = GT(0);
#pragma unroll
          for (int b = 0; b < D; ++b) sum = fma(Kt[a1][b], Kt[a2][b], sum);
          KK[a1][a2] = sum;
        }
      const GT mu = GT(p.mu), lambda = GT(p.lambda);
#pragma unroll
      for (int c1 = 0; c1 < D; ++c1)
#pragma unroll
        for (int c2 = 0; c2 < D; ++c2)
#pragma unroll
          for (int a1 = 0; a1 < D; ++a1)
#pragma unroll
            for (int a2 = 0; a2 < D; ++a2) {
              GT v = mu * Kt[a1][c2] * Kt[a2][c1] + lambda * Kt[a1][c1] * Kt[a2][c2];
              if (c1 == c2) v += mu * KK[a1][a2];
              g[(c1 * D + c2) * C::KRP + a1 * D + a2] = live ? dett * v : T(0);
            }
    }
#pragma unroll
    for (int b = 0; b < C::NB; ++b)
      for (int k = C::KR; k < C::KRP; ++k) g[b * C::KRP + k] = T(0);
  }
  __syncthreads();
  // ---- contraction: the thread's slots x the group's cells
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr bool DIAG = C::DIAG;
  constexpr int NPOS = DIAG ? D * D : D;  // element-tensor entries a slot writes per cell
  const int grp = C::NT >= C::NSL ? t / C::NSL : 0;
  const long long left = p.n_elem - e0;
  const int nc = int(left < C::E ? left : C::E);
  // R[(s1,s2)] . block
  auto contract = [&](const T* gblk, int j, const T* rrow) {
    const V* gv = reinterpret_cast<const V*>(gblk);
    T acc = T(0);
#pragma unroll
    for (int kv = 0; kv < C::KRP / C::VEC; ++kv) {
      const V x = gv[kv];
      T xs[C::VEC];
      if constexpr (sizeof(T) == 4) {
        xs[0] = x.x;
        xs[1] = x.y;
        xs[2] = x.z;
        xs[3] = x.w;
      } else {
        xs[0] = x.x;
        xs[1] = x.y;
      }
#pragma unroll
      for (int m = 0; m < C::VEC; ++m) {
        const int k = kv * C::VEC + m;
        if (k < C::KR) {
          if constexpr (C::REG_R) acc = fma(xs[m], br.rr[j][k < C::KR ? k : 0], acc);
          else acc = fma(xs[m], rrow[k], acc);
        }
      }
    }
    return acc;
  };
  using SG = BlockStaging<C, T, ASSEMBLE>;
  if constexpr (SG::ON) {
    // chunks of SG::CELLS cells; within a chunk the groups take cells grp, grp + GRP, ...
    T* stage = reinterpret_cast<T*>(smem + C::SMEM);
    for (int c0 = 0; c0 < nc; c0 += SG::CELLS) {
      const int b = *staged_chunks & 1;
      T* buf = stage + b * (SG::BUF / sizeof(T));
      if (*staged_chunks >= 2 && t == 0) bulk_wait_read<1>();  // the copy that last read buf is done
      __syncthreads();
      const int ncc = nc - c0 < SG::CELLS ? nc - c0 : SG::CELLS;
#pragma unroll
      for (int j = 0; j < C::PPT; ++j) {
        const int q = slot_of<C>(t, j);
        if (q < 0) continue;
        const int s2 = q % C::NS;
        const int s1 = DIAG ? q / C::NS : q / (C::NS * D);
        const int c2 = DIAG ? 0 : (q / C::NS) % D;
        const T* rrow = Rs + size_t(s1 * C::NS + s2) * C::KRP;
        for (int el = c0 + grp; el < c0 + ncc; el += C::GRP) {
          const T* gcell = Gs + size_t(el) * C::NB * C::KRP;
          T* cb = buf + size_t(el - c0) * C::NN;
          if constexpr (DIAG) {  // one value on the d diagonal positions
            const T v = contract(gcell, j, rrow);
#pragma unroll
            for (int c = 0; c < D; ++c) cb[(c * C::NS + s1) * C::N + c * C::NS + s2] = v;
          } else {  // the row slot's d entries ((c1, s1), (c2, s2))
#pragma unroll
            for (int c1 = 0; c1 < D; ++c1)
              cb[(c1 * C::NS + s1) * C::N + c2 * C::NS + s2] = contract(gcell + (c1 * D + c2) * C::KRP, j, rrow);
          }
        }
      }
      fence_async_smem();
      __syncthreads();
      if (t == 0) {
        bulk_s2g(static_cast<T*>(p.out) + (e0 + c0) * C::NN, buf, unsigned(ncc * C::NN * sizeof(T)));
        bulk_commit();
      }
      ++*staged_chunks;
    }
  } else {
#pragma unroll
    for (int j = 0; j < C::PPT; ++j) {
      const int q = slot_of<C>(t, j);
      if (q < 0) continue;
      int s1, s2, c2 = 0;
      if constexpr (DIAG) {
        s1 = q / C::NS;
        s2 = q % C::NS;
      } else {
        s2 = q % C::NS;
        c2 = (q / C::NS) % D;
        s1 = q / (C::NS * D);
      }
      const T* rrow = Rs + size_t(s1 * C::NS + s2) * C::KRP;
      // positions of the slot's entries: all d*d blocks (c1, c2) of the pair (convection),
      // or the d entries ((c1,s1),(c2,s2)) of the row slot (elasticity)
      int pos[NPOS];
      bool live_pos[NPOS];  // assembly: structural zeros add nothing
#pragma unroll
      for (int m = 0; m < NPOS; ++m) {
        const int c1 = DIAG ? m / D : m;
        const int cc2 = DIAG ? m % D : c2;
        pos[m] = (c1 * C::NS + s1) * C::N + cc2 * C::NS + s2;
        live_pos[m] = !DIAG || c1 == cc2;
      }
      // assembly: the slots of the next cell are loaded while this cell's atomics issue
      int sl_next[ASSEMBLE ? NPOS : 1];
      if constexpr (ASSEMBLE) {
#pragma unroll
        for (int m = 0; m < NPOS; ++m)
          sl_next[m] = (grp < nc && live_pos[m]) ? __ldg(p.slot + (e0 + grp) * C::NN + pos[m]) : -1;
      }
#pragma unroll 1
      for (int el = grp; el < nc; el += C::GRP) {
        const long long e = e0 + el;
        int sl[ASSEMBLE ? NPOS : 1];
        if constexpr (ASSEMBLE) {
          const int en = el + C::GRP;
#pragma unroll
          for (int m = 0; m < NPOS; ++m) {
            sl[m] = sl_next[m];
            sl_next[m] = (en < nc && live_pos[m]) ? __ldg(p.slot + (e0 + en) * C::NN + pos[m]) : -1;
          }
        }
        const T* gcell = Gs + size_t(el) * C::NB * C::KRP;
        T vdiag = T(0);
        if constexpr (DIAG) vdiag = contract(gcell, j, rrow);
#pragma unroll
        for (int m = 0; m < NPOS; ++m) {
          if (ASSEMBLE && !live_pos[m]) continue;
          const T v = DIAG ? (live_pos[m] ? vdiag : T(0)) : contract(gcell + (m * D + c2) * C::KRP, j, rrow);
          if constexpr (ASSEMBLE) {
            const int sv = sl[m];
            if (sv >= 0 && sv < p.nnz) atomicAdd(p.csr_val + sv, double(v));
            else atomicOr(p.status, FFC_FLAG_BOUNDS);
          } else {
            __stcs(static_cast<T*>(p.out) + e * C::NN + pos[m], v);
          }
        }
      }
    }
  }
  __syncthreads();
}

template <int D, int FORM, int Q, typename T, bool ASSEMBLE>
__global__ void __launch_bounds__(BlockCfg<D, FORM, Q, T>::NT, BlockCfg<D, FORM, Q, T>::MIN_BLOCKS)
    simt_block_kernel(SimtParams p) {
  using C = BlockCfg<D, FORM, Q, T>;
  using SG = BlockStaging<C, T, ASSEMBLE>;
  extern __shared__ __align__(16) unsigned char smem[];
  BlockRows<C, T> rows;
  block_rows_init<C, D, FORM, T>(p.a0, rows, smem);
  if constexpr (SG::ON) {  // the zero blocks of both staging buffers, written once
    T* stage = reinterpret_cast<T*>(smem + C::SMEM);
    for (size_t k = threadIdx.x; k < SG::BYTES / sizeof(T); k += C::NT) stage[k] = T(0);
  }
  int staged_chunks = 0;
  const long long n_tiles = (p.n_elem + C::E - 1) / C::E;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x)
    block_tile<C, D, FORM, Q, T, ASSEMBLE>(p, tile, smem, rows, &staged_chunks);
  if constexpr (SG::ON) {
    if (threadIdx.x == 0) bulk_wait_all();  // shared memory stays valid until the copies are done
  }
}

}  // namespace ffc
