// CUDA-core kernels for the tensor representation A^K_i = A0_{i alpha} G_K^alpha
// (Section 3.2, eq. (tensorproduct)) with an optional fused scatter into CSR
// (Section 2.2, Algorithm 2).
//
// One CTA processes tiles of E consecutive cells (persistent grid-stride loop):
//   phase 1  one thread per cell: FP64 geometry J, |det J|, J^{-1} and G_K -> shared
//            memory (cast to the contraction type T);
//   phase 2  the tile's E*n^2 outputs form one contiguous block of A_K. Thread t owns
//            the element-tensor entries i = ti + r*NTI (r < R) for cells
//            e = eg + k*EG, with t = eg*NTI + ti, so consecutive threads write
//            consecutive addresses. Each output is sum_alpha G[e][alpha] A0[i][alpha];
//            G is read from shared memory as a broadcast, A0 either sits in the
//            thread's registers (small |alpha| * R) or is streamed from the L1/L2-
//            resident transposed copy A0T[alpha][i], reused over KE cells.
//   epilogue store (tabulate) or atomic add at csr_val[slot] in FP64 (assemble).
#pragma once

#include <cstdint>
#include <type_traits>

#include "geometry.cuh"

namespace ffc {

// BLOCK = 0: the block size follows from n^2 (single-form kernels); BLOCK > 0: a fixed
// block size shared by several forms (the batched kernel), KE_T = cells per thread
// group per tile (0 = default).
template <int D, int FORM, int Q, typename T, int BLOCK = 0, int KE_T = 0, bool ASM = true>
struct SimtCfg {
  static constexpr int N = nlocal(FORM, D, Q);
  static constexpr int NN = N * N;
  static constexpr int NA = nalpha_k(FORM, D, Q);
  static constexpr bool PAIR = FORM == FFC_PAIR_MASS_POISSON;  // two outputs per entry
  static constexpr int VEC = 16 / int(sizeof(T));
  static constexpr int NAP = (NA + VEC - 1) / VEC * VEC;
  static constexpr int RMAX_THREADS = BLOCK > 0 ? BLOCK : 512;
  // symmetric forms on the FP64 pipe contract only the entries i1 <= i2 (Section 3.5:
  // a symmetric form needs fewer operations) and store each result at (i1, i2) and
  // (i2, i1); the FP32 paths stay HBM-bound on stores and keep the full, coalesced layout
  static constexpr bool SYMM =
      BLOCK == 0 && sizeof(T) == 8 && (FORM == FFC_POISSON || FORM == FFC_ELASTICITY);
  static constexpr int NE = SYMM ? N * (N + 1) / 2 : NN;  // entries contracted per cell
  // FP32 tabulate of the Poisson form with element tensors of 256 entries or more made of
  // whole 16-byte groups (P3 on tetrahedra): a thread owns four consecutive entries of each
  // cell and stores them at once, a quarter of the store instructions and their address
  // arithmetic (P3 0.295 -> 0.177 ms; mass P3 and the P2 tensors, measured, were a little
  // slower this way and keep one entry per thread)
  static constexpr bool VEC4 = BLOCK == 0 && !ASM && sizeof(T) == 4 && FORM == FFC_POISSON && NN % 4 == 0 &&
                               NN >= 256 && NN / 4 <= 512;
  static constexpr int R = VEC4 ? 4 : (NE + RMAX_THREADS - 1) / RMAX_THREADS;
  static constexpr int NTI = VEC4 ? NN / 4 : (NE + R - 1) / R;
  static constexpr int EG = BLOCK > 0 ? BLOCK / NTI : (NTI >= 256 ? 1 : 256 / NTI);
  static constexpr int NT = BLOCK > 0 ? BLOCK : NTI * EG;
  // register-resident reference tensor rows; a shared block size (several forms in one
  // kernel) keeps it only for small |alpha| so the kernel's register count stays low
  static constexpr bool REG_A0 = (R * NA * int(sizeof(T)) / 4) <= (BLOCK > 0 ? 32 : 96);
  // cells per thread group and tile, measured on tetrahedra: register path 64 for mass,
  // 128 for Poisson P1-P3 (its heavier geometry phase amortised over more stores);
  // element tensors above 512 entries (one thread group per CTA) 32, or 16 for mass
  static constexpr int KE_TARGET =
      KE_T > 0 ? KE_T : (REG_A0 ? ((R > 1 && !VEC4) ? (NA == 1 ? 16 : 32) : (NA > 1 ? 128 : 64)) : 16);
  static constexpr int KE = (KE_TARGET + EG - 1) / EG;
  static constexpr int E = EG * KE;
  static constexpr int NCOEF = (FORM == FFC_NS_CONVECTION) ? N : 0;
  static constexpr size_t SMEM = size_t(E) * NAP * sizeof(T) + size_t(E) * NCOEF * sizeof(double);
  // two resident CTAs per SM where the register-held reference tensor is small
  static constexpr int MIN_BLOCKS = (VEC4 || (REG_A0 && R * NA * int(sizeof(T)) / 4 <= 16)) ? 2 : 1;
};

struct SimtParams {
  const int32_t* cells;
  const double* vertices;
  long long n_vert;
  const double* coeffs;
  const void* a0;       // REG_A0: [NN][NA]; otherwise [NA][NN] (rows by element-tensor position)
  const void* a0b;      // mass + Poisson pair: the Poisson rows [NN][NA - 1] (a0: the mass rows [NN][1])
  double* csr_val2;     // mass + Poisson pair: the Poisson matrix (csr_val: the mass matrix)
  void* out;            // A_K [n_elem][NN]
  const int32_t* slot;  // [n_elem][NN]
  double* csr_val;
  long long nnz;
  long long n_elem;
  double mu, lambda;
  unsigned* status;
};

template <typename OutT>
__device__ __forceinline__ void put(OutT* p, OutT v) {
  __stcs(p, v);
}

// Element-tensor positions of contracted entry u: (u, u) for the full layout; for the
// symmetric one, u numbers the entries i1 <= i2 row by row (row i1 starts at
// i1*N - i1*(i1-1)/2) and the positions are i1*N + i2 and i2*N + i1.
template <class C>
__device__ __forceinline__ void entry_positions(int u, int& p1, int& p2) {
  if constexpr (C::SYMM) {
    constexpr int N = C::N;
    auto start = [](int i) { return i * N - i * (i - 1) / 2; };
    const float h = float(N) + 0.5f;
    int i1 = int(h - sqrtf(h * h - 2.0f * float(u)));
    i1 = i1 < 0 ? 0 : (i1 > N - 1 ? N - 1 : i1);
    while (i1 > 0 && start(i1) > u) --i1;
    while (i1 < N - 1 && start(i1 + 1) <= u) ++i1;
    const int i2 = i1 + (u - start(i1));
    p1 = i1 * N + i2;
    p2 = i2 * N + i1;
  } else {
    p1 = u;
    p2 = u;
  }
}

// Loads the thread's rows of the reference tensor into registers (register path). The
// mass + Poisson pair takes column 0 from the mass rows `a0` and the rest from the
// Poisson rows `a0b`.
template <class C, typename T>
__device__ __forceinline__ void load_a0_rows(const void* a0, int t, T (&a0r)[C::REG_A0 ? C::R : 1][C::REG_A0 ? C::NA : 1],
                                             const void* a0b = nullptr) {
  if constexpr (C::REG_A0) {
    const int ti = t % C::NTI;
    const T* A0 = static_cast<const T*>(a0);
    const T* A0b = static_cast<const T*>(a0b);
#pragma unroll
    for (int r = 0; r < C::R; ++r) {
      const int u = C::VEC4 ? 4 * ti + r : ti + r * C::NTI;
      int p1 = 0, p2 = 0;
      if (u < C::NE) entry_positions<C>(u, p1, p2);
#pragma unroll
      for (int a = 0; a < C::NA; ++a) {
        if constexpr (C::PAIR)
          a0r[r][a] = (u < C::NE) ? (a == 0 ? A0[p1] : A0b[size_t(p1) * (C::NA - 1) + a - 1]) : T(0);
        else
          a0r[r][a] = (u < C::NE) ? A0[size_t(p1) * C::NA + a] : T(0);
      }
    }
  }
}

// One tile of E cells: geometry into shared memory, then contraction and store or
// atomic scatter. Called by every thread of the block; contains block barriers.
template <class C, int D, int FORM, int Q, typename T, bool ASSEMBLE>
__device__ __forceinline__ void simt_tile(const SimtParams& p, long long tile, unsigned char* smem_raw,
                                          const T (&a0r)[C::REG_A0 ? C::R : 1][C::REG_A0 ? C::NA : 1]) {
  using OutT = T;
  T* Gs = reinterpret_cast<T*>(smem_raw);                                                // [E][NAP]
  double* Ws = reinterpret_cast<double*>(smem_raw + size_t(C::E) * C::NAP * sizeof(T));  // [E][NCOEF]
  const int t = threadIdx.x;
  const int ti = t % C::NTI;
  const int eg = t / C::NTI;
  {
    const long long e0 = tile * C::E;
    // ---- phase 1: geometry tensors of the tile's cells
    if constexpr (C::NCOEF > 0) {
      const long long lim = (p.n_elem - e0) * C::NCOEF;
      const double* src = p.coeffs + e0 * C::NCOEF;
      for (int k = t; k < C::E * C::NCOEF; k += C::NT) Ws[k] = (k < lim) ? __ldg(src + k) : 0.0;
      __syncthreads();
    }
    for (int el = t; el < C::E; el += C::NT) {
      const long long e = e0 + el;
      T* g = Gs + el * C::NAP;
      if (e < p.n_elem) {
        bool degenerate, bad_index;
        if constexpr (C::PAIR) {
          // mass G = |det J| (the value the mass kernel takes), then the Poisson G_K
          float K[D][D], det;
          cell_geometry_f32<D>(p.cells, p.vertices, p.n_vert, e, K, det, degenerate, bad_index);
          g[0] = det;
          geometry_tensor_f32<D, FFC_POISSON, Q, true>(K, det, nullptr, 0.0, 0.0, g + 1);
        } else if constexpr (sizeof(T) == 4 && FORM != FFC_MASS) {
          // FP32 contraction: FP64 J, adj(J), det J; K and G_K in FP32
          float K[D][D], det;
          cell_geometry_f32<D>(p.cells, p.vertices, p.n_vert, e, K, det, degenerate, bad_index);
          geometry_tensor_f32<D, FORM, Q, true>(K, det, Ws + el * C::NCOEF, p.mu, p.lambda, g);
        } else {
          double K[D][D] = {}, det;
          if constexpr (FORM == FFC_MASS) {  // G = |det J|: no inverse needed
            cell_det<D>(p.cells, p.vertices, p.n_vert, e, det, degenerate, bad_index);
          } else {
            cell_geometry<D>(p.cells, p.vertices, p.n_vert, e, K, det, degenerate, bad_index);
          }
          geometry_tensor_k<D, FORM, Q>(K, det, Ws + el * C::NCOEF, p.mu, p.lambda,
                                      [&](int a, double v) { g[a] = T(v); });
        }
        if (degenerate) atomicOr(p.status, FFC_FLAG_DEGENERATE);
        if (bad_index) atomicOr(p.status, FFC_FLAG_BOUNDS);
      } else {
#pragma unroll 1
        for (int a = 0; a < C::NA; ++a) g[a] = T(0);
      }
#pragma unroll
      for (int a = C::NA; a < C::NAP; ++a) g[a] = T(0);
    }
    __syncthreads();
    // ---- phase 2: contraction and epilogue (thread groups beyond EG idle)
    if (eg >= C::EG) {
    } else if constexpr (C::VEC4) {
      // entries 4*ti .. 4*ti+3 of each of the group's cells: one 16-byte store per cell
#pragma unroll 1
      for (int k = 0; k < C::KE; ++k) {
        const int el = eg + k * C::EG;
        const long long e = e0 + el;
        if (e >= p.n_elem) break;
        const T* g = Gs + el * C::NAP;
        T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int a = 0; a < C::NA; ++a) {
          const T gv = g[a];
#pragma unroll
          for (int r = 0; r < 4; ++r) acc[r] = fma(gv, a0r[r][a], acc[r]);
        }
        __stcs(reinterpret_cast<float4*>(static_cast<float*>(p.out) + e * C::NN + 4 * ti),
               make_float4(acc[0], acc[1], acc[2], acc[3]));
      }
    } else if constexpr (C::REG_A0) {
      // element-tensor positions of the thread's entries (two for an off-diagonal entry
      // of the symmetric layout)
      int pos1[C::R], pos2[C::R];
#pragma unroll
      for (int r = 0; r < C::R; ++r) {
        const int u = ti + r * C::NTI;
        pos1[r] = pos2[r] = -1;
        if (u < C::NE) entry_positions<C>(u, pos1[r], pos2[r]);
      }
      constexpr int NS_ = C::SYMM ? 2 : 1;  // slots per entry
      // assembly: the slots of the next cell are loaded while this cell's atomics issue
      int slot_next[ASSEMBLE ? C::R : 1][NS_];
      if constexpr (ASSEMBLE) {
        const long long e = e0 + eg;
#pragma unroll
        for (int r = 0; r < C::R; ++r) {
          const bool ok = e < p.n_elem && pos1[r] >= 0;
          slot_next[r][0] = ok ? __ldg(p.slot + e * C::NN + pos1[r]) : -1;
          if constexpr (C::SYMM) slot_next[r][1] = (ok && pos2[r] != pos1[r]) ? __ldg(p.slot + e * C::NN + pos2[r]) : -1;
        }
      }
#pragma unroll 1
      for (int k = 0; k < C::KE; ++k) {
        const int el = eg + k * C::EG;
        const long long e = e0 + el;
        if (e >= p.n_elem) break;
        int slot_cur[ASSEMBLE ? C::R : 1][NS_];
        if constexpr (ASSEMBLE) {
          const long long en = e + C::EG;
          const bool more = (k + 1 < C::KE) && (en < p.n_elem);
#pragma unroll
          for (int r = 0; r < C::R; ++r) {
            const bool ok = more && pos1[r] >= 0;
            slot_cur[r][0] = slot_next[r][0];
            slot_next[r][0] = ok ? __ldg(p.slot + en * C::NN + pos1[r]) : -1;
            if constexpr (C::SYMM) {
              slot_cur[r][1] = slot_next[r][1];
              slot_next[r][1] = (ok && pos2[r] != pos1[r]) ? __ldg(p.slot + en * C::NN + pos2[r]) : -1;
            }
          }
        }
        const T* g = Gs + el * C::NAP;
        T acc[C::R], acc2[C::PAIR ? C::R : 1];
#pragma unroll
        for (int r = 0; r < C::R; ++r) acc[r] = T(0);
        if constexpr (C::PAIR) {  // mass: column 0; Poisson: columns 1.., in the Poisson kernel's order
#pragma unroll
          for (int r = 0; r < C::R; ++r) {
            acc[r] = fma(g[0], a0r[r][0], T(0));
            acc2[r] = T(0);
          }
#pragma unroll
          for (int a = 1; a < C::NA; ++a) {
            const T gv = g[a];
#pragma unroll
            for (int r = 0; r < C::R; ++r) acc2[r] = fma(gv, a0r[r][a], acc2[r]);
          }
        } else {
#pragma unroll
          for (int a = 0; a < C::NA; ++a) {
            const T gv = g[a];
#pragma unroll
            for (int r = 0; r < C::R; ++r) acc[r] = fma(gv, a0r[r][a], acc[r]);
          }
        }
#pragma unroll
        for (int r = 0; r < C::R; ++r) {
          if (pos1[r] < 0) continue;
          if constexpr (ASSEMBLE) {
#pragma unroll
            for (int m = 0; m < NS_; ++m) {
              if (m == 1 && pos2[r] == pos1[r]) continue;
              const int s = slot_cur[r][m];
              if (s >= 0 && s < p.nnz) {
                atomicAdd(p.csr_val + s, double(acc[r]));
                if constexpr (C::PAIR) atomicAdd(p.csr_val2 + s, double(acc2[r]));
              } else {
                atomicOr(p.status, FFC_FLAG_BOUNDS);
              }
            }
          } else {
            put(static_cast<OutT*>(p.out) + e * C::NN + pos1[r], acc[r]);
            if (C::SYMM && pos2[r] != pos1[r]) put(static_cast<OutT*>(p.out) + e * C::NN + pos2[r], acc[r]);
          }
        }
      }
    } else {
      static_assert(!C::PAIR, "the mass + Poisson pair keeps its reference tensor rows in registers");
      const T* A0T = static_cast<const T*>(p.a0);
#pragma unroll 1
      for (int r = 0; r < C::R; ++r) {
        const int u = ti + r * C::NTI;
        if (u >= C::NE) break;
        int p1, p2;
        entry_positions<C>(u, p1, p2);
        T acc[C::KE];
#pragma unroll
        for (int k = 0; k < C::KE; ++k) acc[k] = T(0);
        // VEC alphas per step: one 16-byte shared-memory load of G feeds VEC FMAs
        using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
#pragma unroll 1
        for (int a0 = 0; a0 < C::NAP; a0 += C::VEC) {
          T av[C::VEC];
#pragma unroll
          for (int j = 0; j < C::VEC; ++j) av[j] = (a0 + j < C::NA) ? __ldg(A0T + size_t(a0 + j) * C::NN + p1) : T(0);
#pragma unroll
          for (int k = 0; k < C::KE; ++k) {
            const V gv = *reinterpret_cast<const V*>(Gs + (eg + k * C::EG) * C::NAP + a0);
            if constexpr (sizeof(T) == 4) {
              acc[k] = fma(gv.x, av[0], acc[k]);
              acc[k] = fma(gv.y, av[1], acc[k]);
              acc[k] = fma(gv.z, av[2], acc[k]);
              acc[k] = fma(gv.w, av[3], acc[k]);
            } else {
              acc[k] = fma(gv.x, av[0], acc[k]);
              acc[k] = fma(gv.y, av[1], acc[k]);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < C::KE; ++k) {
          const long long e = e0 + eg + k * C::EG;
          if (e < p.n_elem) {
#pragma unroll
            for (int m = 0; m < (C::SYMM ? 2 : 1); ++m) {
              if (m == 1 && p2 == p1) continue;
              const long long o = e * C::NN + (m == 0 ? p1 : p2);
              if constexpr (ASSEMBLE) {
                const int s = __ldg(p.slot + o);
                if (s >= 0 && s < p.nnz) atomicAdd(p.csr_val + s, double(acc[k]));
                else atomicOr(p.status, FFC_FLAG_BOUNDS);
              } else {
                put(static_cast<OutT*>(p.out) + o, acc[k]);
              }
            }
          }
        }
      }
    }
    __syncthreads();
  }
}

template <int D, int FORM, int Q, typename T, bool ASSEMBLE>
__global__ void __launch_bounds__(SimtCfg<D, FORM, Q, T, 0, 0, ASSEMBLE>::NT,
                                  SimtCfg<D, FORM, Q, T, 0, 0, ASSEMBLE>::MIN_BLOCKS)
    simt_tabulate_kernel(SimtParams p) {
  using C = SimtCfg<D, FORM, Q, T, 0, 0, ASSEMBLE>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T a0r[C::REG_A0 ? C::R : 1][C::REG_A0 ? C::NA : 1];
  load_a0_rows<C, T>(p.a0, threadIdx.x, a0r, p.a0b);
  const long long n_tiles = (p.n_elem + C::E - 1) / C::E;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x)
    simt_tile<C, D, FORM, Q, T, ASSEMBLE>(p, tile, smem_raw, a0r);
}

// Host-side launcher for one instantiation.
template <int D, int FORM, int Q, typename T, bool ASSEMBLE>
int launch_simt_one(const SimtParams& prm, const void* a0_rows, const void* a0_cols, cudaStream_t stream) {
  using C = SimtCfg<D, FORM, Q, T, 0, 0, ASSEMBLE>;
  auto kern = simt_tabulate_kernel<D, FORM, Q, T, ASSEMBLE>;
  int sms = 0, blocks_per_sm = 1;
  if (launch_config(reinterpret_cast<const void*>(kern), C::NT, C::SMEM, -1, &sms, &blocks_per_sm) != FFC_OK)
    return FFC_ECUDA;
  SimtParams p = prm;
  p.a0 = C::REG_A0 ? a0_rows : a0_cols;
  const long long n_tiles = (p.n_elem + C::E - 1) / C::E;
  long long grid = (long long)sms * blocks_per_sm;
  if (grid > n_tiles) grid = n_tiles;
  if (grid < 1) grid = 1;
  kern<<<unsigned(grid), C::NT, C::SMEM, stream>>>(p);
  return cudaPeekAtLastError() == cudaSuccess ? FFC_OK : FFC_ECUDA;
}

}  // namespace ffc
