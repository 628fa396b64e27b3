// FP64 contraction of the quadrature representation (Section 3.4) on the tensor cores by
// exact products of small-integer digits: the splitting of Ozaki, Ogita, Oishi and Rump,
// "Error-free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications" (Numer. Algorithms 59, 2012), with BF16 digits and
// FP32 accumulation in TMEM, whose sums are exact integers under the bound below (this
// target has no integer MMA).
//
// A_K[i] = sum_j A~0[i][j] G~_K[j]. Row i of A~0 is scaled by 2^e_i and column (cell) c of
// G~ by 2^e_c, powers of two not below the row's / column's largest magnitude, and each
// scaled value x (|x| <= 1) is written as a 56-bit fixed-point number in balanced base-128
// digits,
//   x = sgn(x) sum_{s=0}^{7} D_s 2^(-7 - 7s),  D_0 in [0, 128], D_s in [-64, 63] for s >= 1,
// read off F = round(|x| 2^56) plus 64 in every digit position below the first (its base-128
// digits are D_0 and D_s + 64). A digit has at most 8 significant bits, so it is exact in
// BF16 and a product of two digits is exact in FP32. The products D^A_s D^B_t with s + t = g
// share the weight 2^(-14 - 7g): for each g the tensor cores add them over j and over the
// pairs (s, t) into one FP32 accumulator, and every partial sum is an integer of magnitude
// below
//   K (2 * 135 * 64 + 6 * 64 * 64) < 2^24   (K <= 400),
// hence exact (pairs s + t <= 7: 36 products; D_0 may reach 135 when a column's scale, taken
// from an FP32 estimate of its largest value with a 2^-10 margin, is a little low). Then
//   A_K[i] = 2^(e_i + e_c - 63) (H 2^28 + L),  H = sum_{g<4} P_g 2^(7(3-g)),  L = sum_{g>=4} P_g 2^(7(7-g)),
// H and L exact 64-bit integers, converted to FP64 and added with one rounding. The digits
// beyond the eighth and the products with s + t >= 8 are below 2^-56 (2^(e_i + e_c)) K per
// entry, under FP64's own rounding of a K-term dot product.
//
// Kernel: 64 cells per tile (MMA N = 64, M = 128 entries), 384 threads: warps 0-3 form
// G~ in FP64 (two lanes per cell, half of each 48-column chunk each) and write its eight
// digit planes; 4-7 drain the eight TMEM accumulators (8 x 64 columns) into FP64 A_K; 8
// issues the MMAs; 9 streams the digit planes of A~0 in 16-column pieces; 10-11 form each
// cell's FP64 Jacobian coefficients and its column scale one tile ahead. The FP64 per-point
// geometry is the floor of this kernel (GB300's FP64 pipe); the contraction runs on the
// tensor cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "ffc_internal.h"
#include "quadrature.h"
#include "tc_common.cuh"

namespace ffc {
namespace {
namespace oz {
using namespace ffc::tc;

constexpr int OZ_S = 8;             // digit planes per operand (7 bits each)
constexpr int OZ_N = 64;            // cells per tile
constexpr int OZ_KB = 48;           // K columns per G~ chunk (whole points for n_g = 1, 3, 6)
constexpr int OZ_KA = 16;           // K columns per A~0 piece (one BF16 MMA K step)
constexpr int OZ_PIECES = OZ_KB / OZ_KA;
constexpr int OZ_ASTAGES = 3;
constexpr int OZ_THREADS = 384;
constexpr int OZ_PROD_WARPS = 4, OZ_DRAIN_WARP0 = 4, OZ_MMA_WARP = 8, OZ_TMA_WARP = 9, OZ_GEO_WARP0 = 10;
constexpr int OZ_GEO_THREADS = OZ_THREADS - 32 * OZ_GEO_WARP0;  // one per cell of a tile
constexpr int OZ_KMAX = 400;
constexpr uint32_t OZ_APLANE = M_TILE * OZ_KA * 2;  // bytes of one digit plane of a piece
constexpr uint32_t OZ_ASTAGE = OZ_S * OZ_APLANE;
constexpr uint32_t OZ_BPLANE = OZ_N * OZ_KB * 2;    // bytes of one digit plane of a chunk
constexpr uint32_t OZ_BSTAGE = OZ_S * OZ_BPLANE;
constexpr int OZ_NBARS = 18;
// 64 in every digit position below the first: sum_{s=1}^{7} 64 * 2^(49 - 7s)
constexpr unsigned long long OZ_OFF = 64ull * ((1ull << 42) + (1ull << 35) + (1ull << 28) + (1ull << 21) +
                                               (1ull << 14) + (1ull << 7) + 1ull);
static_assert(OZ_N == OZ_GEO_THREADS && 2 * OZ_N == 32 * OZ_PROD_WARPS, "one geometry thread, two producers per cell");

using quad::det_adj;
using quad::qpair;

template <int D, int FORM, int G>
struct OzCfg {
  static constexpr int NG = FORM == FFC_MASS ? 1 : D * (D + 1) / 2;
  static constexpr int PPC = OZ_KB / NG;  // points per chunk
  static constexpr int PPH = PPC / 2;     // points per producer lane and chunk
  static constexpr int NGEO = G == 1 ? D + 1 : (D + 1) * (D + 2) / 2;
  // F'(X)[a][b] = J0[a][b] + sum_c H[a][(b,c)] X_c (affine in X for geometry degree <= 2)
  static constexpr int NH = G == 2 ? D * (D + 1) / 2 : 0;
  static constexpr int NJ = D * D + D * NH;
  static_assert(OZ_KB % NG == 0 && PPC % 2 == 0, "chunk of whole points, split in two");
  // table (doubles): [NGEO][D] dPsi(0), [NGEO][NH] second derivatives, [nq][D] points;
  // then the row exponents e_i [128]
  static constexpr size_t table_doubles(int nq) { return size_t(NGEO) * D + size_t(NGEO) * NH + size_t(nq) * D; }
  static constexpr size_t off_table() { return size_t(OZ_ASTAGES) * OZ_ASTAGE + 2 * size_t(OZ_BSTAGE); }
  static constexpr size_t off_x32(int nq) { return off_table() + table_doubles(nq) * 8; }
  static constexpr size_t off_cell(int nq) { return off_x32(nq) + (size_t(nq) * D * 4 + 15) / 16 * 16; }
  // cell slot: J0/H [NJ][64] doubles, degenerate thresholds [64] doubles, scale exponents [64] ints
  static constexpr size_t off_tau(int nq) { return off_cell(nq) + size_t(NJ + 1) * OZ_N * 8 + OZ_N * 4; }
  static constexpr size_t off_bars(int nq) { return off_tau(nq) + 2 * OZ_N * 4; }
  static constexpr size_t smem_bytes(int nq) { return off_bars(nq) + OZ_NBARS * 8 + 16; }
};

struct OzParams {
  const int32_t* cells;
  const double* nodes;
  long long n_nodes, n_elem;
  const double* table;   // see OzCfg::table_doubles, then e_i [128]
  const void* a_digits;  // [pieces][8 planes][128 x 16] BF16, core-matrix layout
  double* out;           // A_K [n_elem][nn], or (slot set) CSR values csr_val[slot] += A_K
  const int32_t* slot;
  double* csr_val;
  long long nnz;
  int nn, nq, nch;
  unsigned* status;
};

__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t phase, volatile int* abort_flag) {
  const bool ok = mbar_wait_or_abort(bar, phase, abort_flag);
  return __all_sync(0xffffffffu, ok);
}

// G~ entries of one point from its Jacobian: mass |det|, Poisson adj adj^T / |det| in the
// pair order (diagonal first, then (0,1) [, (0,2), (1,2)])
template <int D, int FORM, typename T>
__device__ __forceinline__ T point_values(const T (&J)[D][D], T* v) {
  T A[D][D];
  const T det = det_adj<D, T>(J, A);
  T ad;
  if constexpr (sizeof(T) == 8) ad = __longlong_as_double(__double_as_longlong(det) & 0x7FFFFFFFFFFFFFFFll);
  else ad = fabsf(det);
  if constexpr (FORM == FFC_MASS) {
    v[0] = ad;
  } else {
    T r;
    if constexpr (sizeof(T) == 8) r = __drcp_rn(ad);
    else r = __frcp_rn(ad);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = a; b < D; ++b) {
        T sq = T(0);
#pragma unroll
        for (int cc = 0; cc < D; ++cc) sq = fma(A[a][cc], A[b][cc], sq);
        v[qpair<D>(a, b)] = sq * r;
      }
  }
  return ad;
}

// round(|x| 2^(56 - ec)) in integer arithmetic, for |x| <= 2^ec (1 + 7 * 2^-7); larger
// magnitudes (and inf, NaN) are clamped to 2^56 and reported through `over`
__device__ __forceinline__ unsigned long long oz_fixed(double x, int ec, bool& over) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull;
  const int E = int(b >> 52);
  if (E == 0) return 0ull;  // zero, or below 2^-1022
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = E - 1075 + 56 - ec;  // F = m 2^sh
  unsigned long long F;
  if (sh >= 0) {
    if (sh > 4) {
      over = true;
      return 1ull << 56;
    }
    F = m << sh;
  } else if (sh > -64) {
    F = (m + (1ull << (-sh - 1))) >> (-sh);
  } else {
    F = 0ull;
  }
  if (F > (1ull << 56) + (7ull << 49)) {
    over = true;
    F = 1ull << 56;
  }
  return F;
}

// digit t of the offset fixed-point value Fp = F + OZ_OFF: D_0 = Fp >> 49, D_t = ((Fp >> (49 -
// 7t)) & 127) - 64
template <int T>
__device__ __forceinline__ int oz_digit(unsigned long long Fp) {
  if constexpr (T == 0) return int(Fp >> 49);
  else return int((Fp >> (49 - 7 * T)) & 127ull) - 64;
}

// v 2^E by multiplications with normal powers of two (one when 2^E is normal)
__device__ __forceinline__ double oz_scale(double v, int E) {
  if (E >= -1022 && E <= 1023) return v * __longlong_as_double(static_cast<long long>(E + 1023) << 52);
  const int E1 = max(-1022, min(1023, E));
  const int E2 = max(-1022, min(1023, E - E1));
  const double p1 = __longlong_as_double(static_cast<long long>(E1 + 1023) << 52);
  const double p2 = __longlong_as_double(static_cast<long long>(E2 + 1023) << 52);
  return v * p1 * p2;
}

template <int D, int FORM, int G>
__global__ void __launch_bounds__(OZ_THREADS, 1) oz_kernel(OzParams p) {
  using C = OzCfg<D, FORM, G>;
  constexpr int NG = C::NG, NGEO = C::NGEO, NH = C::NH, NJ = C::NJ;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* As = smem;                                    // OZ_ASTAGES x OZ_ASTAGE
  unsigned char* Bs = smem + OZ_ASTAGES * OZ_ASTAGE;           // 2 x OZ_BSTAGE
  double* tab = reinterpret_cast<double*>(smem + C::off_table());
  const double* g0 = tab;                                      // [NGEO][D]
  const double* hs = tab + NGEO * D;                           // [NGEO][NH]
  const double* xq = hs + NGEO * NH;                           // [nq][D]
  float* xq32 = reinterpret_cast<float*>(smem + C::off_x32(p.nq));  // [nq][D]
  double* cellj = reinterpret_cast<double*>(smem + C::off_cell(p.nq));  // [NJ][64]
  double* thr_s = cellj + NJ * OZ_N;                           // [64]
  int* ec_s = reinterpret_cast<int*>(thr_s + OZ_N);            // [64]
  int* tau_s = reinterpret_cast<int*>(smem + C::off_tau(p.nq));  // [2][64]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::off_bars(p.nq));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + OZ_NBARS);
  __shared__ int abort_flag;
  constexpr int A_FULL = 0, A_EMPTY = 3, B_FULL = 6, B_EMPTY = 8, ACC_FULL = 10, ACC_EMPTY = 11, GEO_FULL = 12,
                GEO_EMPTY = 13, TAU_FULL = 14, TAU_EMPTY = 16;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  auto bar = [&](int k) { return smem_u32(&bars[k]); };
  const int ntab = int(C::table_doubles(p.nq));
  for (int i = t; i < ntab; i += OZ_THREADS) tab[i] = p.table[i];
  for (int i = t; i < p.nq * D; i += OZ_THREADS) xq32[i] = float(p.table[NGEO * D + NGEO * NH + i]);
  if (t == 0) {
    for (int k = 0; k < OZ_ASTAGES; ++k) {
      mbar_init(bar(A_FULL + k), 1);
      mbar_init(bar(A_EMPTY + k), 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(bar(B_FULL + k), OZ_PROD_WARPS);
      mbar_init(bar(B_EMPTY + k), 1);
      mbar_init(bar(TAU_FULL + k), OZ_PROD_WARPS);
      mbar_init(bar(TAU_EMPTY + k), 4);
    }
    mbar_init(bar(ACC_FULL), 1);
    mbar_init(bar(ACC_EMPTY), 4);
    mbar_init(bar(GEO_FULL), OZ_GEO_THREADS / 32);
    mbar_init(bar(GEO_EMPTY), OZ_PROD_WARPS);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const long long n_tiles = (p.n_elem + OZ_N - 1) / OZ_N;
  const long long my_tiles = blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int npieces = p.nch * OZ_PIECES;
  if (warp == OZ_TMA_WARP) {
    // ---------------------------------------------------------------- digit planes of A~0
    if (lane == 0) {
      bool ok = true;
      const long long total = my_tiles * npieces;
      for (long long g = 0; g < total && ok; ++g) {
        const int s = int(g % OZ_ASTAGES);
        if (g >= OZ_ASTAGES)
          ok = mbar_wait_or_abort(bar(A_EMPTY + s), uint32_t(g / OZ_ASTAGES - 1) & 1u, &abort_flag);
        if (!ok) break;
        mbar_expect_tx(bar(A_FULL + s), OZ_ASTAGE);
        bulk_g2s(smem_u32(As + s * OZ_ASTAGE),
                 static_cast<const unsigned char*>(p.a_digits) + size_t(g % npieces) * OZ_ASTAGE, OZ_ASTAGE,
                 bar(A_FULL + s));
      }
      if (!ok) {
        atomicOr(p.status, FFC_FLAG_TIMEOUT);
        abort_flag = 1;
      }
    }
  } else if (warp == OZ_MMA_WARP) {
    // ---------------------------------------------------------------- 36 digit products per piece
    if (lane == 0) {
      constexpr uint32_t IDESC = mma_idesc(false, M_TILE, OZ_N);
      bool ok = true;
      long long ga = 0, gb = 0;
      for (long long ct = 0; ct < my_tiles && ok; ++ct) {
        if (ct >= 1) ok = mbar_wait_or_abort(bar(ACC_EMPTY), uint32_t(ct - 1) & 1u, &abort_flag);
        for (int c = 0; c < p.nch && ok; ++c, ++gb) {
          const int sb = int(gb & 1);
          ok = mbar_wait_or_abort(bar(B_FULL + sb), uint32_t(gb >> 1) & 1u, &abort_flag);
          for (int j = 0; j < OZ_PIECES && ok; ++j, ++ga) {
            const int sa = int(ga % OZ_ASTAGES);
            ok = mbar_wait_or_abort(bar(A_FULL + sa), uint32_t(ga / OZ_ASTAGES) & 1u, &abort_flag);
            if (!ok) break;
            fence_after();
#pragma unroll
            for (int s = 0; s < OZ_S; ++s) {
              const uint64_t da = smem_desc(smem_u32(As + sa * OZ_ASTAGE + s * OZ_APLANE), 128, 2 * 128);
#pragma unroll
              for (int tt = 0; tt < OZ_S - s; ++tt) {
                const uint64_t db =
                    smem_desc(smem_u32(Bs + sb * OZ_BSTAGE + tt * OZ_BPLANE) + j * 256, 128, (OZ_KB / 8) * 128);
                mma<true>(tmem + uint32_t((s + tt) * OZ_N), da, db, IDESC, (c == 0 && j == 0 && s == 0) ? 0u : 1u);
              }
            }
            mma_commit(bar(A_EMPTY + sa));
          }
          if (ok) mma_commit(bar(B_EMPTY + sb));
        }
        if (ok) mma_commit(bar(ACC_FULL));
      }
      if (!ok) {
        atomicOr(p.status, FFC_FLAG_TIMEOUT);
        abort_flag = 1;
      }
      if (ga > 0) mbar_wait(bar(A_EMPTY + int((ga - 1) % OZ_ASTAGES)), uint32_t((ga - 1) / OZ_ASTAGES) & 1u);
    }
  } else if (warp >= OZ_GEO_WARP0) {
    // ---------------------------------------------------------------- per-cell coefficients and scale
    const int c = t - 32 * OZ_GEO_WARP0;
    bool ok = true;
    for (long long ct = 0; ct < my_tiles && ok; ++ct) {
      const long long e = (blockIdx.x + ct * gridDim.x) * OZ_N + c;
      const bool live = e < p.n_elem;
      long long id0 = live ? p.cells[e * NGEO] : 0;
      if (id0 < 0 || id0 >= p.n_nodes) {
        atomicOr(p.status, FFC_FLAG_BOUNDS);
        id0 = 0;
      }
      double x0[D];
#pragma unroll
      for (int a = 0; a < D; ++a) x0[a] = p.nodes[id0 * D + a];
      double cj[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) cj[j] = 0.0;
      double h2 = 0.0;
#pragma unroll
      for (int nd = 1; nd < NGEO; ++nd) {
        long long id = live ? p.cells[e * NGEO + nd] : id0;
        if (id < 0 || id >= p.n_nodes) {
          atomicOr(p.status, FFC_FLAG_BOUNDS);
          id = id0;
        }
        double xr[D], sq = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          xr[a] = p.nodes[id * D + a] - x0[a];
          sq = fma(xr[a], xr[a], sq);
        }
        if (nd <= D) h2 = fmax(h2, sq);
#pragma unroll
        for (int a = 0; a < D; ++a) {
#pragma unroll
          for (int b = 0; b < D; ++b) cj[a * D + b] = fma(xr[a], g0[nd * D + b], cj[a * D + b]);
#pragma unroll
          for (int h = 0; h < NH; ++h) cj[D * D + a * NH + h] = fma(xr[a], hs[nd * NH + h], cj[D * D + a * NH + h]);
        }
      }
      const double thr = 1e-14 * (D == 2 ? h2 : h2 * sqrt(h2));
      // the column's scale: an FP32 estimate of its largest |G~| over the points, with a
      // 2^-10 margin, rounded up to a power of two. The estimate runs on the coefficients
      // times 2^-eh (2^eh about the cell's size h), which keeps it inside FP32's range for
      // any cell size; G~ of the map scaled by l is l^D G~ (mass) or l^(D-2) G~ (Poisson),
      // so the exponent found is shifted back by eh times that power.
      int eh = 0;
      if (h2 > 0.0 && h2 < DBL_MAX) {
        frexp(h2, &eh);
        eh /= 2;
      }
      const double down = __longlong_as_double(static_cast<long long>(1023 - eh) << 52);
      float c32[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) c32[j] = float(cj[j] * down);
      float mx = 0.f;
      const int npts = G == 1 ? 1 : p.nq;
      for (int k = 0; k < npts; ++k) {
        float J[D][D], v[NG];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b) {
            float x = c32[a * D + b];
#pragma unroll
            for (int cc = 0; cc < D; ++cc)
              if constexpr (NH > 0) x = fmaf(c32[D * D + a * NH + qpair<D>(b, cc)], xq32[k * D + cc], x);
            J[a][b] = x;
          }
        point_values<D, FORM, float>(J, v);
#pragma unroll
        for (int gg = 0; gg < NG; ++gg) mx = fmaxf(mx, fabsf(v[gg]));
      }
      int ec = 0;
      if (mx > 0.f && mx <= FLT_MAX) {
        frexp(double(mx) * (1.0 + 0.0009765625), &ec);
        ec += eh * (FORM == FFC_MASS ? D : D - 2);
      }
      if (ct >= 1) ok = warp_wait(bar(GEO_EMPTY), uint32_t(ct - 1) & 1u, &abort_flag);
      if (!ok) break;
#pragma unroll
      for (int j = 0; j < NJ; ++j) cellj[j * OZ_N + c] = cj[j];
      thr_s[c] = thr;
      ec_s[c] = ec;
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(GEO_FULL));
    }
    if (!ok) {
      if (lane == 0) atomicOr(p.status, FFC_FLAG_TIMEOUT);
      abort_flag = 1;
    }
  } else if (warp < OZ_PROD_WARPS) {
    // ---------------------------------------------------------------- G~ digit planes
    // lanes 0-7 / 8-15 take cells 0-7 of the warp's 16 (first / second half of the chunk's
    // columns), lanes 16-31 cells 8-15: every 8-lane phase of a 16-byte store writes eight
    // rows of one core matrix
    const int c = warp * 16 + (lane & 7) + ((lane >> 4) << 3), hlf = (lane >> 3) & 1;
    bool ok = true;
    long long gb = 0;
    for (long long ct = 0; ct < my_tiles && ok; ++ct) {
      ok = warp_wait(bar(GEO_FULL), uint32_t(ct) & 1u, &abort_flag);
      if (!ok) break;
      const int ec = ec_s[c];
      const double thr = thr_s[c];
      const long long e = (blockIdx.x + ct * gridDim.x) * OZ_N + c;
      const bool live = e < p.n_elem;
      if (ct >= 2) ok = warp_wait(bar(TAU_EMPTY + int(ct & 1)), uint32_t((ct - 2) >> 1) & 1u, &abort_flag);
      if (!ok) break;
      if (hlf == 0) tau_s[int(ct & 1) * OZ_N + c] = ec;
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(TAU_FULL + int(ct & 1)));
      bool degenerate = false, over = false;
      double gconst[NG];  // geometry degree 1: the same G~ at every point
      if constexpr (G == 1) {
        double J[D][D];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b) J[a][b] = cellj[(a * D + b) * OZ_N + c];
        const double ad = point_values<D, FORM, double>(J, gconst);
        if (!(__double_as_longlong(ad) > __double_as_longlong(thr))) degenerate = true;
      }
      for (int ch = 0; ch < p.nch && ok; ++ch, ++gb) {
        const int sb = int(gb & 1);
        if (gb >= 2) ok = warp_wait(bar(B_EMPTY + sb), uint32_t((gb - 2) >> 1) & 1u, &abort_flag);
        if (!ok) break;
        unsigned long long fp[OZ_KB / 2];
        unsigned neg = 0u;
#pragma unroll
        for (int pp = 0; pp < C::PPH; ++pp) {
          const int k = ch * C::PPC + hlf * C::PPH + pp;
          double v[NG];
          if (!live || k >= p.nq) {
#pragma unroll
            for (int gg = 0; gg < NG; ++gg) v[gg] = 0.0;
          } else if constexpr (G == 1) {
#pragma unroll
            for (int gg = 0; gg < NG; ++gg) v[gg] = gconst[gg];
          } else {
            double J[D][D];
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
              for (int b = 0; b < D; ++b) {
                double x = cellj[(a * D + b) * OZ_N + c];
#pragma unroll
                for (int cc = 0; cc < D; ++cc)
                  x = fma(cellj[(D * D + a * NH + qpair<D>(b, cc)) * OZ_N + c], xq[k * D + cc], x);
                J[a][b] = x;
              }
            const double ad = point_values<D, FORM, double>(J, v);
            // |det| and the threshold are non-negative: their bit patterns order them (a NaN
            // |det| saturates in oz_fixed and is reported there)
            if (!(__double_as_longlong(ad) > __double_as_longlong(thr))) degenerate = true;
          }
#pragma unroll
          for (int gg = 0; gg < NG; ++gg) {
            const int col = pp * NG + gg;
            fp[col] = oz_fixed(v[gg], ec, over) + OZ_OFF;
            if (__double_as_longlong(v[gg]) < 0) neg |= 1u << col;
          }
        }
        // eight digit planes of this lane's half of the cell's chunk row, 16 bytes at a time
        unsigned char* bs = Bs + sb * OZ_BSTAGE;
        auto plane = [&](auto tc) {
          constexpr int T = decltype(tc)::value;
#pragma unroll
          for (int kc = 0; kc < OZ_KB / 16; ++kc) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int c0 = kc * 8 + 2 * q, c1 = c0 + 1;
              int d0 = oz_digit<T>(fp[c0]), d1 = oz_digit<T>(fp[c1]);
              if ((neg >> c0) & 1u) d0 = -d0;
              if ((neg >> c1) & 1u) d1 = -d1;
              const __nv_bfloat162 h = __floats2bfloat162_rn(float(d0), float(d1));
              memcpy(&w[q], &h, 4);
            }
            const uint32_t o = core_offset(c, (hlf * (OZ_KB / 16) + kc) * 8, OZ_KB / 8, 8) * 2;
            *reinterpret_cast<uint4*>(bs + T * OZ_BPLANE + o) = make_uint4(w[0], w[1], w[2], w[3]);
          }
        };
        plane(std::integral_constant<int, 0>{});
        plane(std::integral_constant<int, 1>{});
        plane(std::integral_constant<int, 2>{});
        plane(std::integral_constant<int, 3>{});
        plane(std::integral_constant<int, 4>{});
        plane(std::integral_constant<int, 5>{});
        plane(std::integral_constant<int, 6>{});
        plane(std::integral_constant<int, 7>{});
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_FULL + sb));
      }
      // the cell slot is read at every point: released once the tile's chunks are written
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(GEO_EMPTY));
      if (live && degenerate) atomicOr(p.status, FFC_FLAG_DEGENERATE);
      if (live && over) atomicOr(p.status, FFC_FLAG_DEGENERATE);
    }
    if (!ok) {
      if (lane == 0) atomicOr(p.status, FFC_FLAG_TIMEOUT);
      abort_flag = 1;
    }
  } else {
    // ---------------------------------------------------------------- drainers: TMEM -> FP64 A_K
    const int q4 = warp - OZ_DRAIN_WARP0;  // TMEM lanes 32 q4 .. 32 q4 + 31
    const int i = q4 * 32 + lane;          // element-tensor entry
    const int ei = i < p.nn ? int(p.table[C::table_doubles(p.nq) + i]) : 0;
    bool ok = true;
    for (long long ct = 0; ct < my_tiles && ok; ++ct) {
      ok = warp_wait(bar(ACC_FULL), uint32_t(ct) & 1u, &abort_flag) &&
           warp_wait(bar(TAU_FULL + int(ct & 1)), uint32_t(ct >> 1) & 1u, &abort_flag);
      if (!ok) break;
      fence_after();
      const int* tau = tau_s + int(ct & 1) * OZ_N;
      const long long e0 = (blockIdx.x + ct * gridDim.x) * OZ_N;
      const uint32_t taddr = tmem + (uint32_t(q4 * 32) << 16);
#pragma unroll 1
      for (int cb = 0; cb < OZ_N / 8; ++cb) {
        uint32_t r[OZ_S][8];
#pragma unroll
        for (int g = 0; g < OZ_S; ++g) tmem_ld8_issue(taddr + uint32_t(g * OZ_N + cb * 8), r[g]);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          long long P[OZ_S];
#pragma unroll
          for (int g = 0; g < OZ_S; ++g) P[g] = __float2int_rn(__uint_as_float(r[g][j]));
          const long long H = P[0] * 2097152ll + P[1] * 16384ll + P[2] * 128ll + P[3];
          const long long L = P[4] * 2097152ll + P[5] * 16384ll + P[6] * 128ll + P[7];
          const double v = oz_scale(fma(double(H), 268435456.0, double(L)), ei + tau[cb * 8 + j] - 63);
          const long long e = e0 + cb * 8 + j;
          if (i < p.nn && e < p.n_elem) {
            if (p.slot) {  // Algorithm 2: FP64 atomic add into the CSR values
              const int sl = __ldg(p.slot + e * p.nn + i);
              if (sl >= 0 && sl < p.nnz) atomicAdd(p.csr_val + sl, v);
              else atomicOr(p.status, FFC_FLAG_BOUNDS);
            } else {
              __stcs(p.out + e * p.nn + i, v);
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(bar(ACC_EMPTY));
        mbar_arrive(bar(TAU_EMPTY + int(ct & 1)));
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

int oz_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return FFC_ECUDA;
}

// Host: the digit planes of A~0 (row scales 2^e_i, e_i the exponent of the row's largest
// magnitude rounded up to a power of two) and the producers' geometry table.
int upload_oz(ffc_qform* f, ffc_qform::Dev* dv, int nch) {
  std::lock_guard<std::mutex> g(f->lock);
  if (dv->oz_a && dv->oz_table) return FFC_OK;
  const int nn = f->n * f->n, K = f->K, d = f->d;
  const int pieces = nch * OZ_PIECES;
  const size_t per_piece = size_t(OZ_S) * M_TILE * OZ_KA;  // BF16 elements
  std::vector<uint16_t> planes(per_piece * pieces, 0);
  std::vector<double> erow(M_TILE, 0.0);
  for (int i = 0; i < nn; ++i) {
    double mx = 0.0;
    for (int j = 0; j < K; ++j) mx = std::max(mx, std::fabs(f->At[size_t(i) * K + j]));
    int e = 0;
    if (mx > 0.0) std::frexp(mx, &e);  // mx < 2^e
    erow[i] = e;
    for (int j = 0; j < K; ++j) {
      const double x = f->At[size_t(i) * K + j];
      const unsigned long long F = static_cast<unsigned long long>(std::llround(std::ldexp(std::fabs(x), 56 - e)));
      const unsigned long long Fp = F + OZ_OFF;
      const size_t base = size_t(j / OZ_KA) * per_piece + core_offset(i, j % OZ_KA, OZ_KA / 8, 8);
      for (int s = 0; s < OZ_S; ++s) {
        int dig = s == 0 ? int(Fp >> 49) : int((Fp >> (49 - 7 * s)) & 127ull) - 64;
        if (x < 0.0) dig = -dig;
        planes[base + size_t(s) * M_TILE * OZ_KA] = host_bf16_bits(double(dig));
      }
    }
  }
  // the geometry table, then e_i [128]
  std::vector<double> tab = quad::geometry_table(f);
  tab.insert(tab.end(), erow.begin(), erow.end());
  cudaError_t e = cudaSuccess;
  void* a = nullptr;
  double* tb = nullptr;
  if ((e = cudaMalloc(&a, planes.size() * 2)) != cudaSuccess ||
      (e = cudaMemcpy(a, planes.data(), planes.size() * 2, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMalloc(&tb, tab.size() * sizeof(double))) != cudaSuccess ||
      (e = cudaMemcpy(tb, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) {
    cudaFree(a);
    cudaFree(tb);
    return oz_fail(e, "ffc_tabulate_quadrature: digit planes");
  }
  dv->oz_a = a;
  dv->oz_table = tb;
  return FFC_OK;
}

template <int D, int FORM, int G>
int launch_oz(ffc_qform* f, ffc_qform::Dev* dv, long long n_elem, const int32_t* cells, const double* nodes,
              long long n_nodes, const QOut& o, unsigned* status, cudaStream_t s) {
  using C = OzCfg<D, FORM, G>;
  const int nch = (f->K + OZ_KB - 1) / OZ_KB;
  const size_t smem = C::smem_bytes(f->nq);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > size_t(optin)) {
    set_error("ffc_tabulate_quadrature: the rule's points do not fit next to the digit planes");
    return FFC_EUNSUPPORTED;
  }
  int rc = upload_oz(f, dv, nch);
  if (rc != FFC_OK) return rc;
  OzParams p{};
  p.cells = cells;
  p.nodes = nodes;
  p.n_nodes = n_nodes;
  p.n_elem = n_elem;
  p.table = dv->oz_table;
  p.a_digits = dv->oz_a;
  p.out = static_cast<double*>(o.out);
  p.slot = o.slot;
  p.csr_val = o.csr_val;
  p.nnz = o.nnz;
  p.nn = f->n * f->n;
  p.nq = f->nq;
  p.nch = nch;
  p.status = status;
  auto kern = oz_kernel<D, FORM, G>;
  int sms = 0;
  if (launch_config(reinterpret_cast<const void*>(kern), OZ_THREADS, smem, -1, &sms, nullptr) != FFC_OK)
    return FFC_ECUDA;
  const long long n_tiles = (n_elem + OZ_N - 1) / OZ_N;
  const long long grid = std::min<long long>(sms, n_tiles);
  kern<<<unsigned(std::max<long long>(grid, 1)), OZ_THREADS, smem, s>>>(p);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FFC_OK : oz_fail(e, "oz_kernel launch");
}

}  // namespace oz
}  // namespace

int ozaki_supported(const ffc_qform* f) {
  if (f->n * f->n > tc::M_TILE) {
    set_error("ffc_tabulate_quadrature: FFC_FP64_OZAKI takes element tensors of at most 128 entries");
    return FFC_EUNSUPPORTED;
  }
  if (f->K > oz::OZ_KMAX) {
    set_error("ffc_tabulate_quadrature: FFC_FP64_OZAKI takes contractions of at most 400 terms (points x "
              "geometry entries); lower the quadrature degree");
    return FFC_EUNSUPPORTED;
  }
  return FFC_OK;
}

int run_ozaki(ffc_qform* f, ffc_qform::Dev* dv, long long n_elem, const int32_t* cells, const double* nodes,
              long long n_nodes, const QOut& out, unsigned* status, cudaStream_t s) {
  const bool mass = f->kind == FFC_MASS;
  if (f->d == 2) {
    if (f->g == 1)
      return mass ? oz::launch_oz<2, FFC_MASS, 1>(f, dv, n_elem, cells, nodes, n_nodes, out, status, s)
                  : oz::launch_oz<2, FFC_POISSON, 1>(f, dv, n_elem, cells, nodes, n_nodes, out, status, s);
    return mass ? oz::launch_oz<2, FFC_MASS, 2>(f, dv, n_elem, cells, nodes, n_nodes, out, status, s)
                : oz::launch_oz<2, FFC_POISSON, 2>(f, dv, n_elem, cells, nodes, n_nodes, out, status, s);
  }
  if (f->g == 1)
    return mass ? oz::launch_oz<3, FFC_MASS, 1>(f, dv, n_elem, cells, nodes, n_nodes, out, status, s)
                : oz::launch_oz<3, FFC_POISSON, 1>(f, dv, n_elem, cells, nodes, n_nodes, out, status, s);
  return mass ? oz::launch_oz<3, FFC_MASS, 2>(f, dv, n_elem, cells, nodes, n_nodes, out, status, s)
              : oz::launch_oz<3, FFC_POISSON, 2>(f, dv, n_elem, cells, nodes, n_nodes, out, status, s);
}

}  // namespace ffc
