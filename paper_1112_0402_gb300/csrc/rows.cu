// Row-owner assembly: Algorithm 2 (Section 2.2) with its loops ordered by global row.
//
// Algorithm 2 adds each element tensor into the global matrix, A[iota(i1), iota(i2)] +=
// A^K[i1][i2]; done cell by cell on a GPU, every addition is a global FP64 atomic and the
// matrix must be zeroed first. Here the same sums are taken row by row instead: the
// entries of global row r receive exactly the rows A^K[i1][:] of the cells K that hold r
// as local dof i1 (the "pairs" (K, i1) of row r). The rows are cut into chunks of
// consecutive rows (at most 4096 values and 320 pairs each); a CTA sums one chunk at a
// time in shared memory, computing every element-tensor entry on the fly from a per-cell
// geometry tensor G_K (A^K[i1][i2] = sum_alpha A0[i1][i2][alpha] G_K[alpha], Section
// 3.2), and then writes the chunk's CSR values once, in order: no global atomics, no
// zeroing pass, every value written exactly once.
//
// Work layout inside a chunk. The plan stores each chunk's pairs grouped by local index
// i1 (a "class"; within a class the pairs of different rows alternate), the work units
// (pieces of a class), and per pair the chunk-relative positions of its columns i2 =
// 0..n-1. A warp takes one unit: the reference-tensor entries A0[i1][i2][.] its lanes
// need stay in registers for the whole unit, each pair's G_K is a shared-memory
// broadcast, and one warp instruction adds the contributions of one element-tensor row
// (or of a few rows of different global rows), whose positions are distinct: the
// shared-memory atomics meet no same-address conflicts and few bank conflicts. For n
// >= 32 lane l takes column l of every pair (and the columns beyond 32 are spread over the
// lanes); for n < 32 the unit's (pair, column) items are spread over the lanes in order.
// Later chunks' plan data and geometry tensors are staged in shared memory with cp.async
// while the current chunk is summed and the previous one written out.
//
// Fixed-point accumulation. The sums are kept in fixed point with one unit per chunk and
// form, where 2^(eb-1) bounds every partial sum of every entry of the chunk (the largest
// |contribution| bound of a pair, a0max[i1] * sum|G_K|, times the largest number of pairs
// of one row). An FP32 contribution x is one 31-bit digit, x 2^(31-eb) rounded to the
// nearest integer (u = 2^(eb-31)): the scaling is exact and the sums stay within 2^30 u,
// so one 32-bit shared-memory atomic per contribution adds it, whatever the number of
// contributions. An FP64 contribution is split into three signed 21-bit digits on the
// grids 2^(eb-20), 2^(eb-41), 2^(eb-62) (u = 2^(eb-62)), each added with a 32-bit atomic
// into its own array (a digit sum of up to 1023 contributions cannot overflow 32 bits):
// 32-bit shared atomics run about seven times faster than 64-bit ones on this GPU.
// Chunks whose bound lies outside the range of the FP32 scale, and FP64 contributions,
// take an integer conversion instead (truncation, error < u). The value of an entry is
// the digit sums' value in units u, rounded once to FP64 in integer arithmetic (the FP64
// pipe's integer conversion takes half of them where it is exact). Integer addition is
// exact and associative, so the result does not depend on the order of the additions:
// per entry |result - exact sum of the contributions| <= m u / 2 + an ulp of the result
// (m contributions; u / 2 < 2^-30 B for FP32, 2^-61 B for FP64, B the chunk's bound), and
// the matrix is reproducible bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include "ffc_internal.h"
#include "geometry.cuh"

namespace ffc {
namespace {

constexpr int ROWS_VMAX = 4096;           // values of one chunk (shared-memory accumulators)
constexpr int ROWS_VSTRIDE = ROWS_VMAX + 4;  // ints of one digit array: a chunk's values, shifted by 0 or 1
constexpr int ROWS_PMAX = 320;            // pairs of one chunk
constexpr int ROWS_MAX_INCIDENCE = 1023;  // digit sums of 21-bit digits stay within 32 bits
constexpr int ROWS_MAX_LOCAL = 64;        // local dofs per cell the plan carries

// Pairs of one work unit: a warp takes the pairs of one class i1 in pieces of at most this
// many (larger pieces for small element tensors, whose units hold several pairs per step;
// short ones where a lane takes a column of a pair, so that an iteration's tasks are many
// and short and its warps finish together).
#ifndef ROWS_UMAX_WIDE
#define ROWS_UMAX_WIDE 16
#endif
__host__ __device__ constexpr int rows_umax(int n) { return n <= 6 ? 32 : (n < 32 ? 16 : ROWS_UMAX_WIDE); }
// Work units a chunk of P pairs can have: every non-empty class gives ceil(m / umax) <=
// m / umax + 1 pieces.
__host__ __device__ constexpr int region_unit_slots(int n, long long P) {
  return int((n < P ? n : P) + P / rows_umax(n));
}

// A chunk's region of plan data (16-byte aligned, a multiple of 16 bytes):
//   uint32 n_units
//   uint32 unit[region_unit_slots(n, P)]  work units i1 | k0 << 7 | k1 << 19: pairs
//                                        [k0, k1) of class i1, in class order
//   int32  pr[P]       the pairs e * n + i1, grouped by class
//   uint16 pos[P][n]   chunk-relative value index of column i2 of each pair
__host__ __device__ constexpr long long region_pr_offset(int n, long long P) {
  return 4ll * (1 + region_unit_slots(n, P));
}
__host__ __device__ constexpr long long region_bytes(int n, long long P) {
  return (region_pr_offset(n, P) + 4 * P + 2 * P * n + 15) / 16 * 16;
}

}  // namespace
}  // namespace ffc

struct ffc_row_plan {
  int device = 0;
  int64_t n_elem = 0;
  int n_local = 0;
  int64_t n_dof = 0;
  int64_t nnz = 0;
  int max_row = 0;
  int max_incidence = 0;
  int vmax = 0;                     // values of the largest chunk
  int max_pairs = 0;                // pairs of the largest chunk
  int max_region = 0;               // bytes of the largest chunk region
  int64_t n_chunks = 0;
  int64_t region_total = 0;         // bytes of all regions
  int64_t* row_ptr = nullptr;       // [n_dof + 1] copy of the pattern's row offsets
  int32_t* chunk_row = nullptr;     // [n_chunks + 1] first row of each chunk
  int32_t* chunk_pair = nullptr;    // [n_chunks + 1] first pair of each chunk (row order)
  int64_t* chunk_off = nullptr;     // [n_chunks + 1] byte offset of each chunk's region
  int64_t* chunk_val = nullptr;     // [n_chunks + 1] first CSR value of each chunk
  int32_t* chunk_inc = nullptr;     // [n_chunks] most pairs of one row in the chunk
  unsigned char* region = nullptr;  // [region_total] chunk regions (see region_bytes)
  void* geom = nullptr;             // per-cell geometry scratch, [n_elem][12] doubles
};

namespace ffc {
namespace {

constexpr unsigned PLAN_BAD_DOF = 1u, PLAN_MISSING = 2u, PLAN_BAD_ROW_PTR = 8u;

int cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FFC_ENOMEM : FFC_ECUDA;
}

// ---------------------------------------------------------------- plan construction

__global__ void plan_count(const int32_t* __restrict__ dofmap, long long total, long long n_dof,
                           int32_t* __restrict__ cnt, unsigned* err) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = dofmap[t];
    if (r < 0 || r >= n_dof) {
      atomicOr(err, PLAN_BAD_DOF);
      continue;
    }
    atomicAdd(cnt + r, 1);
  }
}

constexpr int SCAN_T = 1024, SCAN_V = 4, SCAN_CHUNK = SCAN_T * SCAN_V;

// Exclusive scan of one value per thread over a block of SCAN_T threads; `total` gets
// the block's sum. Uses `tot` (32 ints of shared memory); ends with a barrier.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t s, int32_t* tot, int32_t& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t t = tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    tot[lane] = t;
  }
  __syncthreads();
  const int32_t ex = x - s + (w > 0 ? tot[w - 1] : 0);
  total = tot[31];
  __syncthreads();
  return ex;
}

// exclusive scan of a[0, n) in chunks of SCAN_CHUNK, each chunk's total to sums[chunk]
__global__ void __launch_bounds__(SCAN_T) scan_chunks(int32_t* __restrict__ a, long long n,
                                                      int32_t* __restrict__ sums) {
  __shared__ int32_t tot[32];
  const long long base = blockIdx.x * (long long)SCAN_CHUNK + threadIdx.x * SCAN_V;
  int32_t v[SCAN_V], s = 0;
#pragma unroll
  for (int j = 0; j < SCAN_V; ++j) {
    v[j] = base + j < n ? a[base + j] : 0;
    s += v[j];
  }
  int32_t total;
  int32_t ex = block_exclusive_scan(s, tot, total);
#pragma unroll
  for (int j = 0; j < SCAN_V; ++j) {
    if (base + j < n) a[base + j] = ex;
    ex += v[j];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// exclusive scan of the chunk totals in place (one block, sequential over SCAN_T pieces)
__global__ void __launch_bounds__(SCAN_T) scan_sums(int32_t* __restrict__ sums, int nb) {
  __shared__ int32_t tot[32];
  int32_t carry = 0;
  for (int b0 = 0; b0 < nb; b0 += SCAN_T) {
    const int i = b0 + threadIdx.x;
    const int32_t s = i < nb ? sums[i] : 0;
    int32_t total;
    const int32_t ex = block_exclusive_scan(s, tot, total);
    if (i < nb) sums[i] = carry + ex;
    carry += total;
  }
}

__global__ void __launch_bounds__(SCAN_T) scan_add(int32_t* __restrict__ a, long long n,
                                                   const int32_t* __restrict__ sums) {
  const long long base = blockIdx.x * (long long)SCAN_CHUNK;
  const int32_t off = sums[blockIdx.x];
  for (int j = threadIdx.x; j < SCAN_CHUNK; j += SCAN_T)
    if (base + j < n) a[base + j] += off;
}

// the pairs (e, i1) of each row, grouped by row (order within a row: arbitrary)
__global__ void plan_fill(const int32_t* __restrict__ dofmap, long long total, long long n_dof,
                          const int32_t* __restrict__ inc_ptr, int32_t* __restrict__ fill,
                          int32_t* __restrict__ inc_tmp) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = dofmap[t];
    if (r < 0 || r >= n_dof) continue;
    const int j = atomicAdd(fill + r, 1);
    inc_tmp[inc_ptr[r] + j] = int32_t(t);
  }
}

// One thread per chunk: the chunk's pairs grouped by class i1; within a class ordered by
// (rank of the pair among the class's pairs of its row, row, cell), so consecutive pairs
// of a class belong to different rows where the class has several. Writes the ordered
// pairs and the work units (each class cut into pieces of at most rows_umax(n) pairs)
// into the chunk's region. `key` is scratch [total].
__global__ void plan_sort(const int32_t* __restrict__ dofmap, const int32_t* __restrict__ chunk_row,
                          const int32_t* __restrict__ chunk_pair, const int64_t* __restrict__ chunk_off,
                          long long n_chunks, int n, const int32_t* __restrict__ inc_tmp,
                          unsigned long long* __restrict__ key, unsigned char* __restrict__ region) {
  constexpr unsigned long long E_MASK = (1ull << 30) - 1;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n_chunks;
       c += (long long)gridDim.x * blockDim.x) {
    const int r0 = chunk_row[c];
    const int p0 = chunk_pair[c], P = chunk_pair[c + 1] - p0;
    unsigned char* reg = region + chunk_off[c];
    uint32_t* unit = reinterpret_cast<uint32_t*>(reg);
    int32_t* pr = reinterpret_cast<int32_t*>(reg + region_pr_offset(n, P));
    unsigned long long* kk = key + p0;
    // key (i1, row - r0, e) of each pair (i1 < 64, row - r0 < 2^16, e < 2^30), by insertion
    for (int j = 0; j < P; ++j) {
      const int t = inc_tmp[p0 + j];
      const unsigned long long kv = (static_cast<unsigned long long>(t % n) << 58) |
                                    (static_cast<unsigned long long>(dofmap[t] - r0) << 30) |
                                    static_cast<unsigned long long>(t / n);
      int q = j;
      while (q > 0 && kk[q - 1] > kv) {
        kk[q] = kk[q - 1];
        --q;
      }
      kk[q] = kv;
    }
    // each class: its pairs (the pairs of a row get ranks 0, 1, ..., emitted by (rank,
    // row, e)) and its work units
    const int umax = rows_umax(n);
    int a = 0, n_units = 0;
    for (int i = 0; i < n; ++i) {
      int b = a;
      while (b < P && int(kk[b] >> 58) == i) ++b;
      int out = a;
      for (int rank = 0; out < b; ++rank) {
        int rr = -1, run = 0;
        for (int j = a; j < b; ++j) {
          const int row = int((kk[j] >> 30) & 0xFFFFull);
          run = (row == rr) ? run + 1 : 0;
          rr = row;
          if (run == rank) pr[out++] = int32_t((kk[j] & E_MASK) * n + i);
        }
      }
      for (int k0 = a; k0 < b; k0 += umax)
        unit[1 + n_units++] = uint32_t(i) | (uint32_t(k0) << 7) | (uint32_t(min(k0 + umax, b)) << 19);
      a = b;
    }
    unit[0] = uint32_t(n_units);
  }
}

// One CTA per chunk: the chunk-relative position of every contribution (pair k, column
// i2): binary search of column dofmap[e][i2] in the sorted columns of row dofmap[e][i1].
__global__ void plan_positions(const int32_t* __restrict__ dofmap, int n, const int64_t* __restrict__ row_ptr,
                               const int32_t* __restrict__ col, const int32_t* __restrict__ chunk_row,
                               const int32_t* __restrict__ chunk_pair, const int64_t* __restrict__ chunk_off,
                               long long n_chunks, unsigned char* __restrict__ region, unsigned* err) {
  for (long long c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    const int r0 = chunk_row[c], r1 = chunk_row[c + 1];
    const int P = chunk_pair[c + 1] - chunk_pair[c];
    const long long base = row_ptr[r0];
    unsigned char* reg = region + chunk_off[c];
    const int32_t* pr = reinterpret_cast<const int32_t*>(reg + region_pr_offset(n, P));
    uint16_t* pos = reinterpret_cast<uint16_t*>(reg + region_pr_offset(n, P) + 4ll * P);
    for (int w = threadIdx.x; w < P * n; w += blockDim.x) {
      const int k = w / n, i2 = w - k * n;
      const int t = pr[k];
      const int e = t / n, i1 = t - e * n;
      const int r = dofmap[(long long)e * n + i1];
      const int cj = dofmap[(long long)e * n + i2];
      uint16_t q = 0;
      if (r < r0 || r >= r1) {
        atomicOr(err, PLAN_MISSING);
      } else {
        long long lo = row_ptr[r], hi = row_ptr[r + 1];
        const long long end = hi;
        while (lo < hi) {
          const long long mid = (lo + hi) >> 1;
          if (col[mid] < cj) lo = mid + 1;
          else hi = mid;
        }
        if (lo < end && col[lo] == cj) q = uint16_t(lo - base);
        else atomicOr(err, PLAN_MISSING);
      }
      pos[w] = q;
    }
  }
}

// ---------------------------------------------------------------- fixed point

// smallest eb with 2^(eb-1) >= b for a bound b >= 0 (zero and denormal bounds give the
// smallest exponent of the type)
__device__ __forceinline__ int bound_exponent(float b) { return int((__float_as_uint(b) >> 23) & 0xffu) - 125; }
__device__ __forceinline__ int bound_exponent(double b) {
  return int((static_cast<unsigned long long>(__double_as_longlong(b)) >> 52) & 0x7ffull) - 1021;
}

// 1.5 * 2^e as a float, for -126 <= e <= 127
__device__ __forceinline__ float one_and_half_pow2(int e) { return __int_as_float(((e + 127) << 23) | (1 << 22)); }

// x / 2^ulog truncated toward zero, for |x| / 2^ulog < 2^62 (integer arithmetic only)
__device__ __forceinline__ long long to_fixed(float x, int ulog) {
  const unsigned b = __float_as_uint(x);
  const int ex = int((b >> 23) & 0xffu);
  unsigned m = b & 0x7fffffu;
  int ee = 1;
  if (ex) {
    m |= 0x800000u;
    ee = ex;
  }
  const int sh = ee - 150 - ulog;  // x = m 2^(ee - 150)
  unsigned long long f;
  if (sh >= 0) f = static_cast<unsigned long long>(m) << (sh < 63 ? sh : 63);
  else f = -sh < 32 ? static_cast<unsigned long long>(m >> -sh) : 0ull;
  return (b >> 31) ? -static_cast<long long>(f) : static_cast<long long>(f);
}

__device__ __forceinline__ long long to_fixed(double x, int ulog) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int ex = int((b >> 52) & 0x7ffull);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  int ee = 1;
  if (ex) {
    m |= 1ull << 52;
    ee = ex;
  }
  const int sh = ee - 1075 - ulog;  // x = m 2^(ee - 1075)
  unsigned long long f;
  if (sh >= 0) f = m << (sh < 63 ? sh : 63);
  else f = -sh < 64 ? (m >> -sh) : 0ull;
  return (b >> 63) ? -static_cast<long long>(f) : static_cast<long long>(f);
}

__device__ __noinline__ double scaled_to_double(long long v, int ulog) { return scalbn(static_cast<double>(v), ulog); }

// v * 2^ulog rounded to the nearest double (ties to even), in integer arithmetic (the
// hardware int64 -> FP64 conversion runs on GB300's narrow FP64 pipe): the magnitude is
// normalised to a leading one at bit 63, its top 53 bits are added to (exponent - 1) << 52
// (the leading one completes the exponent field, and a carry out of the significand on
// rounding moves the value to the next binade by itself). Zero is a select; results
// outside the normal range (bounds far from 1) take a called slow path, so the common
// path never issues FP64 instructions.
__device__ __forceinline__ double fixed_to_double(long long v, int ulog) {
  const unsigned long long sign = static_cast<unsigned long long>(v) & (1ull << 63);
  unsigned long long m = sign ? 0ull - static_cast<unsigned long long>(v) : static_cast<unsigned long long>(v);
  const int lz = __clzll(static_cast<long long>(m));
  m <<= (lz & 63);
  const int e = 63 - lz + ulog + 1023;
  const unsigned long long sig = m >> 11, rb = m & 0x7ffull;
  const unsigned long long up = (rb > 0x400ull) | ((rb == 0x400ull) & sig & 1ull);
  unsigned long long bits = sign | ((static_cast<unsigned long long>(e - 1) << 52) + sig + up);
  if (m == 0) bits = sign;
  if (m != 0 && (e <= 0 || e >= 2047)) return scaled_to_double(v, ulog);
  return __longlong_as_double(static_cast<long long>(bits));
}

// v * 2^ulog for |v| < 2^53, which a double holds exactly: the magnitude's leading one is
// placed at bit 52 and (exponent - 1) << 52 added (the leading one completes the exponent
// field); no rounding step. Zero is a select; results outside the normal range take the
// called slow path.
__device__ __forceinline__ double fixed_to_double_exact(long long v, int ulog) {
  const unsigned long long sign = static_cast<unsigned long long>(v) & (1ull << 63);
  unsigned long long m = sign ? 0ull - static_cast<unsigned long long>(v) : static_cast<unsigned long long>(v);
  const int lz = __clzll(static_cast<long long>(m));  // >= 11
  const int e = 63 - lz + ulog + 1023;
  m <<= ((lz - 11) & 63);
  unsigned long long bits = sign | ((static_cast<unsigned long long>(e - 1) << 52) + m);
  if (m == 0) bits = sign;
  if (m != 0 && (e <= 0 || e >= 2047)) return scaled_to_double(v, ulog);
  return __longlong_as_double(static_cast<long long>(bits));
}

// Digits of the fixed-point sums: one 31-bit digit for FP32 contributions, three 21-bit
// digits (63 bits) for FP64 ones.
template <typename T>
__host__ __device__ constexpr int rows_ndig() { return sizeof(T) == 4 ? 1 : 3; }

// The digits of one contribution for |x| <= 2^(eb-1): NDIG = 3 on the grids 2^(eb-20),
// 2^(eb-41), 2^(eb-62) (unit u = 2^(eb-62)); NDIG = 2 on the first two (u = 2^(eb-41));
// NDIG = 1 one digit on the grid 2^(eb-31) (u = 2^(eb-31): a chunk's sums stay within
// 2^30 u, so one 32-bit integer holds them whatever the number of contributions).
// `magic`: the FP32 rounding constants are normal floats (-87 <= eb <= 124); otherwise
// the integer conversion.
template <int NDIG>
struct Digits {
  float c1, c2, c3;
  int b1, b2, b3, ulog;
  bool magic;
  __device__ __forceinline__ void init(int eb) {
    if constexpr (NDIG == 1) {
      // the scale 2^(31 - eb) must be a normal float
      magic = eb >= -96 && eb <= 157;
      c1 = __int_as_float((31 - (magic ? eb : 0) + 127) << 23);
      c2 = c3 = 0.f;
      b1 = b2 = b3 = 0;
      ulog = eb - 31;
      return;
    }
    magic = eb >= -87 && eb <= 124;
    const int e = magic ? eb : 0;
    c1 = one_and_half_pow2(e + 3);
    c2 = one_and_half_pow2(e - 18);
    c3 = one_and_half_pow2(e - 39);
    b1 = __float_as_int(c1);
    b2 = __float_as_int(c2);
    b3 = __float_as_int(c3);
    ulog = NDIG == 3 ? eb - 62 : eb - 41;
  }
  // MAGIC: the FP32 rounding constants (valid when `magic`); otherwise the integer conversion
  template <bool MAGIC>
  __device__ __forceinline__ void split(float x, int (&d)[NDIG]) const {
    if constexpr (NDIG == 1) {
      // x 2^(31 - eb) rounded to the nearest integer (the scaling is exact); |x| <= 2^(eb-1)
      // keeps it within 2^30
      if constexpr (MAGIC) d[0] = __float2int_rn(x * c1);
      else d[0] = int(to_fixed(x, ulog));
    } else if constexpr (MAGIC) {
      const float t1 = __fadd_rn(x, c1);
      const float r1 = __fsub_rn(x, __fsub_rn(t1, c1));
      const float t2 = __fadd_rn(r1, c2);
      d[0] = __float_as_int(t1) - b1;
      d[1] = __float_as_int(t2) - b2;
      if constexpr (NDIG == 3) {
        const float r2 = __fsub_rn(r1, __fsub_rn(t2, c2));
        const float t3 = __fadd_rn(r2, c3);
        d[2] = __float_as_int(t3) - b3;
      }
    } else {
      split_int(to_fixed(x, ulog), d);
    }
  }
  template <bool MAGIC>
  __device__ __forceinline__ void split(double x, int (&d)[NDIG]) const {
    split_int(to_fixed(x, ulog), d);
  }
  __device__ __forceinline__ static void split_int(long long f, int (&d)[NDIG]) {
    if constexpr (NDIG == 1) {
      d[0] = int(f);
    } else if constexpr (NDIG == 3) {
      d[2] = int(f & 0x1FFFFFll);
      d[1] = int((f >> 21) & 0x1FFFFFll);
      d[0] = int(f >> 42);
    } else {
      d[1] = int(f & 0x1FFFFFll);
      d[0] = int(f >> 21);
    }
  }
  // the 2-digit value v * 2^ulog through the FP64 pipe's int64 -> double conversion (exact:
  // |v| < 2^53) and an exponent add for 2^ulog; for chunks whose results stay normal
  // (fp64_ok), so the other lanes' integer conversions and this one use different pipes
  __device__ __forceinline__ bool fp64_ok() const { return ulog >= -1022 && ulog <= 980; }
  __device__ __forceinline__ double value_fp64(const int (&s)[NDIG]) const {
    static_assert(NDIG <= 2, "FP64-pipe conversion of the 31- or 42-bit sums");
    if constexpr (NDIG == 1) {
      const long long bits = __double_as_longlong(static_cast<double>(s[0])) + (static_cast<long long>(ulog) << 52);
      return __longlong_as_double(s[0] == 0 ? 0ll : bits);
    } else {
      const long long v = static_cast<long long>(s[0]) * (1ll << 21) + s[1];
      const long long bits = __double_as_longlong(static_cast<double>(v)) + (static_cast<long long>(ulog) << 52);
      return __longlong_as_double(v == 0 ? 0ll : bits);
    }
  }
  // the entry's value from its digit sums, rounded once to FP64
  __device__ __forceinline__ double value(const int (&s)[NDIG]) const {
    if constexpr (NDIG == 1) {  // |v| < 2^31: exact in a double
      return fixed_to_double_exact(static_cast<long long>(s[0]), ulog);
    } else if constexpr (NDIG == 3) {
      const long long v = static_cast<long long>(s[0]) * (1ll << 42) + static_cast<long long>(s[1]) * (1ll << 21) + s[2];
      return fixed_to_double(v, ulog);
    } else {  // |v| < 2^52: exact in a double
      return fixed_to_double_exact(static_cast<long long>(s[0]) * (1ll << 21) + s[1], ulog);
    }
  }
};

// ---------------------------------------------------------------- geometry

// Form codes of the row kernels: FFC_MASS, FFC_POISSON, or the (mass, Poisson) pair.
constexpr int ROWS_PAIR = FFC_PAIR_MASS_POISSON;

template <int D, int FORM>
struct RowsGeo {
  static constexpr int NF = FORM == ROWS_PAIR ? 2 : 1;        // matrices
  static constexpr int NP = D * (D + 1) / 2;                  // symmetric Poisson G_K entries
  static constexpr int NAK = FORM == FFC_POISSON ? NP : 1;    // G entries of a single form
  // stored per cell: mass [|det|, |det|]; Poisson [G (NP), sum|G|, pad to 8];
  // pair [|det|, G (NP), pad, sum|G| in slot 7]
  static constexpr int GS = FORM == FFC_MASS ? 2 : 8;
  // G_K slots of the contribution bounds' sums: |G| of a single form, and for the pair the
  // mass's |det J| (slot 0) and the Poisson sum|G| (slot 7)
  static constexpr int SUM_A = FORM == ROWS_PAIR ? 0 : (FORM == FFC_POISSON ? NP : 1);
  static constexpr int SUM_B = 7;
};

// One thread per cell: G_K exactly as the fused CUDA-core element-tensor kernels form it
// (FP32: mass |det J| from the FP64 determinant; Poisson the FP64 adjugate and
// determinant, K and the symmetric G in FP32; FP64: everything in FP64), and the sums
// of |G_K| for the bounds.
template <int D, int FORM, typename T>
__global__ void __launch_bounds__(256) rows_geometry(const int32_t* __restrict__ cells,
                                                     const double* __restrict__ vertices, long long n_vert,
                                                     long long n_elem, T* __restrict__ G, unsigned* status) {
  using C = RowsGeo<D, FORM>;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n_elem;
       e += (long long)gridDim.x * blockDim.x) {
    T g[C::GS];
#pragma unroll
    for (int a = 0; a < C::GS; ++a) g[a] = T(0);
    bool degenerate = false, bad_index = false;
    if constexpr (FORM == FFC_MASS || FORM == ROWS_PAIR) {
      double det;
      cell_det<D>(cells, vertices, n_vert, e, det, degenerate, bad_index);
      g[0] = T(det);
      if constexpr (FORM == FFC_MASS) g[1] = fabs(g[0]);
    }
    if constexpr (FORM == FFC_POISSON || FORM == ROWS_PAIR) {
      constexpr int o = FORM == ROWS_PAIR ? 1 : 0;
      bool dg, bi;
      if constexpr (sizeof(T) == 4) {
        float K[D][D], det;
        cell_geometry_f32<D>(cells, vertices, n_vert, e, K, det, dg, bi);
        geometry_tensor_f32<D, FFC_POISSON, 1, true>(K, det, nullptr, 0.0, 0.0, reinterpret_cast<float*>(g) + o);
      } else {
        double K[D][D], det;
        cell_geometry<D>(cells, vertices, n_vert, e, K, det, dg, bi);
        geometry_tensor_k<D, FFC_POISSON, 1>(K, det, nullptr, 0.0, 0.0, [&](int a, double v) { g[o + a] = T(v); });
      }
      T s = T(0);
#pragma unroll
      for (int a = 0; a < C::NP; ++a) s += fabs(g[o + a]);
      g[FORM == ROWS_PAIR ? C::SUM_B : C::NP] = s;
      degenerate |= dg;
      bad_index |= bi;
    }
    T* dst = G + e * C::GS;
#pragma unroll
    for (int a = 0; a < C::GS; ++a) dst[a] = g[a];
    if (degenerate) atomicOr(status, FFC_FLAG_DEGENERATE);
    if (bad_index) atomicOr(status, FFC_FLAG_BOUNDS);
  }
}

// ---------------------------------------------------------------- assembly

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct RowsParams {
  const int64_t* chunk_off;
  const int32_t* chunk_pair;
  const int64_t* chunk_val;
  const int32_t* chunk_inc;
  const unsigned char* region;
  const void* G;
  const void* a0a;  // mass or single-form reference tensor [N][NAK][N] in T
  const void* a0b;  // pair: the Poisson reference tensor [N][NP][N]
  double* out_a;
  double* out_b;
  long long n_chunks;
  int meta_off;  // byte offset of the chunk-extent ring in shared memory
  int pmax;   // pairs of the largest chunk
  int rmax;   // bytes of the largest chunk region
  unsigned* status;
};

__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

#ifndef ROWS_WB
#define ROWS_WB 256
#endif
#ifndef ROWS_TB
#define ROWS_TB 256
#endif

template <int D, int FORM, int Q>
struct RowsCfg {
  static constexpr int N = nscalar(D, Q);
  static constexpr bool MAIN = N >= 32;              // lane l takes column l of every pair
  static constexpr int W = MAIN ? N - 32 : N;        // columns spread over the lanes in order
  static constexpr int I0 = MAIN ? 32 : 0;           // first of those columns
  static constexpr int PER = W > 0 ? W / gcd_c(32, W) : 1;  // steps after which a lane's column repeats
  static constexpr int NP = D * (D + 1) / 2;
  static constexpr int NA = FORM == ROWS_PAIR ? 1 + NP : (FORM == FFC_POISSON ? NP : 1);  // A0 values per entry
  static constexpr int NG = FORM == FFC_MASS ? 1 : 8;  // G_K values read per pair (vector loads)
  static constexpr int TB = ROWS_TB;    // items of one task of the columns beyond the first 32
  // Order of an iteration's tasks after the staging ones: for n >= 32 (lane per column)
  // the work units first and the write-out blocks, shorter (128 indices), last, so that
  // the iteration ends on short tasks (P4 tets: mass + Poisson 4.28 -> 4.04 ms at 48^3);
  // otherwise units and write-out blocks alternate while both last (P3: 1.64 ms, 1.69
  // units first)
  static constexpr bool UNITS_FIRST = MAIN;
  static constexpr int WB = MAIN ? 128 : ROWS_WB;  // digit indices of one write-out task
};

// A0 entry (i1, i2) of the kernel's form(s), in the order the contraction uses, from the
// [i1][alpha][i2] copies (lanes of consecutive i2 read consecutive words)
template <int FORM, int N, int NA, int NP, typename T>
__device__ __forceinline__ void load_a0(const T* __restrict__ A0a, const T* __restrict__ A0b, int i1, int i2,
                                        T (&a)[NA]) {
  if constexpr (FORM == ROWS_PAIR) {
    a[0] = __ldg(A0a + i1 * N + i2);
#pragma unroll
    for (int j = 0; j < NP; ++j) a[1 + j] = __ldg(A0b + (i1 * NP + j) * N + i2);
  } else {
#pragma unroll
    for (int j = 0; j < NA; ++j) a[j] = __ldg(A0a + (i1 * NA + j) * N + i2);
  }
}

// the first NG values of a pair's G_K from shared memory (16-byte aligned rows for NG = 8)
template <int NG, typename T>
__device__ __forceinline__ void load_gk(const T* gs, T (&g)[NG]) {
  if constexpr (NG == 1) {
    g[0] = gs[0];
  } else if constexpr (sizeof(T) == 4) {
    const float4 x = reinterpret_cast<const float4*>(gs)[0], y = reinterpret_cast<const float4*>(gs)[1];
    g[0] = x.x, g[1] = x.y, g[2] = x.z, g[3] = x.w, g[4] = y.x, g[5] = y.y, g[6] = y.z, g[7] = y.w;
  } else {
#pragma unroll
    for (int j = 0; j < NG / 2; ++j) {
      const double2 x = reinterpret_cast<const double2*>(gs)[j];
      g[2 * j] = x.x;
      g[2 * j + 1] = x.y;
    }
  }
}

// the contributions of one element-tensor entry: sum_alpha G_K[alpha] A0[i1][i2][alpha]
// (FMA order as in the fused element-tensor kernels, so FP32 values agree bit for bit)
template <int FORM, int NA, int NG, int NF, typename T>
__device__ __forceinline__ void contract(const T (&g)[NG], const T (&a)[NA], T (&v)[NF]) {
  if constexpr (FORM == ROWS_PAIR) {
    v[0] = fma(g[0], a[0], T(0));
    T s = T(0);
#pragma unroll
    for (int j = 1; j < NA; ++j) s = fma(g[j], a[j], s);
    v[1] = s;
  } else {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < NA; ++j) s = fma(g[j], a[j], s);
    v[0] = s;
  }
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Adds one entry's contributions (digits) at chunk position q; base[f] is form f's first
// digit array (the arrays of one form ROWS_VSTRIDE ints apart).
template <bool MAGIC, int NF, int NDIG, typename T>
__device__ __forceinline__ void add_digits(int* const (&base)[NF], const Digits<NDIG> (&dig)[NF], const T (&v)[NF],
                                           int q) {
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    int d[NDIG];
    dig[f].template split<MAGIC>(v[f], d);
    int* a = base[f] + q;
#pragma unroll
    for (int j = 0; j < NDIG; ++j) atomicAdd(a + j * ROWS_VSTRIDE, d[j]);
  }
}

// Positions come from a validated plan (every (row, col) pair was found in the pattern when
// the plan was built, so q < V); the mask only keeps a shared-memory index in range.
__device__ __forceinline__ int rows_pos(int q) { return q & (ROWS_VMAX - 1); }

#ifndef ROWS_UNROLL
#define ROWS_UNROLL 2
#endif
constexpr int kRowsUnroll = ROWS_UNROLL;  // pairs of a work unit in flight per loop step



// One work unit (class i1, pairs [k0, k1)) of a chunk, by one warp: for n >= 32 lane l takes
// column l of every pair (the A0 column in registers), for n < 32 the unit's (pair, column)
// items in order.
template <class K, int FORM, int NF, int GS, bool MAGIC, int NDIG, typename T>
__device__ __forceinline__ void unit_task(unsigned ud, const T* gs, const uint16_t* pos, int* const (&base)[NF],
                                          const Digits<NDIG> (&dig)[NF], const T* A0a, const T* A0b) {
  constexpr int N = K::N, NA = K::NA, NG = K::NG;
  const int lane = threadIdx.x & 31;
  const int i1 = int(ud & 127u), k0 = int((ud >> 7) & 4095u), k1 = int(ud >> 19);
  if constexpr (K::MAIN) {
    T am[NA];
    load_a0<FORM, N, NA, K::NP, T>(A0a, A0b, i1, lane, am);
    const uint16_t* pl = pos + lane;
#pragma unroll kRowsUnroll
    for (int k = k0; k < k1; ++k) {
      T g[NG];
      load_gk<NG, T>(gs + k * GS, g);
      const int q = rows_pos(pl[k * N]);
      T v[NF];
      contract<FORM, NA, NG, NF, T>(g, am, v);
      add_digits<MAGIC, NF, NDIG, T>(base, dig, v, q);
    }
  } else {
    T af[K::PER][NA];
#pragma unroll
    for (int s = 0; s < K::PER; ++s) load_a0<FORM, N, NA, K::NP, T>(A0a, A0b, i1, (lane + 32 * s) % K::W, af[s]);
    const int total = (k1 - k0) * K::W;
    for (int f0 = 0; f0 < total; f0 += 32 * K::PER) {
#pragma unroll
      for (int s = 0; s < K::PER; ++s) {
        const int f = f0 + 32 * s + lane;
        if (f < total) {
          const int kk = k0 + f / K::W;
          const int i2 = K::I0 + f % K::W;
          T g[NG];
          load_gk<NG, T>(gs + kk * GS, g);
          const int q = rows_pos(pos[kk * N + i2]);
          T v[NF];
          contract<FORM, NA, NG, NF, T>(g, af[s], v);
          add_digits<MAGIC, NF, NDIG, T>(base, dig, v, q);
        }
      }
    }
  }
}

// Items [b * TB, (b + 1) * TB) of the columns beyond the first 32 (n > 32), packed over
// the lanes: item f is pair f / W, column 32 + f % W.
template <class K, int FORM, int NF, int GS, bool MAGIC, int NDIG, typename T>
__device__ __forceinline__ void tail_task(int b, int P, const int32_t* pr, const T* gs, const uint16_t* pos,
                                          int* const (&base)[NF], const Digits<NDIG> (&dig)[NF], const T* A0a,
                                          const T* A0b) {
  constexpr int N = K::N, NA = K::NA, NG = K::NG;
  if constexpr (K::MAIN && K::W > 0) {
    const int total = P * K::W, end = min(total, (b + 1) * K::TB);
    for (int f = b * K::TB + (threadIdx.x & 31); f < end; f += 32) {
      const int k = f / K::W, i2 = 32 + f % K::W;
      const int i1 = pr[k] % N;
      T a[NA], g[NG];
      load_a0<FORM, N, NA, K::NP, T>(A0a, A0b, i1, i2, a);
      load_gk<NG, T>(gs + k * GS, g);
      const int q = rows_pos(pos[k * N + i2]);
      T v[NF];
      contract<FORM, NA, NG, NF, T>(g, a, v);
      add_digits<MAGIC, NF, NDIG, T>(base, dig, v, q);
    }
  }
}

// Per-chunk state prepared one iteration ahead (three slots, by chunk index mod 3), read by
// every warp of the iteration that uses it.
template <int NDIG>
struct RowsSlot {
  Digits<NDIG> dig[2];  // fixed-point digits of each form (from its bound's exponent)
  int finite[2];        // the form's bound is finite
  int shift[2];         // chunk position q of form f sits at digit index q + shift[f]: the
                        // output address of index 0 is then 16-byte aligned
  int n_units, n_items;  // work units, and units + column-tail blocks
  int P, V;              // pairs and CSR values of the chunk
};

// mbarrier helpers of the staging copies: cp.async issued by one warp, tracked by an
// mbarrier of arrival count 32 (each lane arrives when its own copies have landed)
__device__ __forceinline__ uint32_t rows_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void rows_bar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(rows_smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void rows_cp_async_arrive(unsigned long long* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(rows_smem_u32(bar)) : "memory");
}
// Bounded wait for the completion of the phase of parity `parity`: false after ~2^22 polls.
__device__ __forceinline__ bool rows_bar_wait(unsigned long long* bar, unsigned parity) {
  const uint32_t addr = rows_smem_u32(bar);
  for (uint32_t it = 0; it < (1u << 22); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Values (of each 4 consecutive ones a lane converts) that take the FP64 pipe's integer
// conversion where it is exact: bit c set for value c.
#ifndef ROWS_FP64_MASK
#define ROWS_FP64_MASK 0xA
#endif

// The chunks of this CTA are c_i = blockIdx.x + i * gridDim.x. Iteration i is one queue of
// independent warp tasks, handed out by a shared counter: three staging tasks (chunk i + 3's
// plan region, chunk i + 2's geometry and digits, chunk i + 5's extents), then the work
// units of chunk i (into accumulator buffer i % 2) interleaved with the write-out blocks of
// chunk i - 1 (from the other buffer, which they clear). The region copy is cp.async
// tracked by an mbarrier that only its consumer (the geometry task, an iteration later)
// waits for; the geometry task gathers the pairs' G_K, waits for its own copies, and
// derives the chunk's fixed-point digits from the largest contribution bound. The work
// units come with the plan. One CTA-wide barrier closes each iteration. Staging depths:
// regions 4 buffers (i .. i + 3), geometry 3 (i .. i + 2), per-chunk state 4 slots
// (i - 1 .. i + 2), extents a ring of 8. A wait that gives up sets FFC_FLAG_TIMEOUT and
// ends the CTA's work after the iteration.
// One CTA per SM: 32 warps for FP32 (64 registers a thread), 16 for FP64.
template <int D, int FORM, int Q, typename T>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 1024 : 512, 1) rows_assemble(RowsParams p) {
  using C = RowsGeo<D, FORM>;
  using K = RowsCfg<D, FORM, Q>;
  constexpr int N = K::N, NF = C::NF, GS = C::GS, TH = sizeof(T) == 4 ? 1024 : 512;
  constexpr int NDIG = rows_ndig<T>();  // digits: 31-bit fixed point for FP32, 63-bit for FP64
  constexpr int ACC = NF * NDIG * ROWS_VSTRIDE;  // ints of one accumulator buffer
  constexpr int NSPECIAL = 3;
  using Slot = RowsSlot<NDIG>;
  extern __shared__ __align__(16) unsigned char smem[];
  int* acc = reinterpret_cast<int*>(smem);                                   // [2][NF][NDIG][ROWS_VSTRIDE]
  unsigned char* rbuf = smem + size_t(2) * ACC * 4;                          // [4][rmax] plan regions
  T* gbuf = reinterpret_cast<T*>(rbuf + 4 * size_t(p.rmax));                 // [3][pmax][GS]
  T* a0max = gbuf + 3 * size_t(p.pmax) * GS;                                 // [NF][N]
  Slot* slot = reinterpret_cast<Slot*>(a0max + NF * N);                      // [4]
  int* tq = reinterpret_cast<int*>(slot + 4);                                // [2] task counters, [2] abort
  long long* meta = reinterpret_cast<long long*>(smem + p.meta_off);          // [8][8]: chunk extents
  unsigned long long* rbar = reinterpret_cast<unsigned long long*>(meta + 64);  // [4] region copies
  const T* A0a = static_cast<const T*>(p.a0a);
  const T* A0b = static_cast<const T*>(p.a0b);
  const T* Gall = static_cast<const T*>(p.G);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const T big = sizeof(T) == 4 ? T(FLT_MAX) : T(DBL_MAX);
  const int G1 = int(gridDim.x);
  const int n_iter = blockIdx.x < p.n_chunks ? int((p.n_chunks - blockIdx.x + G1 - 1) / G1) : 0;
  // largest |A0| entry of each reference-tensor row i1 (the contribution bound's factor)
  for (int i = t; i < NF * N; i += TH) {
    const int f = i / N, i1 = i - f * N;
    const int na = (FORM == ROWS_PAIR && f == 1) ? C::NP : C::NAK;
    const T* A = (FORM == ROWS_PAIR && f == 1) ? A0b : A0a;
    T m = T(0);
    for (int k = 0; k < N * na; ++k) m = fmax(m, fabs(A[size_t(i1) * N * na + k]));
    a0max[i] = m;
  }
  for (int i = 4 * t; i < 2 * ACC; i += 4 * TH) *reinterpret_cast<int4*>(acc + i) = make_int4(0, 0, 0, 0);
  if (t < 3) tq[t] = 0;
  if (t < 4) rows_bar_init(rbar + t, 32);
  // extents of the chunk of iteration i, ring slot i % 8: pairs [0] .. [1), region bytes
  // [2] .. [3), CSR values [4] .. [5), most pairs of a row [6]
  auto meta_at = [&](int i) { return meta + (i & 7) * 8; };
  auto meta_task = [&](int i) {  // one warp
    const long long c = blockIdx.x + (long long)i * G1;
    if (i < n_iter && lane < 7) {
      long long v;
      if (lane < 2) v = p.chunk_pair[c + lane];
      else if (lane < 4) v = p.chunk_off[c + lane - 2];
      else if (lane < 6) v = p.chunk_val[c + lane - 4];
      else v = p.chunk_inc[c];
      meta_at(i)[lane] = v;
    }
  };
  auto region_at = [&](int i) { return rbuf + (i & 3) * p.rmax; };
  auto geom_at = [&](unsigned i3) { return gbuf + i3 * p.pmax * GS; };  // i3 = i % 3
  // the plan region of chunk i (a multiple of 16 bytes, at most rmax) into buffer i % 4
  auto region_task = [&](int i) {  // one warp
    const long long* m = meta_at(i);
    const unsigned char* src = p.region + m[2];
    unsigned char* dst = region_at(i);
    const int nb = int(m[3] - m[2]);
    for (int o = 16 * lane; o < nb; o += 512) cp_async16(dst + o, src + o);
    rows_cp_async_arrive(rbar + (i & 3));
  };
  // chunk i's geometry (one warp, once its region has landed): the pairs' G_K gathered
  // into buffer i % 3, then its per-chunk state in slot i % 4: fixed-point digits from the
  // bound (largest pair bound times the most pairs of a row), output alignment shifts,
  // counts
  auto geometry_task = [&](int i) {
    Slot& sl = slot[i & 3];
    if (!rows_bar_wait(rbar + (i & 3), unsigned(i >> 2) & 1u)) {
      if (lane == 0) {
        atomicOr(p.status, FFC_FLAG_TIMEOUT);
        tq[2] = 1;
        sl.n_units = sl.n_items = sl.P = sl.V = 0;
      }
      return;
    }
    const long long* m = meta_at(i);
    const int P = int(m[1] - m[0]);
    const unsigned char* reg = region_at(i);
    const int32_t* pr = reinterpret_cast<const int32_t*>(reg + region_pr_offset(N, P));
    T* gs = geom_at(unsigned(i) % 3u);
    for (int k = lane; k < P; k += 32) {
      const T* src = Gall + (long long)(pr[k] / N) * GS;
      if constexpr (GS * sizeof(T) == 8) {
        cp_async8(gs + k * GS, src);
      } else {
#pragma unroll
        for (int x = 0; x < int(GS * sizeof(T)) / 16; ++x)
          cp_async16(reinterpret_cast<unsigned char*>(gs + k * GS) + 16 * x,
                     reinterpret_cast<const unsigned char*>(src) + 16 * x);
      }
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncwarp();
    T pb[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) pb[f] = T(0);
    for (int k = lane; k < P; k += 32) {
      const int i1 = pr[k] % N;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const T x = a0max[f * N + i1] * fabs(gs[k * GS + (f == 0 ? C::SUM_A : C::SUM_B)]);
        pb[f] = fmax(pb[f], x == x ? x : big * T(2));  // NaN -> inf
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const T bnd = warp_max(pb[f]) * T(m[6]);
      if (lane == f) {
        sl.finite[f] = bnd <= big;
        Digits<NDIG> dg;
        dg.init(bnd <= big ? bound_exponent(bnd) : 0);
        sl.dig[f] = dg;
        const double* out = (f == 0 ? p.out_a : p.out_b) + m[4];
        sl.shift[f] = int((reinterpret_cast<uintptr_t>(out) >> 3) & 1);
      }
    }
    if (lane == 31) {
      const int nu = int(*reinterpret_cast<const uint32_t*>(reg));
      sl.n_units = nu;
      sl.n_items = nu + (K::MAIN && K::W > 0 ? (P * K::W + K::TB - 1) / K::TB : 0);
      sl.P = P;
      sl.V = int(m[5] - m[4]);
    }
  };
  // digit indices [b * WB, (b + 1) * WB) of chunk i from accumulator buffer i % 2 (cleared),
  // one warp: each lane converts four consecutive indices per step and stores them as two
  // 16-byte pairs (index x is output value x - shift, and output index 0 is 16-byte
  // aligned); where the FP64 pipe's conversion is exact, the values of ROWS_FP64_MASK take
  // it, so two pipes share the conversions
  auto write_task = [&](int i, int b) {
    const Slot& sl = slot[i & 3];
    const long long v0 = meta_at(i)[4];
    const int V = sl.V;
    int* ab = acc + (i & 1) * ACC;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const Digits<NDIG> dg = sl.dig[f];
      const bool fin = sl.finite[f] != 0;
      const int sh = sl.shift[f];
      double* out = (f == 0 ? p.out_a : p.out_b) + v0 - sh;
      int* a = ab + f * NDIG * ROWS_VSTRIDE;
      const bool split_pipes = NDIG <= 2 && fin && dg.fp64_ok();
      const int hi = V + sh, end = min(hi, (b + 1) * K::WB);
      for (int x = b * K::WB + 4 * lane; x < end; x += 128) {
        int4 dd[NDIG];
#pragma unroll
        for (int d = 0; d < NDIG; ++d) {
          dd[d] = *reinterpret_cast<const int4*>(a + d * ROWS_VSTRIDE + x);
          *reinterpret_cast<int4*>(a + d * ROWS_VSTRIDE + x) = make_int4(0, 0, 0, 0);
        }
        double r[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          int sd[NDIG];
#pragma unroll
          for (int d = 0; d < NDIG; ++d) sd[d] = c == 0 ? dd[d].x : c == 1 ? dd[d].y : c == 2 ? dd[d].z : dd[d].w;
          if constexpr (NDIG <= 2) {
            if (((ROWS_FP64_MASK >> c) & 1) && split_pipes) {
              r[c] = dg.value_fp64(sd);
              continue;
            }
          }
          r[c] = fin ? dg.value(sd) : nan;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int y = x + 2 * h;
          if (y >= sh && y + 1 < hi) {
            __stcs(reinterpret_cast<double2*>(out + y), make_double2(r[2 * h], r[2 * h + 1]));
          } else {
            if (y >= sh && y < hi) __stcs(out + y, r[2 * h]);
            if (y + 1 >= sh && y + 1 < hi) __stcs(out + y + 1, r[2 * h + 1]);
          }
        }
      }
    }
  };
  // ---- prologue: extents of iterations 0..4; regions of chunks 0..2; geometry of chunks
  // 0..1 (each waits for what it reads)
  if (w < 5) meta_task(w);
  __syncthreads();
  if (w < 3 && w < n_iter) region_task(w);
  if (w == 3 && n_iter > 0) geometry_task(0);
  if (w == 4 && n_iter > 1) geometry_task(1);
  __syncthreads();
  unsigned i3 = 0;  // i % 3
  for (int i = 0; i <= n_iter && tq[2] == 0; ++i, i3 = i3 == 2 ? 0 : i3 + 1) {
    if (t == 0) tq[(i + 1) & 1] = 0;  // the next iteration's queue (last used two iterations ago)
    // this iteration's work: units (and column tails) of chunk i, write-out blocks of chunk i - 1
    const Slot& cur = slot[i & 3];
    int nI = 0, nU = 0, nW = 0, P = 0;
    if (i < n_iter) {
      P = cur.P;
      nU = cur.n_units;
      nI = cur.n_items;
    }
    if (i >= 1) nW = (slot[(i - 1) & 3].V + 1 + K::WB - 1) / K::WB;  // indices up to V + shift
    const int nMix = 2 * min(nI, nW), n_tasks = NSPECIAL + nI + nW;
    const unsigned char* reg = region_at(i);
    const unsigned* un = reinterpret_cast<const unsigned*>(reg) + 1;
    const int32_t* pr = reinterpret_cast<const int32_t*>(reg + region_pr_offset(N, P));
    const uint16_t* pos = reinterpret_cast<const uint16_t*>(reg + region_pr_offset(N, P) + 4 * P);
    const T* gs = geom_at(i3);
    int* ab = acc + (i & 1) * ACC;
    Digits<NDIG> dig[NF];
    int* base[NF];
    bool magic = sizeof(T) == 4;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      base[f] = ab + f * NDIG * ROWS_VSTRIDE;
      if (i < n_iter) {
        dig[f] = cur.dig[f];
        magic = magic && dig[f].magic;
        base[f] += cur.shift[f];
      }
    }
    for (;;) {
      int k = 0;
      if (lane == 0) k = atomicAdd(tq + (i & 1), 1);
      k = __shfl_sync(0xffffffffu, k, 0);
      if (k >= n_tasks) break;
      if (k < NSPECIAL) {
        if (k == 0 && i + 3 < n_iter) region_task(i + 3);
        if (k == 1 && i + 2 < n_iter) geometry_task(i + 2);
        if (k == 2) meta_task(i + 5);
        continue;
      }
      k -= NSPECIAL;
      bool item;
      int j;
      if constexpr (K::UNITS_FIRST) {
        item = k < nI;
        j = item ? k : k - nI;
      } else if (k < nMix) {  // items and write-out blocks alternate while both last
        item = (k & 1) == 0;
        j = k >> 1;
      } else {
        item = nI > nW;
        j = k - nMix / 2;
      }
      if (item) {
        if (j < nU) {
          if (magic) unit_task<K, FORM, NF, GS, true, NDIG, T>(un[j], gs, pos, base, dig, A0a, A0b);
          else unit_task<K, FORM, NF, GS, false, NDIG, T>(un[j], gs, pos, base, dig, A0a, A0b);
        } else {
          if (magic) tail_task<K, FORM, NF, GS, true, NDIG, T>(j - nU, P, pr, gs, pos, base, dig, A0a, A0b);
          else tail_task<K, FORM, NF, GS, false, NDIG, T>(j - nU, P, pr, gs, pos, base, dig, A0a, A0b);
        }
      } else {
        write_task(i - 1, j);
      }
    }
    __syncthreads();
  }
  cp_async_commit();
  cp_async_wait_all();  // copies of chunks this CTA no longer needed (a wait that gave up)
}

template <int D, int FORM, int Q, typename T>
int launch_rows_t(const ffc_row_plan* plan, const void* a0a, const void* a0b, double* out_a, double* out_b,
                  unsigned* status, cudaStream_t s) {
  using C = RowsGeo<D, FORM>;
  constexpr int N = nscalar(D, Q);
  const int pmax = std::max(plan->max_pairs, 1);
  using K = RowsCfg<D, FORM, Q>;
  constexpr int NDIG = rows_ndig<T>();
  const int rmax = std::max(plan->max_region, 16);
  const size_t meta_off = (2 * size_t(C::NF) * NDIG * ROWS_VSTRIDE * 4 + 4 * size_t(rmax) +
                           (3 * size_t(pmax) * C::GS + size_t(C::NF) * N) * sizeof(T) +
                           4 * sizeof(RowsSlot<NDIG>) + 3 * 4 + 15) / 16 * 16;
  const size_t smem = meta_off + 8 * 8 * sizeof(long long) + 4 * sizeof(unsigned long long);
  auto kern = rows_assemble<D, FORM, Q, T>;
  int dev = 0, smem_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > size_t(smem_optin)) return FFC_EUNSUPPORTED;  // the pair then runs as two single passes
  if (plan->n_chunks > (long long)INT_MAX) {  // iteration counters are 32-bit
    set_error("row-owner assembly: more than 2^31 - 1 chunks");
    return FFC_EINVAL;
  }
  int sms = 0, per_sm = 1;
  constexpr int TH = sizeof(T) == 4 ? 1024 : 512;
  if (launch_config(reinterpret_cast<const void*>(kern), TH, smem, -1, &sms, &per_sm) != FFC_OK)
    return FFC_ECUDA;
  long long blocks = (long long)sms * per_sm;
  if (blocks > plan->n_chunks) blocks = plan->n_chunks;
  if (blocks < 1) return FFC_OK;
  RowsParams prm{plan->chunk_off, plan->chunk_pair, plan->chunk_val, plan->chunk_inc, plan->region, plan->geom,
                 a0a, a0b, out_a, out_b, (long long)plan->n_chunks, int(meta_off), pmax, rmax, status};
  kern<<<unsigned(blocks), TH, smem, s>>>(prm);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FFC_OK : cuda_fail(e, "rows_assemble launch");
}

template <int D, int FORM, typename T>
int launch_rows_geometry(const ffc_row_plan* plan, const int32_t* cells, const double* vertices, int64_t n_vert,
                         unsigned* status, cudaStream_t s) {
  if (plan->n_elem == 0) return FFC_OK;
  int sms = 0;
  if (launch_config(reinterpret_cast<const void*>(rows_geometry<D, FORM, T>), 256, 0, -1, &sms, nullptr) != FFC_OK)
    return FFC_ECUDA;
  long long blocks = (plan->n_elem + 255) / 256;
  if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
  rows_geometry<D, FORM, T><<<unsigned(blocks), 256, 0, s>>>(cells, vertices, n_vert, plan->n_elem,
                                                              static_cast<T*>(plan->geom), status);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FFC_OK : cuda_fail(e, "rows_geometry launch");
}

template <int D, int FORM, typename T>
int launch_rows_q(const ffc_row_plan* plan, int q, const int32_t* cells, const double* vertices, int64_t n_vert,
                  const void* a0a, const void* a0b, double* out_a, double* out_b, unsigned* status,
                  cudaStream_t s) {
  int rc = launch_rows_geometry<D, FORM, T>(plan, cells, vertices, n_vert, status, s);
  if (rc != FFC_OK) return rc;
  switch (q) {
    case 1: return launch_rows_t<D, FORM, 1, T>(plan, a0a, a0b, out_a, out_b, status, s);
    case 2: return launch_rows_t<D, FORM, 2, T>(plan, a0a, a0b, out_a, out_b, status, s);
    case 3: return launch_rows_t<D, FORM, 3, T>(plan, a0a, a0b, out_a, out_b, status, s);
    case 4: return launch_rows_t<D, FORM, 4, T>(plan, a0a, a0b, out_a, out_b, status, s);
    default: return FFC_EUNSUPPORTED;
  }
}

template <typename T>
int launch_rows_form(int form, int d, int q, const ffc_row_plan* plan, const int32_t* cells, const double* vertices,
                     int64_t n_vert, const void* a0a, const void* a0b, double* out_a, double* out_b,
                     unsigned* status, cudaStream_t s) {
  if (d == 3) {
    if (form == FFC_MASS)
      return launch_rows_q<3, FFC_MASS, T>(plan, q, cells, vertices, n_vert, a0a, a0b, out_a, out_b, status, s);
    if (form == FFC_POISSON)
      return launch_rows_q<3, FFC_POISSON, T>(plan, q, cells, vertices, n_vert, a0a, a0b, out_a, out_b, status, s);
    return launch_rows_q<3, ROWS_PAIR, T>(plan, q, cells, vertices, n_vert, a0a, a0b, out_a, out_b, status, s);
  }
  if (form == FFC_MASS)
    return launch_rows_q<2, FFC_MASS, T>(plan, q, cells, vertices, n_vert, a0a, a0b, out_a, out_b, status, s);
  if (form == FFC_POISSON)
    return launch_rows_q<2, FFC_POISSON, T>(plan, q, cells, vertices, n_vert, a0a, a0b, out_a, out_b, status, s);
  return launch_rows_q<2, ROWS_PAIR, T>(plan, q, cells, vertices, n_vert, a0a, a0b, out_a, out_b, status, s);
}

void free_plan(ffc_row_plan* p) {
  if (!p) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  cudaFree(p->row_ptr);
  cudaFree(p->chunk_row);
  cudaFree(p->chunk_pair);
  cudaFree(p->chunk_off);
  cudaFree(p->chunk_val);
  cudaFree(p->chunk_inc);
  cudaFree(p->region);
  cudaFree(p->geom);
  cudaSetDevice(cur);
  delete p;
}

template <typename T>
int dev_alloc(T** p, size_t count) {
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T));
  return e == cudaSuccess ? FFC_OK : cuda_fail(e, "cudaMalloc");
}

// Common checks of the row assemblies; fills the device tensors of the form(s).
int rows_checks(const char* who, const ffc_form* f, const ffc_row_plan* plan, const int32_t* cells,
                const double* vertices, int64_t n_vert, const double* out, int precision) {
  if (!f || !plan || n_vert < 0 || (precision != FFC_FP64 && precision != FFC_FP32)) {
    set_error(std::string(who) + ": invalid argument");
    return FFC_EINVAL;
  }
  if ((f->kind != FFC_MASS && f->kind != FFC_POISSON) || f->rank != 2) {
    set_error(std::string(who) + ": mass and Poisson forms only");
    return FFC_EUNSUPPORTED;
  }
  if (f->n != plan->n_local) {
    set_error(std::string(who) + ": the plan was built for another number of local dofs");
    return FFC_EINVAL;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != plan->device) {
    set_error(std::string(who) + ": the plan lives on another device");
    return FFC_EINVAL;
  }
  if (plan->nnz == 0) return FFC_OK;
  if (!out || (reinterpret_cast<uintptr_t>(out) & 7) ||
      (plan->n_elem > 0 && (!cells || !vertices || n_vert == 0 || (reinterpret_cast<uintptr_t>(cells) & 15) ||
                            (reinterpret_cast<uintptr_t>(vertices) & 7)))) {
    set_error(std::string(who) + ": null or misaligned pointer");
    return FFC_EINVAL;
  }
  return FFC_OK;
}

}  // namespace
}  // namespace ffc

using namespace ffc;

extern "C" {

int ffc_row_plan_create(int64_t n_elem, int n_local, const int32_t* dofmap, int64_t n_dof, const int64_t* row_ptr,
                        const int32_t* col, int64_t nnz, void* stream, ffc_row_plan** out) {
  if (!out || n_elem < 0 || n_local < 2 || n_local > ROWS_MAX_LOCAL || n_dof < 1 || n_dof >= INT32_MAX || nnz < 0 ||
      !row_ptr || (n_elem > 0 && !dofmap) || (nnz > 0 && !col)) {
    set_error("ffc_row_plan_create: invalid argument (2 <= n_local <= 64)");
    return FFC_EINVAL;
  }
  if (n_elem * (long long)n_local >= INT32_MAX) {
    set_error("ffc_row_plan_create: n_elem * n_local must be below 2^31");
    return FFC_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(dofmap) & 3) || (reinterpret_cast<uintptr_t>(row_ptr) & 7) ||
      (reinterpret_cast<uintptr_t>(col) & 3)) {
    set_error("ffc_row_plan_create: misaligned pointer");
    return FFC_EINVAL;
  }
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ffc_row_plan* p = new ffc_row_plan();
  cudaGetDevice(&p->device);
  p->n_elem = n_elem;
  p->n_local = n_local;
  p->n_dof = n_dof;
  p->nnz = nnz;
  const long long total = n_elem * (long long)n_local;
  const long long nb = (n_dof + 1 + SCAN_CHUNK - 1) / SCAN_CHUNK;
  int32_t *inc_ptr = nullptr, *inc_tmp = nullptr, *fill = nullptr, *sums = nullptr;
  unsigned long long* key = nullptr;
  unsigned* err = nullptr;
  int rc = FFC_OK;
  cudaError_t e = cudaSuccess;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  const unsigned grid = unsigned(sms > 0 ? sms * 8 : 1024);
  unsigned host_err = 0;
  std::vector<int64_t> h_row_ptr(size_t(n_dof) + 1);
  std::vector<int32_t> h_inc_ptr(size_t(n_dof) + 1);
  std::vector<int32_t> h_chunk_row, h_chunk_pair, h_chunk_inc;
  std::vector<int64_t> h_chunk_off, h_chunk_val;
  if ((rc = dev_alloc(&p->row_ptr, size_t(n_dof) + 1)) || (rc = dev_alloc(&inc_ptr, size_t(n_dof) + 1)) ||
      (rc = dev_alloc(&inc_tmp, size_t(total))) || (rc = dev_alloc(&fill, size_t(n_dof))) ||
      (rc = dev_alloc(&sums, size_t(nb))) || (rc = dev_alloc(&err, 1)) ||
      (rc = dev_alloc(reinterpret_cast<double**>(&p->geom), size_t(n_elem) * 12)))
    goto fail;
  if ((e = cudaMemcpyAsync(p->row_ptr, row_ptr, (size_t(n_dof) + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                           s)) != cudaSuccess ||
      (e = cudaMemsetAsync(inc_ptr, 0, (size_t(n_dof) + 1) * sizeof(int32_t), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(fill, 0, size_t(n_dof) * sizeof(int32_t), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(err, 0, sizeof(unsigned), s)) != cudaSuccess) {
    rc = cuda_fail(e, "ffc_row_plan_create: memset");
    goto fail;
  }
  if (total > 0) plan_count<<<grid, 256, 0, s>>>(dofmap, total, n_dof, inc_ptr, err);
  scan_chunks<<<unsigned(nb), SCAN_T, 0, s>>>(inc_ptr, n_dof + 1, sums);
  scan_sums<<<1, SCAN_T, 0, s>>>(sums, int(nb));
  scan_add<<<unsigned(nb), SCAN_T, 0, s>>>(inc_ptr, n_dof + 1, sums);
  if (total > 0) plan_fill<<<grid, 256, 0, s>>>(dofmap, total, n_dof, inc_ptr, fill, inc_tmp);
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(h_row_ptr.data(), row_ptr, h_row_ptr.size() * sizeof(int64_t), cudaMemcpyDeviceToHost,
                           s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h_inc_ptr.data(), inc_ptr, h_inc_ptr.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                           s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&host_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    rc = cuda_fail(e, "ffc_row_plan_create");
    goto fail;
  }
  if (host_err & PLAN_BAD_DOF) {
    set_error("ffc_row_plan_create: dof id out of range");
    rc = FFC_EBOUNDS;
    goto fail;
  }
  {
    // rows -> chunks (host, one pass): consecutive rows while the chunk holds at most
    // ROWS_VMAX values, ROWS_PMAX pairs and 65536 rows
    if (h_row_ptr[0] != 0 || h_row_ptr[n_dof] != nnz) host_err |= PLAN_BAD_ROW_PTR;
    int32_t cur_v = 0, cur_p = 0, cur_inc = 0, r_start = 0;
    int64_t off = 0;
    auto close_chunk = [&](int64_t r) {
      const int64_t bytes = region_bytes(n_local, cur_p);
      off += bytes;
      h_chunk_inc.push_back(cur_inc);
      p->vmax = std::max(p->vmax, int(cur_v));
      p->max_pairs = std::max(p->max_pairs, int(cur_p));
      p->max_region = std::max(p->max_region, int(bytes));
      h_chunk_row.push_back(int32_t(r));
      h_chunk_pair.push_back(h_inc_ptr[r]);
      h_chunk_off.push_back(off);
      h_chunk_val.push_back(h_row_ptr[r]);
      cur_v = cur_p = cur_inc = 0;
      r_start = int32_t(r);
    };
    h_chunk_row.push_back(0);
    h_chunk_pair.push_back(0);
    h_chunk_off.push_back(0);
    h_chunk_val.push_back(0);
    for (int64_t r = 0; r < n_dof && !(host_err & PLAN_BAD_ROW_PTR); ++r) {
      const int64_t L = h_row_ptr[r + 1] - h_row_ptr[r];
      const int32_t c = h_inc_ptr[r + 1] - h_inc_ptr[r];
      if (L < 0 || h_row_ptr[r + 1] > nnz) {
        host_err |= PLAN_BAD_ROW_PTR;
        break;
      }
      if (L > ROWS_VMAX || c > ROWS_PMAX || c > ROWS_MAX_INCIDENCE) {
        set_error("ffc_row_plan_create: row " + std::to_string(r) + " has " + std::to_string(L) + " entries and " +
                  std::to_string(c) + " (cell, local dof) pairs; at most " + std::to_string(ROWS_VMAX) + " and " +
                  std::to_string(std::min(ROWS_PMAX, ROWS_MAX_INCIDENCE)) + " are supported");
        rc = FFC_EINVAL;
        goto fail;
      }
      if (r > r_start && (cur_v + L > ROWS_VMAX || cur_p + c > ROWS_PMAX || r - r_start >= 65536)) close_chunk(r);
      cur_v += int32_t(L);
      cur_p += c;
      cur_inc = std::max(cur_inc, c);
      p->max_row = std::max(p->max_row, int(L));
      p->max_incidence = std::max(p->max_incidence, int(c));
    }
    if (host_err & PLAN_BAD_ROW_PTR) {
      set_error("ffc_row_plan_create: row_ptr is not monotone within [0, nnz]");
      rc = FFC_EINVAL;
      goto fail;
    }
    close_chunk(n_dof);
    p->n_chunks = int64_t(h_chunk_inc.size());
    p->region_total = off;
  }
  if ((rc = dev_alloc(&p->chunk_row, h_chunk_row.size())) || (rc = dev_alloc(&p->chunk_pair, h_chunk_pair.size())) ||
      (rc = dev_alloc(&p->chunk_off, h_chunk_off.size())) || (rc = dev_alloc(&p->chunk_val, h_chunk_val.size())) ||
      (rc = dev_alloc(&p->chunk_inc, h_chunk_inc.size())) ||
      (rc = dev_alloc(&p->region, size_t(p->region_total) + 16)) ||
      (rc = dev_alloc(&key, size_t(total))))
    goto fail;
  if ((e = cudaMemcpyAsync(p->chunk_row, h_chunk_row.data(), h_chunk_row.size() * 4, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(p->chunk_pair, h_chunk_pair.data(), h_chunk_pair.size() * 4, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(p->chunk_off, h_chunk_off.data(), h_chunk_off.size() * 8, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(p->chunk_val, h_chunk_val.data(), h_chunk_val.size() * 8, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(p->chunk_inc, h_chunk_inc.data(), h_chunk_inc.size() * 4, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemsetAsync(p->region, 0, size_t(p->region_total) + 16, s)) != cudaSuccess) {
    rc = cuda_fail(e, "ffc_row_plan_create: chunk table");
    goto fail;
  }
  plan_sort<<<unsigned((p->n_chunks + 127) / 128), 128, 0, s>>>(dofmap, p->chunk_row, p->chunk_pair, p->chunk_off,
                                                                p->n_chunks, n_local, inc_tmp, key, p->region);
  if (total > 0)
    plan_positions<<<grid, 256, 0, s>>>(dofmap, n_local, p->row_ptr, col, p->chunk_row, p->chunk_pair, p->chunk_off,
                                        p->n_chunks, p->region, err);
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(&host_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    rc = cuda_fail(e, "ffc_row_plan_create");
    goto fail;
  }
  if (host_err & PLAN_MISSING) {
    set_error("ffc_row_plan_create: a (row, col) pair of a cell is not in the pattern");
    rc = FFC_EBOUNDS;
    goto fail;
  }
  cudaFree(inc_ptr);
  cudaFree(inc_tmp);
  cudaFree(fill);
  cudaFree(sums);
  cudaFree(err);
  cudaFree(key);
  *out = p;
  return FFC_OK;
fail:
  cudaStreamSynchronize(s);
  cudaFree(inc_ptr);
  cudaFree(inc_tmp);
  cudaFree(fill);
  cudaFree(sums);
  cudaFree(err);
  cudaFree(key);
  free_plan(p);
  return rc;
}

int ffc_row_plan_info(const ffc_row_plan* p, int64_t* n_dof, int64_t* nnz, int* max_row, int* max_incidence) {
  if (!p) return FFC_EINVAL;
  if (n_dof) *n_dof = p->n_dof;
  if (nnz) *nnz = p->nnz;
  if (max_row) *max_row = p->max_row;
  if (max_incidence) *max_incidence = p->max_incidence;
  return FFC_OK;
}

int ffc_row_plan_layout(const ffc_row_plan* p, int64_t* n_chunks, int* max_chunk_values, int* max_chunk_pairs,
                        int* max_region_bytes, int64_t* device_bytes) {
  if (!p) return FFC_EINVAL;
  if (n_chunks) *n_chunks = p->n_chunks;
  if (max_chunk_values) *max_chunk_values = p->vmax;
  if (max_chunk_pairs) *max_chunk_pairs = p->max_pairs;
  if (max_region_bytes) *max_region_bytes = p->max_region;
  if (device_bytes)
    *device_bytes = (p->n_dof + 1) * 8 + (p->n_chunks + 1) * (4 + 4 + 8 + 8) + p->n_chunks * 4 +
                    p->region_total + 16 + p->n_elem * 96;
  return FFC_OK;
}

void ffc_row_plan_destroy(ffc_row_plan* p) { free_plan(p); }

int ffc_assemble_rows(const ffc_form* f, const ffc_row_plan* plan, const int32_t* cells, const double* vertices,
                      int64_t n_vert, double* csr_val, int precision, void* stream) {
  int rc = rows_checks("ffc_assemble_rows", f, plan, cells, vertices, n_vert, csr_val, precision);
  if (rc != FFC_OK || plan->nnz == 0) return rc;
  DeviceTensors* t = nullptr;
  if ((rc = ensure_device_tensors(const_cast<ffc_form*>(f), &t)) != FFC_OK) return rc;
  uint32_t* st = status_word();
  if (!st) {
    set_error("status word allocation failed");
    return FFC_ECUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = precision == FFC_FP32 ? launch_rows_form<float>(f->kind, f->d, f->q, plan, cells, vertices, n_vert, t->a0s_f32,
                                                       nullptr, csr_val, nullptr, st, s)
                             : launch_rows_form<double>(f->kind, f->d, f->q, plan, cells, vertices, n_vert,
                                                        t->a0s_f64, nullptr, csr_val, nullptr, st, s);
  if (rc == FFC_EUNSUPPORTED) set_error("ffc_assemble_rows: the plan's chunks need more shared memory than a CTA has");
  return rc;
}

int ffc_assemble_rows_pair(const ffc_form* fa, const ffc_form* fb, const ffc_row_plan* plan, const int32_t* cells,
                           const double* vertices, int64_t n_vert, double* csr_val_a, double* csr_val_b,
                           int precision, void* stream) {
  int rc = rows_checks("ffc_assemble_rows_pair", fa, plan, cells, vertices, n_vert, csr_val_a, precision);
  if (rc != FFC_OK) return rc;
  if ((rc = rows_checks("ffc_assemble_rows_pair", fb, plan, cells, vertices, n_vert, csr_val_b, precision)) != FFC_OK)
    return rc;
  if (fa->d != fb->d || fa->q != fb->q || csr_val_a == csr_val_b) {
    set_error("ffc_assemble_rows_pair: two forms on one space, two distinct matrices");
    return FFC_EINVAL;
  }
  if (plan->nnz == 0) return FFC_OK;
  if (fa->kind == fb->kind) {  // not the (mass, Poisson) pair: two single passes
    if ((rc = ffc_assemble_rows(fa, plan, cells, vertices, n_vert, csr_val_a, precision, stream)) != FFC_OK) return rc;
    return ffc_assemble_rows(fb, plan, cells, vertices, n_vert, csr_val_b, precision, stream);
  }
  const ffc_form* fm = fa->kind == FFC_MASS ? fa : fb;
  const ffc_form* fp = fa->kind == FFC_MASS ? fb : fa;
  double* vm = fa->kind == FFC_MASS ? csr_val_a : csr_val_b;
  double* vp = fa->kind == FFC_MASS ? csr_val_b : csr_val_a;
  DeviceTensors *tm = nullptr, *tp = nullptr;
  if ((rc = ensure_device_tensors(const_cast<ffc_form*>(fm), &tm)) != FFC_OK ||
      (rc = ensure_device_tensors(const_cast<ffc_form*>(fp), &tp)) != FFC_OK)
    return rc;
  uint32_t* st = status_word();
  if (!st) {
    set_error("status word allocation failed");
    return FFC_ECUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == FFC_FP32) {
    rc = launch_rows_form<float>(ROWS_PAIR, fm->d, fm->q, plan, cells, vertices, n_vert, tm->a0s_f32, tp->a0s_f32, vm,
                                 vp, st, s);
    if (rc != FFC_EUNSUPPORTED) return rc;
  }
  // FP64 (whose double-buffered 63-bit accumulators of two matrices exceed the shared
  // memory), and chunks too large for one pass: two single passes
  if ((rc = ffc_assemble_rows(fm, plan, cells, vertices, n_vert, vm, precision, stream)) != FFC_OK) return rc;
  return ffc_assemble_rows(fp, plan, cells, vertices, n_vert, vp, precision, stream);
}

}  // extern "C"
