// Row-owner assembly: Algorithm 2 (Section 2.2) with its loops ordered by global row.
//
// Algorithm 2 adds each element tensor into the global matrix, A[iota(i1), iota(i2)] +=
// A^K[i1][i2]; done cell by cell on a GPU, every addition is a global FP64 atomic and the
// matrix must be zeroed first. Here the same sums are taken row by row instead: the
// entries of global row r receive exactly the rows A^K[i1][:] of the cells K that hold r
// as local dof i1. A warp owns a row, computes those element-tensor rows on the fly from
// a per-cell geometry tensor G_K (A^K[i1][i2] = sum_alpha A0[i1][i2][alpha] G_K[alpha],
// Section 3.2) and sums them in shared memory, then writes the finished row once: no
// global atomics, no zeroing pass, every CSR value written exactly once.
//
// Exact accumulation. The sums are kept in 64-bit two's-complement fixed point with a
// per-row unit u = 2^(eb - 64), where 2^eb is at least four times a bound on the sum of
// the magnitudes of every contribution to the row (|A^K[i1][i2]| <= max|A0[i1][.][.]| *
// sum|G_K|), so every partial sum stays below 2^62 units. An FP32 contribution is split
// into three signed 21-bit digits on the grids 2^(eb-22), 2^(eb-43), 2^(eb-64) by adding
// and subtracting the constants 1.5 * 2^(grid + 23) (each add rounds to the grid, each
// subtraction is exact, and the digit is the difference of the float bit patterns): seven
// FP32 additions and three integer subtractions, error <= u / 2. Rows whose bound lies
// outside the range where those constants are normal floats, and FP64 contributions, take
// an integer conversion (truncation, error < u). Integer addition is exact and
// associative, so the result does not depend on the order of the additions; the final
// value is rounded once to FP64 (round to nearest even). Absolute error per entry <=
// (contributions) * u + half an ulp of the result: far below the rounding of the
// contributions themselves.
//
// The row plan (built once per dof map on the device) stores, for every row, the
// (cell, local index) pairs that hold it and, for each such pair, the position of every
// column dofmap[e][i2] inside the row (uint16, relative to the row start).
#include <cuda_runtime.h>

#include <cfloat>
#include <climits>
#include <cstring>
#include <string>

#include "ffc_internal.h"
#include "geometry.cuh"

struct ffc_row_plan {
  int device = 0;
  int64_t n_elem = 0;
  int n_local = 0;
  int64_t n_dof = 0;
  int64_t nnz = 0;
  int max_row = 0;
  int max_incidence = 0;
  int64_t* row_ptr = nullptr;  // [n_dof + 1] copy of the pattern's row offsets
  int32_t* inc_ptr = nullptr;  // [n_dof + 1]
  int32_t* inc = nullptr;      // [n_elem * n_local] (+16 bytes), entries e * n_local + i1
  uint16_t* pos = nullptr;     // [n_elem * n_local * n_local] (+16 bytes)
  void* geom = nullptr;        // per-cell geometry scratch, [n_elem][8] doubles
};

namespace ffc {
namespace {

constexpr unsigned PLAN_BAD_DOF = 1u, PLAN_MISSING = 2u, PLAN_LONG_ROW = 4u, PLAN_BAD_ROW_PTR = 8u;

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

// A warp per row: orders the row's (cell, i1) pairs by e * n + i1 (they are distinct, so
// each one's rank is the count of smaller ones), then finds the position of every
// column dofmap[e][i2] in the row's sorted columns by binary search.
__global__ void plan_rows(const int32_t* __restrict__ dofmap, int n, long long n_dof,
                          const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, long long nnz,
                          const int32_t* __restrict__ inc_ptr, const int32_t* __restrict__ inc_tmp,
                          int32_t* __restrict__ inc, uint16_t* __restrict__ pos, int* max_row, int* max_inc,
                          unsigned* err) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; r < n_dof; r += warps) {
    const int k0 = inc_ptr[r], c = inc_ptr[r + 1] - k0;
    const long long rp0 = row_ptr[r], rp1 = row_ptr[r + 1];
    if (rp0 < 0 || rp1 < rp0 || rp1 > nnz) {
      if (lane == 0) atomicOr(err, PLAN_BAD_ROW_PTR);
      continue;
    }
    const long long L = rp1 - rp0;
    if (L > 65535) {
      if (lane == 0) atomicOr(err, PLAN_LONG_ROW);
      continue;
    }
    if (lane == 0) {
      atomicMax(max_row, int(L));
      atomicMax(max_inc, c);
    }
    for (int j = lane; j < c; j += 32) {
      const int x = inc_tmp[k0 + j];
      int rank = 0;
      for (int m = 0; m < c; ++m) rank += inc_tmp[k0 + m] < x;
      inc[k0 + rank] = x;
    }
    __syncwarp();
    const long long items = (long long)c * n;
    for (long long it = lane; it < items; it += 32) {
      const int k = int(it / n), i2 = int(it - (long long)k * n);
      const int e = inc[k0 + k] / n;
      const int cj = dofmap[(long long)e * n + i2];
      long long lo = rp0, hi = rp1;
      while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (col[mid] < cj) lo = mid + 1;
        else hi = mid;
      }
      uint16_t q = 0xFFFF;
      if (lo < rp1 && col[lo] == cj) q = uint16_t(lo - rp0);
      else atomicOr(err, PLAN_MISSING);
      pos[(long long)k0 * n + it] = q;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- fixed point

// 2^eb >= 4 * bnd for a bound bnd >= 0 (denormal and zero bounds give the smallest eb)
__device__ __forceinline__ int bound_exponent(float b) { return int((__float_as_uint(b) >> 23) & 0xffu) - 124; }
__device__ __forceinline__ int bound_exponent(double b) {
  return int((static_cast<unsigned long long>(__double_as_longlong(b)) >> 52) & 0x7ffull) - 1020;
}

// 1.5 * 2^e as a float, for -126 <= e <= 127
__device__ __forceinline__ float one_and_half_pow2(int e) { return __int_as_float(((e + 127) << 23) | (1 << 22)); }

// x / 2^(eb - 64) for an FP32 x with |x| <= 2^(eb - 2), as three digits on the grids
// 2^(eb-22), 2^(eb-43), 2^(eb-64), each found by rounding to the grid with an added
// constant; valid for -85 <= eb <= 126, where the constants are normal floats.
struct FixedSplit {
  float c1, c2, c3;
  int b1, b2, b3;
  __device__ __forceinline__ void init(int eb) {
    c1 = one_and_half_pow2(eb + 1);
    c2 = one_and_half_pow2(eb - 20);
    c3 = one_and_half_pow2(eb - 41);
    b1 = __float_as_int(c1);
    b2 = __float_as_int(c2);
    b3 = __float_as_int(c3);
  }
  __device__ __forceinline__ long long operator()(float x) const {
    const float t1 = __fadd_rn(x, c1);
    const float r1 = __fsub_rn(x, __fsub_rn(t1, c1));
    const float t2 = __fadd_rn(r1, c2);
    const float r2 = __fsub_rn(r1, __fsub_rn(t2, c2));
    const float t3 = __fadd_rn(r2, c3);
    return static_cast<long long>(__float_as_int(t1) - b1) * (1ll << 42) +
           static_cast<long long>(__float_as_int(t2) - b2) * (1ll << 21) + (__float_as_int(t3) - b3);
  }
};

// x / 2^(eb - 62), truncated toward zero; |x| <= 2^eb keeps it below 2^62
__device__ __forceinline__ long long to_fixed(float x, int eb) {
  const unsigned b = __float_as_uint(x);
  const int ex = int((b >> 23) & 0xffu);
  unsigned m = b & 0x7fffffu;
  int ee = 1;
  if (ex) {
    m |= 0x800000u;
    ee = ex;
  }
  const int sh = ee - 88 - eb;  // x = m 2^(ee - 150)
  unsigned long long f;
  if (sh >= 0) f = static_cast<unsigned long long>(m) << (sh < 63 ? sh : 63);
  else f = -sh < 32 ? static_cast<unsigned long long>(m >> -sh) : 0ull;
  return (b >> 31) ? -static_cast<long long>(f) : static_cast<long long>(f);
}

__device__ __forceinline__ long long to_fixed(double x, int eb) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int ex = int((b >> 52) & 0x7ffull);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  int ee = 1;
  if (ex) {
    m |= 1ull << 52;
    ee = ex;
  }
  const int sh = ee - 1013 - eb;  // x = m 2^(ee - 1075)
  unsigned long long f;
  if (sh >= 0) f = m << (sh < 63 ? sh : 63);
  else f = -sh < 64 ? (m >> -sh) : 0ull;
  return (b >> 63) ? -static_cast<long long>(f) : static_cast<long long>(f);
}

// v * 2^(eb - 62) rounded to the nearest double (ties to even), in integer arithmetic (the
// hardware int64 -> FP64 conversion runs on GB300's narrow FP64 pipe and was slower);
// results outside the normal range (not reached by the bounds of FP32 values) use scalbn.
__device__ __forceinline__ double fixed_to_double(long long v, int eb) {
  if (v == 0) return 0.0;
  const unsigned long long sign = static_cast<unsigned long long>(v) & (1ull << 63);
  unsigned long long m = v < 0 ? 0ull - static_cast<unsigned long long>(v) : static_cast<unsigned long long>(v);
  const int lz = __clzll(static_cast<long long>(m));
  m <<= lz;  // leading one at bit 63: value = 1.f * 2^(eb + 1 - lz)
  int e = eb + 1 - lz + 1023;
  unsigned long long mant = (m >> 11) & ((1ull << 52) - 1);
  const unsigned rb = unsigned(m & 0x7ffull);
  if (rb > 0x400u || (rb == 0x400u && (mant & 1ull))) {
    if (++mant == (1ull << 52)) {
      mant = 0;
      ++e;
    }
  }
  if (e <= 0 || e >= 2047) return scalbn(static_cast<double>(v), eb - 62);
  return __longlong_as_double(static_cast<long long>(sign | (static_cast<unsigned long long>(e) << 52) | mant));
}

// ---------------------------------------------------------------- geometry and rows

template <int D, int FORM>
struct RowsGeo {
  static constexpr int NAK = FORM == FFC_POISSON ? D * (D + 1) / 2 : 1;  // G_K entries (symmetric Poisson G)
  static constexpr int GS = FORM == FFC_POISSON ? (D == 3 ? 8 : 4) : 2;   // stored per cell: G, sum|G|, pad
};

template <typename T, int GS>
__device__ __forceinline__ void load_g(const T* __restrict__ src, T (&g)[GS]) {
  constexpr int BYTES = GS * int(sizeof(T));
  if constexpr (BYTES % 16 == 0) {
#pragma unroll
    for (int j = 0; j < BYTES / 16; ++j) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(src) + j);
      memcpy(reinterpret_cast<char*>(g) + 16 * j, &v, 16);
    }
  } else {
#pragma unroll
    for (int j = 0; j < BYTES / 8; ++j) {
      const float2 v = __ldg(reinterpret_cast<const float2*>(src) + j);
      memcpy(reinterpret_cast<char*>(g) + 8 * j, &v, 8);
    }
  }
}

// One thread per cell: G_K exactly as the CUDA-core element-tensor kernels form it (FP32:
// FP64 adjugate and determinant, K and G in FP32; FP64: everything in FP64), followed by
// sum|G_K| for the row bounds.
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
    bool degenerate, bad_index;
    if constexpr (FORM == FFC_MASS) {
      double det;
      cell_det<D>(cells, vertices, n_vert, e, det, degenerate, bad_index);
      g[0] = T(det);
    } else if constexpr (sizeof(T) == 4) {
      float K[D][D], det;
      cell_geometry_f32<D>(cells, vertices, n_vert, e, K, det, degenerate, bad_index);
      geometry_tensor_f32<D, FORM, 1, true>(K, det, nullptr, 0.0, 0.0, reinterpret_cast<float*>(g));
    } else {
      double K[D][D], det;
      cell_geometry<D>(cells, vertices, n_vert, e, K, det, degenerate, bad_index);
      geometry_tensor_k<D, FORM, 1>(K, det, nullptr, 0.0, 0.0, [&](int a, double v) { g[a] = T(v); });
    }
    T s = T(0);
#pragma unroll
    for (int a = 0; a < C::NAK; ++a) s += fabs(g[a]);
    g[C::NAK] = s;
    T* dst = G + e * C::GS;
#pragma unroll
    for (int a = 0; a < C::GS; ++a) dst[a] = g[a];
    if (degenerate) atomicOr(status, FFC_FLAG_DEGENERATE);
    if (bad_index) atomicOr(status, FFC_FLAG_BOUNDS);
  }
}

struct RowsParams {
  const int64_t* row_ptr;
  const int32_t* inc_ptr;
  const int32_t* inc;
  const uint16_t* pos;
  const void* G;
  const void* a0;  // [N*N][NAK] in T
  double* csr_val;
  long long n_dof;
  int lmax;        // accumulator entries per warp (longest row)
  int max_inc;     // most incidences of one row
  int warp_bytes;  // shared memory of one warp
  unsigned* status;
};

template <int D, int FORM, int Q, typename T>
struct RowsCfg {
  static constexpr int N = nscalar(D, Q);
  static constexpr int NAK = RowsGeo<D, FORM>::NAK;
  static constexpr int GS = RowsGeo<D, FORM>::GS;
  static constexpr size_t A0_BYTES = (size_t(N) * N * NAK * sizeof(T) + size_t(N) * sizeof(T) + 15) / 16 * 16;
};

// Per-warp shared memory: the row accumulator, two staging buffers for the positions and
// two for the incidences of a row (filled by cp.async, 16-byte chunks from an aligned-down
// start, hence the 32 bytes of slack), and the G_K of the row's cells.
struct WarpLayout {
  int acc, pos, inc, g, bytes;  // offsets of acc, pos[0], inc[0], g; pos[1] = pos + pb, inc[1] = inc + ib
  int pb, ib;
  __host__ __device__ WarpLayout(int lmax, int max_inc, int n, int g_bytes) {
    pb = (max_inc * n * 2 + 32 + 15) / 16 * 16;
    ib = (max_inc * 4 + 32 + 15) / 16 * 16;
    acc = 0;
    pos = (lmax * 8 + 15) / 16 * 16;
    inc = pos + 2 * pb;
    g = inc + 2 * ib;
    bytes = g + (max_inc * g_bytes + 15) / 16 * 16;
  }
};

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory"); }

// Copies bytes [b0, b1) of `src` (a 16-byte aligned array padded by 16 bytes) into `dst` as
// 16-byte chunks starting at b0 rounded down to 16; the data of b0 lands at dst + (b0 & 15).
__device__ __forceinline__ void stage_range(unsigned char* dst, const unsigned char* src, long long b0, long long b1,
                                            int lane) {
  const long long a0 = b0 & ~15ll;
  const int chunks = int((b1 - a0 + 15) >> 4);
  for (int j = lane; j < chunks; j += 32) cp_async16(dst + 16 * j, src + a0 + 16 * j);
}

// A warp per global row (grid-stride over rows), software-pipelined: while row r is
// summed, cp.async stages the positions and incidences of the warp's next row, and the
// row offsets of the one after are loaded. Per row: G_K of the row's cells (one gather
// from L2) with the bound, fixed-point accumulation of the contributions in the warp's
// shared-memory row (shared 64-bit atomics: contributions of different cells may hit one
// entry), one rounding per entry and a coalesced streaming store.
template <int D, int FORM, int Q, typename T>
__global__ void __launch_bounds__(512, 1) rows_assemble(RowsParams p) {
  using C = RowsCfg<D, FORM, Q, T>;
  constexpr int N = C::N, NAK = C::NAK, GS = C::GS;
  extern __shared__ __align__(16) unsigned char smem[];
  T* a0s = reinterpret_cast<T*>(smem);  // [N*N][NAK]
  T* a0max = a0s + N * N * NAK;         // [N]: max |A0[i1][.][.]|
  const T* A0 = static_cast<const T*>(p.a0);
  for (int k = threadIdx.x; k < N * N * NAK; k += blockDim.x) a0s[k] = A0[k];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const WarpLayout lay(p.lmax, p.max_inc, N, GS * int(sizeof(T)));
  unsigned char* wbase = smem + C::A0_BYTES + size_t(w) * p.warp_bytes;
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(wbase + lay.acc);
  T* gbuf = reinterpret_cast<T*>(wbase + lay.g);
  for (int j = lane; j < p.lmax; j += 32) acc[j] = 0ull;
  __syncthreads();
  for (int i1 = threadIdx.x; i1 < N; i1 += blockDim.x) {
    T m = T(0);
    for (int k = 0; k < N * NAK; ++k) m = fmax(m, fabs(a0s[i1 * N * NAK + k]));
    a0max[i1] = m;
  }
  __syncthreads();
  const T* G = static_cast<const T*>(p.G);
  const unsigned char* pos_bytes = reinterpret_cast<const unsigned char*>(p.pos);
  const unsigned char* inc_bytes = reinterpret_cast<const unsigned char*>(p.inc);
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  // row offsets of this row and the next: (base, end, k0, k1)
  long long m_base = 0, m_end = 0, n_base = 0, n_end = 0;
  int m_k0 = 0, m_k1 = 0, n_k0 = 0, n_k1 = 0;
  if (r < p.n_dof) {
    m_base = p.row_ptr[r];
    m_end = p.row_ptr[r + 1];
    m_k0 = p.inc_ptr[r];
    m_k1 = p.inc_ptr[r + 1];
    stage_range(wbase + lay.pos, pos_bytes, 2ll * m_k0 * N, 2ll * m_k1 * N, lane);
    stage_range(wbase + lay.inc, inc_bytes, 4ll * m_k0, 4ll * m_k1, lane);
  }
  cp_async_commit();
  if (r + warps < p.n_dof) {
    n_base = p.row_ptr[r + warps];
    n_end = p.row_ptr[r + warps + 1];
    n_k0 = p.inc_ptr[r + warps];
    n_k1 = p.inc_ptr[r + warps + 1];
  }
  int buf = 0;
  for (; r < p.n_dof; r += warps) {
    // stage the next row, load the offsets of the one after
    const long long rn = r + warps, rnn = rn + warps;
    if (rn < p.n_dof) {
      stage_range(wbase + lay.pos + (buf ^ 1) * lay.pb, pos_bytes, 2ll * n_k0 * N, 2ll * n_k1 * N, lane);
      stage_range(wbase + lay.inc + (buf ^ 1) * lay.ib, inc_bytes, 4ll * n_k0, 4ll * n_k1, lane);
    }
    cp_async_commit();
    long long nn_base = 0, nn_end = 0;
    int nn_k0 = 0, nn_k1 = 0;
    if (rnn < p.n_dof) {
      nn_base = p.row_ptr[rnn];
      nn_end = p.row_ptr[rnn + 1];
      nn_k0 = p.inc_ptr[rnn];
      nn_k1 = p.inc_ptr[rnn + 1];
    }
    cp_async_wait<1>();  // this row's copies are done (the next row's may still fly)
    __syncwarp();
    const long long base = m_base, Ll = m_end - m_base;
    const int k0 = m_k0, c = m_k1 - m_k0;
    const uint16_t* pos_s = reinterpret_cast<const uint16_t*>(wbase + lay.pos + buf * lay.pb + ((2ll * k0 * N) & 15));
    int* inc_s = reinterpret_cast<int*>(wbase + lay.inc + buf * lay.ib + ((4ll * k0) & 15));
    if (Ll < 0 || Ll > p.lmax || c < 0 || c > p.max_inc) {
      if (lane == 0) atomicOr(p.status, FFC_FLAG_BOUNDS);
    } else {
      const int L = int(Ll);
      // G_K of the row's cells into shared memory (local index i1 replaces the incidence),
      // and the bound on the row's sum of |contributions|
      T bnd = T(0);
      for (int j = lane; j < c; j += 32) {
        const int t = inc_s[j];
        const int e = t / N, i1 = t - e * N;
        T g[GS];
        load_g<T, GS>(G + (long long)e * GS, g);
#pragma unroll
        for (int a = 0; a < GS; ++a) gbuf[j * GS + a] = g[a];
        inc_s[j] = i1;
        bnd += a0max[i1] * g[NAK];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bnd += __shfl_xor_sync(0xffffffffu, bnd, o);
      __syncwarp();
      const T big = sizeof(T) == 4 ? T(FLT_MAX) : T(DBL_MAX);
      if (!(bnd <= big)) {  // a non-finite G_K (degenerate cell, flagged by the geometry kernel)
        for (int j = lane; j < L; j += 32) p.csr_val[base + j] = __longlong_as_double(0x7ff8000000000000ll);
      } else {
        const int eb = bound_exponent(bnd);
        const bool split_ok = sizeof(T) == 4 && eb >= -85 && eb <= 126;  // uniform over the warp
        FixedSplit split;
        split.init(split_ok ? eb : 0);
        const int items = c * N;
        for (int it = lane; it < items; it += 32) {
          const int k = it / N, i2 = it - k * N;
          const int i1 = inc_s[k];
          const int q = pos_s[it];
          const T* g = gbuf + k * GS;
          const T* a = a0s + (i1 * N + i2) * NAK;
          T v = T(0);
#pragma unroll
          for (int al = 0; al < NAK; ++al) v = fma(g[al], a[al], v);
          long long f;
          if constexpr (sizeof(T) == 4) f = split_ok ? split(v) : to_fixed(v, eb - 2);
          else f = to_fixed(v, eb - 2);
          if (q < L) atomicAdd(acc + q, static_cast<unsigned long long>(f));
          else atomicOr(p.status, FFC_FLAG_BOUNDS);
        }
        __syncwarp();
        for (int j = lane; j < L; j += 32) {
          const long long f = static_cast<long long>(acc[j]);
          acc[j] = 0ull;
          __stcs(p.csr_val + base + j, fixed_to_double(f, eb - 2));
        }
      }
    }
    __syncwarp();  // this row's buffers are free for the copy issued next iteration
    buf ^= 1;
    m_base = n_base;
    m_end = n_end;
    m_k0 = n_k0;
    m_k1 = n_k1;
    n_base = nn_base;
    n_end = nn_end;
    n_k0 = nn_k0;
    n_k1 = nn_k1;
  }
  cp_async_wait<0>();
}

template <int D, int FORM, int Q, typename T>
int launch_rows_t(const ffc_row_plan* plan, const void* a0, double* csr_val, unsigned* status,
                  cudaStream_t s) {
  using C = RowsCfg<D, FORM, Q, T>;
  int dev = 0, sms = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int lmax = plan->max_row > 0 ? plan->max_row : 1;
  const int max_inc = plan->max_incidence > 0 ? plan->max_incidence : 1;
  const WarpLayout lay(lmax, max_inc, C::N, C::GS * int(sizeof(T)));
  auto kern = rows_assemble<D, FORM, Q, T>;
  // warps per block: the count that keeps the most warps resident per SM
  int best_nw = 0, best_warps = 0;
  size_t best_smem = 0;
  for (int nw : {16, 12, 8, 6, 4, 2, 1}) {
    const size_t smem = C::A0_BYTES + size_t(nw) * lay.bytes;
    if (smem > size_t(smem_max)) continue;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nw * 32, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm * nw > best_warps) {
      best_warps = per_sm * nw;
      best_nw = nw;
      best_smem = smem;
    }
  }
  if (best_nw == 0) {
    set_error("row assembly: the longest row does not fit in shared memory");
    return FFC_EUNSUPPORTED;
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(best_smem));
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  long long blocks = (long long)sms * (best_warps / best_nw);
  const long long need = (plan->n_dof + best_nw - 1) / best_nw;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  RowsParams prm{plan->row_ptr, plan->inc_ptr, plan->inc, plan->pos, plan->geom, a0, csr_val,
                 (long long)plan->n_dof, lmax, max_inc, lay.bytes, status};
  kern<<<unsigned(blocks), best_nw * 32, best_smem, s>>>(prm);
  e = cudaGetLastError();
  return e == cudaSuccess ? FFC_OK : cuda_fail(e, "rows_assemble launch");
}

template <int D, int FORM, typename T>
int launch_rows_geometry(const ffc_row_plan* plan, const int32_t* cells, const double* vertices, int64_t n_vert,
                         unsigned* status, cudaStream_t s) {
  if (plan->n_elem == 0) return FFC_OK;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (plan->n_elem + 255) / 256;
  if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
  rows_geometry<D, FORM, T><<<unsigned(blocks), 256, 0, s>>>(cells, vertices, n_vert, plan->n_elem,
                                                              static_cast<T*>(plan->geom), status);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FFC_OK : cuda_fail(e, "rows_geometry launch");
}

template <int D, int FORM, typename T>
int launch_rows_q(const ffc_row_plan* plan, int q, const int32_t* cells, const double* vertices, int64_t n_vert,
                  const void* a0, double* csr_val, unsigned* status, cudaStream_t s) {
  int rc = launch_rows_geometry<D, FORM, T>(plan, cells, vertices, n_vert, status, s);
  if (rc != FFC_OK) return rc;
  switch (q) {
    case 1: return launch_rows_t<D, FORM, 1, T>(plan, a0, csr_val, status, s);
    case 2: return launch_rows_t<D, FORM, 2, T>(plan, a0, csr_val, status, s);
    case 3: return launch_rows_t<D, FORM, 3, T>(plan, a0, csr_val, status, s);
    case 4: return launch_rows_t<D, FORM, 4, T>(plan, a0, csr_val, status, s);
    default: return FFC_EUNSUPPORTED;
  }
}

template <typename T>
int launch_rows_form(const ffc_form* f, const ffc_row_plan* plan, const int32_t* cells, const double* vertices,
                     int64_t n_vert, const void* a0, double* csr_val, unsigned* status, cudaStream_t s) {
  if (f->d == 3) {
    if (f->kind == FFC_MASS) return launch_rows_q<3, FFC_MASS, T>(plan, f->q, cells, vertices, n_vert, a0, csr_val, status, s);
    return launch_rows_q<3, FFC_POISSON, T>(plan, f->q, cells, vertices, n_vert, a0, csr_val, status, s);
  }
  if (f->kind == FFC_MASS) return launch_rows_q<2, FFC_MASS, T>(plan, f->q, cells, vertices, n_vert, a0, csr_val, status, s);
  return launch_rows_q<2, FFC_POISSON, T>(plan, f->q, cells, vertices, n_vert, a0, csr_val, status, s);
}

void free_plan(ffc_row_plan* p) {
  if (!p) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  cudaFree(p->row_ptr);
  cudaFree(p->inc_ptr);
  cudaFree(p->inc);
  cudaFree(p->pos);
  cudaFree(p->geom);
  cudaSetDevice(cur);
  delete p;
}

template <typename T>
int dev_alloc(T** p, size_t count) {
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T));
  return e == cudaSuccess ? FFC_OK : cuda_fail(e, "cudaMalloc");
}

}  // namespace
}  // namespace ffc

using namespace ffc;

extern "C" {

int ffc_row_plan_create(int64_t n_elem, int n_local, const int32_t* dofmap, int64_t n_dof, const int64_t* row_ptr,
                        const int32_t* col, int64_t nnz, void* stream, ffc_row_plan** out) {
  if (!out || n_elem < 0 || n_local < 1 || n_local > 4096 || n_dof < 1 || n_dof >= INT32_MAX || nnz < 0 ||
      !row_ptr || (n_elem > 0 && !dofmap) || (nnz > 0 && !col)) {
    set_error("ffc_row_plan_create: invalid argument");
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
  int32_t *inc_tmp = nullptr, *fill = nullptr, *sums = nullptr;
  int* meta = nullptr;  // err, max_row, max_incidence
  int rc = FFC_OK;
  cudaError_t e = cudaSuccess;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  const unsigned grid = unsigned(sms > 0 ? sms * 8 : 1024);
  int host_meta[3] = {0, 0, 0};
  if ((rc = dev_alloc(&p->row_ptr, size_t(n_dof) + 1)) || (rc = dev_alloc(&p->inc_ptr, size_t(n_dof) + 1)) ||
      (rc = dev_alloc(&p->inc, size_t(total) + 4)) || (rc = dev_alloc(&p->pos, size_t(total) * n_local + 8)) ||
      (rc = dev_alloc(reinterpret_cast<double**>(&p->geom), size_t(n_elem) * 8)) ||
      (rc = dev_alloc(&inc_tmp, size_t(total))) || (rc = dev_alloc(&fill, size_t(n_dof))) ||
      (rc = dev_alloc(&sums, size_t(nb))) || (rc = dev_alloc(&meta, 3)))
    goto fail;
  if ((e = cudaMemcpyAsync(p->row_ptr, row_ptr, (size_t(n_dof) + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                           s)) != cudaSuccess ||
      (e = cudaMemsetAsync(p->inc_ptr, 0, (size_t(n_dof) + 1) * sizeof(int32_t), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(fill, 0, size_t(n_dof) * sizeof(int32_t), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(meta, 0, 3 * sizeof(int), s)) != cudaSuccess) {
    rc = cuda_fail(e, "ffc_row_plan_create: memset");
    goto fail;
  }
  if (total > 0) plan_count<<<grid, 256, 0, s>>>(dofmap, total, n_dof, p->inc_ptr, reinterpret_cast<unsigned*>(meta));
  scan_chunks<<<unsigned(nb), SCAN_T, 0, s>>>(p->inc_ptr, n_dof + 1, sums);
  scan_sums<<<1, SCAN_T, 0, s>>>(sums, int(nb));
  scan_add<<<unsigned(nb), SCAN_T, 0, s>>>(p->inc_ptr, n_dof + 1, sums);
  if (total > 0) plan_fill<<<grid, 256, 0, s>>>(dofmap, total, n_dof, p->inc_ptr, fill, inc_tmp);
  plan_rows<<<grid, 256, 0, s>>>(dofmap, n_local, n_dof, p->row_ptr, col, nnz, p->inc_ptr, inc_tmp, p->inc, p->pos,
                                 meta + 1, meta + 2, reinterpret_cast<unsigned*>(meta));
  if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaMemcpyAsync(host_meta, meta, sizeof(host_meta),
                                                                      cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    rc = cuda_fail(e, "ffc_row_plan_create");
    goto fail;
  }
  if (host_meta[0] & int(PLAN_LONG_ROW | PLAN_BAD_ROW_PTR)) {  // a malformed pattern comes first
    set_error(host_meta[0] & int(PLAN_BAD_ROW_PTR) ? "ffc_row_plan_create: row_ptr is not monotone within [0, nnz]"
                                                    : "ffc_row_plan_create: a row has more than 65535 entries");
    rc = FFC_EINVAL;
    goto fail;
  }
  if (host_meta[0] & int(PLAN_BAD_DOF | PLAN_MISSING)) {
    set_error(host_meta[0] & int(PLAN_BAD_DOF) ? "ffc_row_plan_create: dof id out of range"
                                                : "ffc_row_plan_create: a (row, col) pair is not in the pattern");
    rc = FFC_EBOUNDS;
    goto fail;
  }
  p->max_row = host_meta[1];
  p->max_incidence = host_meta[2];
  cudaFree(inc_tmp);
  cudaFree(fill);
  cudaFree(sums);
  cudaFree(meta);
  *out = p;
  return FFC_OK;
fail:
  cudaStreamSynchronize(s);
  cudaFree(inc_tmp);
  cudaFree(fill);
  cudaFree(sums);
  cudaFree(meta);
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

void ffc_row_plan_destroy(ffc_row_plan* p) { free_plan(p); }

int ffc_assemble_rows(const ffc_form* f, const ffc_row_plan* plan, const int32_t* cells, const double* vertices,
                      int64_t n_vert, double* csr_val, int precision, void* stream) {
  if (!f || !plan || n_vert < 0 || (precision != FFC_FP64 && precision != FFC_FP32)) {
    set_error("ffc_assemble_rows: invalid argument");
    return FFC_EINVAL;
  }
  if ((f->kind != FFC_MASS && f->kind != FFC_POISSON) || f->rank != 2) {
    set_error("ffc_assemble_rows: mass and Poisson forms only");
    return FFC_EUNSUPPORTED;
  }
  if (f->n != plan->n_local) {
    set_error("ffc_assemble_rows: the plan was built for another number of local dofs");
    return FFC_EINVAL;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != plan->device) {
    set_error("ffc_assemble_rows: the plan lives on another device");
    return FFC_EINVAL;
  }
  if (plan->nnz == 0) return FFC_OK;
  if (!csr_val || (reinterpret_cast<uintptr_t>(csr_val) & 7) ||
      (plan->n_elem > 0 && (!cells || !vertices || n_vert == 0 || (reinterpret_cast<uintptr_t>(cells) & 15) ||
                            (reinterpret_cast<uintptr_t>(vertices) & 7)))) {
    set_error("ffc_assemble_rows: null or misaligned pointer");
    return FFC_EINVAL;
  }
  DeviceTensors* t = nullptr;
  int rc = ensure_device_tensors(const_cast<ffc_form*>(f), &t);
  if (rc != FFC_OK) return rc;
  uint32_t* st = status_word();
  if (!st) {
    set_error("status word allocation failed");
    return FFC_ECUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == FFC_FP32)
    return launch_rows_form<float>(f, plan, cells, vertices, n_vert, t->a0_f32, csr_val, st, s);
  return launch_rows_form<double>(f, plan, cells, vertices, n_vert, t->a0_f64, csr_val, st, s);
}

}  // extern "C"
