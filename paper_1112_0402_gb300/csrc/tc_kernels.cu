// Tensor-core (tcgen05, kind::tf32) contraction of the tensor representation
// A^K_i = A0_{i alpha} G_K^alpha (Section 3.2, eq. (tensorproduct)), batched over
// cells as one GEMM (the level-3 BLAS formulation proposed in Section 3.5):
//
//     D[i][e] = sum_alpha A0[i][alpha] * G[e][alpha]        (M = entries i, N = cells e)
//
// Orientation: the MMA's M dimension runs over element-tensor entries i (128 per
// M-tile) and N over 128 cells, so a TMEM lane holds one entry for 128 cells.
// In the epilogue warp w reads lanes 32w..32w+31 and, for each cell, stores 32
// consecutive entries of that cell's row-major A_K block: coalesced 128-byte stores.
//
// Per CTA (128 threads, persistent over cell tiles):
//   1. each thread computes one cell's geometry and G_K in FP64, rounds it to TF32
//      (and the TF32 remainder for the split product) and writes it into the B tile
//      (canonical K-major, no-swizzle core-matrix layout);
//   2. per M-tile, thread 0 issues a bulk TMA copy of the pre-laid-out A0 tile
//      (hi and lo parts) into shared memory, waits on an mbarrier, issues the
//      tcgen05.mma chain (1 or 3 products per K-step of 8), and commits it to a
//      second mbarrier;
//   3. all threads wait, tcgen05.ld the accumulator and store (or atomically add)
//      the results.
// Every mbarrier wait is bounded; on expiry the kernel sets FFC_FLAG_TIMEOUT,
// waits (bounded) for its own work in flight, frees its TMEM and returns.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "ffc_internal.h"
#include "geometry.cuh"

namespace ffc {

namespace tc {

constexpr int M_TILE = 128;   // entries per M-tile (TMEM lanes)
constexpr int N_CELLS = 128;  // cells per tile (MMA N, TMEM columns)
constexpr int THREADS = 128;
constexpr uint32_t WAIT_LIMIT = 1u << 24;

__host__ __device__ constexpr int kpad(int na) { return (na + 7) / 8 * 8; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major, no-swizzle core-matrix layout: 8 rows x 16 bytes per core matrix; core
// matrix (row_group, k_group) at ((row_group * KC) + k_group) * 128 bytes. The
// leading (K) byte offset is 128, the stride (row-group) byte offset KC*128.
__host__ __device__ __forceinline__ uint32_t core_offset_floats(int row, int k, int kc) {
  return uint32_t(((row >> 3) * kc + (k >> 2)) * 32 + (row & 7) * 4 + (k & 3));
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= uint64_t((addr & 0x3FFFF) >> 4);
  d |= uint64_t((lbo >> 4) & 0x3FFF) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFF) << 32;
  d |= uint64_t(1) << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, no swizzle
}

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded wait: true when the phase completed, false after WAIT_LIMIT polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  for (uint32_t it = 0; it < WAIT_LIMIT; ++it)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

struct TcParams {
  const int32_t* cells;
  const double* vertices;
  long long n_vert;
  const double* coeffs;
  const float* a0_hi;  // [MT][128 x KPAD] core-matrix layout per M-tile
  const float* a0_lo;
  float* out;          // A_K [n_elem][NN]
  const int32_t* slot;
  double* csr_val;
  long long nnz;
  long long n_elem;
  double mu, lambda;
  unsigned* status;
};

template <int D, int FORM, int Q, int NPROD>
struct TcCfg {
  static constexpr int N = nlocal(FORM, D, Q);
  static constexpr int NN = N * N;
  static constexpr int NA = nalpha(FORM, D, Q);
  static constexpr int KPAD = kpad(NA);
  static constexpr int KC = KPAD / 4;
  static constexpr int MT = (NN + M_TILE - 1) / M_TILE;
  static constexpr uint32_t A_BYTES = M_TILE * KPAD * 4;
  static constexpr uint32_t B_BYTES = N_CELLS * KPAD * 4;
  static constexpr int NBUF = NPROD == 3 ? 2 : 1;  // hi (+ lo)
  static constexpr size_t SMEM = size_t(NBUF) * (A_BYTES + B_BYTES) + 128 + 128;
};

template <int D, int FORM, int Q, int NPROD, bool ASSEMBLE>
__global__ void __launch_bounds__(THREADS, 1) tc_tabulate_kernel(TcParams p) {
  using C = TcCfg<D, FORM, Q, NPROD>;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* As_hi = reinterpret_cast<float*>(smem);
  float* As_lo = As_hi + (NPROD == 3 ? M_TILE * C::KPAD : 0);
  float* Bs_hi = reinterpret_cast<float*>(smem + C::NBUF * C::A_BYTES);
  float* Bs_lo = Bs_hi + (NPROD == 3 ? N_CELLS * C::KPAD : 0);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::NBUF * (C::A_BYTES + C::B_BYTES));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4);
  __shared__ int abort_flag;

  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int lane = t & 31;
  const uint32_t bar_load = smem_u32(&bars[0]);
  const uint32_t bar_mma = smem_u32(&bars[1]);

  if (t == 0) {
    mbar_init(bar_load, 1);
    mbar_init(bar_mma, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(uint32_t(N_CELLS)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t IDESC = idesc_tf32(M_TILE, N_CELLS);
  uint32_t ph_load = 0, ph_mma = 0;
  bool timed_out = false;
  int pending = 0;  // thread 0: 1 = a bulk copy may still be in flight, 2 = an MMA chain may be

  const long long n_tiles = (p.n_elem + N_CELLS - 1) / N_CELLS;
  for (long long tile = blockIdx.x; tile < n_tiles && !timed_out; tile += gridDim.x) {
    const long long e0 = tile * N_CELLS;
    // ---- 1. geometry tensor of cell e0 + t -> B tile row t
    {
      const long long e = e0 + t;
      double g[C::NA];
      if (e < p.n_elem) {
        double K[D][D], det;
        bool degenerate, bad_index;
        cell_geometry<D>(p.cells, p.vertices, p.n_vert, e, K, det, degenerate, bad_index);
        if (degenerate) atomicOr(p.status, FFC_FLAG_DEGENERATE);
        if (bad_index) atomicOr(p.status, FFC_FLAG_BOUNDS);
        const double* w = (C::NA > 0 && FORM == FFC_NS_CONVECTION) ? p.coeffs + e * C::N : nullptr;
        double wl[FORM == FFC_NS_CONVECTION ? C::N : 1];
        if constexpr (FORM == FFC_NS_CONVECTION) {
#pragma unroll
          for (int k = 0; k < C::N; ++k) wl[k] = __ldg(w + k);
        }
        geometry_tensor<D, FORM, Q>(K, det, wl, p.mu, p.lambda, [&](int a, double v) { g[a] = v; });
      } else {
#pragma unroll
        for (int a = 0; a < C::NA; ++a) g[a] = 0.0;
      }
#pragma unroll
      for (int k = 0; k < C::KPAD; ++k) {
        const double v = k < C::NA ? g[k] : 0.0;
        const float hi = tf32_rna(float(v));
        Bs_hi[core_offset_floats(t, k, C::KC)] = hi;
        if constexpr (NPROD == 3) Bs_lo[core_offset_floats(t, k, C::KC)] = tf32_rna(float(v - double(hi)));
      }
    }
    fence_proxy_async();
    __syncthreads();

    for (int mt = 0; mt < C::MT; ++mt) {
      // ---- 2. stage the A0 M-tile and run the MMA chain
      if (t == 0) {
        mbar_expect_tx(bar_load, C::NBUF * C::A_BYTES);
        bulk_g2s(smem_u32(As_hi), p.a0_hi + size_t(mt) * M_TILE * C::KPAD, C::A_BYTES, bar_load);
        if constexpr (NPROD == 3)
          bulk_g2s(smem_u32(As_lo), p.a0_lo + size_t(mt) * M_TILE * C::KPAD, C::A_BYTES, bar_load);
        bool ok = mbar_wait(bar_load, ph_load);
        if (ok) {
          fence_after();
          const uint32_t a_hi = smem_u32(As_hi), a_lo = smem_u32(As_lo);
          const uint32_t b_hi = smem_u32(Bs_hi), b_lo = smem_u32(Bs_lo);
          constexpr uint32_t SBO = C::KC * 128;
#pragma unroll 1
          for (int ks = 0; ks < C::KPAD / 8; ++ks) {
            const uint32_t off = ks * 256;  // 8 TF32 columns = two core matrices along K
            const uint64_t dah = smem_desc(a_hi + off, 128, SBO), dbh = smem_desc(b_hi + off, 128, SBO);
            if constexpr (NPROD == 3) {
              const uint64_t dal = smem_desc(a_lo + off, 128, SBO), dbl = smem_desc(b_lo + off, 128, SBO);
              mma_tf32(tmem, dal, dbh, IDESC, ks > 0 ? 1u : 0u);
              mma_tf32(tmem, dah, dbl, IDESC, 1u);
              mma_tf32(tmem, dah, dbh, IDESC, 1u);
            } else {
              mma_tf32(tmem, dah, dbh, IDESC, ks > 0 ? 1u : 0u);
            }
          }
          mma_commit(bar_mma);
        } else {
          atomicOr(p.status, FFC_FLAG_TIMEOUT);
          abort_flag = 1;
          pending = 1;
        }
      }
      ph_load ^= 1;
      __syncthreads();
      if (abort_flag) {
        timed_out = true;
        break;
      }
      // ---- 3. wait for the accumulator, then the epilogue
      bool ok = mbar_wait(bar_mma, ph_mma);
      ph_mma ^= 1;
      if (__syncthreads_or(!ok)) {
        if (t == 0) {
          atomicOr(p.status, FFC_FLAG_TIMEOUT);
          pending = 2;
        }
        timed_out = true;
        break;
      }
      fence_after();
      const int i = mt * M_TILE + warp * 32 + lane;
      const uint32_t taddr = tmem + (uint32_t(warp * 32) << 16);
#pragma unroll 1
      for (int c = 0; c < N_CELLS / 16; ++c) {
        float v[16];
        tmem_ld16(taddr + c * 16, v);
        if (i < C::NN) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const long long e = e0 + c * 16 + j;
            if (e < p.n_elem) {
              const long long o = e * C::NN + i;
              if constexpr (ASSEMBLE) {
                const int s = __ldg(p.slot + o);
                if (s >= 0 && s < p.nnz) atomicAdd(p.csr_val + s, double(v[j]));
                else atomicOr(p.status, FFC_FLAG_BOUNDS);
              } else {
                __stcs(p.out + o, v[j]);
              }
            }
          }
        }
      }
      fence_before();
      __syncthreads();
    }
  }
  if (timed_out) {
    // give the copy or MMA chain still in flight a bounded time to land before the
    // shared memory and TMEM are released
    if (t == 0 && pending == 1) mbar_wait(bar_load, ph_load ^ 1);
    if (t == 0 && pending == 2) mbar_wait(bar_mma, ph_mma ^ 1);
    __syncthreads();
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(uint32_t(N_CELLS)));
  }
}

// Host: round-to-nearest (ties away) to TF32, the rounding of cvt.rna.tf32.f32.
inline float host_tf32(double x) {
  float f = float(x);
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u = (u + 0x1000u) & ~0x1FFFu;
  std::memcpy(&f, &u, 4);
  return f;
}

template <int D, int FORM, int Q, int NPROD, bool ASSEMBLE>
int launch_one(const LaunchArgs& a) {
  using C = TcCfg<D, FORM, Q, NPROD>;
  ffc_form* f = const_cast<ffc_form*>(a.f);
  DeviceTensors* t = const_cast<DeviceTensors*>(a.t);
  {
    std::lock_guard<std::mutex> g(f->lock);
    if (!t->b_hi || t->k_pad != C::KPAD) {
      const int nn = C::NN, na = C::NA;
      std::vector<float> hi(size_t(C::MT) * M_TILE * C::KPAD, 0.f), lo(hi.size(), 0.f);
      for (int i = 0; i < nn; ++i)
        for (int k = 0; k < na; ++k) {
          const double v = f->A0[size_t(i) * na + k];
          const int mt = i / M_TILE, r = i % M_TILE;
          const size_t o = size_t(mt) * M_TILE * C::KPAD + core_offset_floats(r, k, C::KC);
          hi[o] = host_tf32(v);
          lo[o] = host_tf32(v - double(hi[o]));
        }
      cudaFree(t->b_hi);
      cudaFree(t->b_lo);
      t->b_hi = t->b_lo = nullptr;
      if (cudaMalloc(&t->b_hi, hi.size() * 4) != cudaSuccess) return FFC_ENOMEM;
      if (cudaMalloc(&t->b_lo, lo.size() * 4) != cudaSuccess) return FFC_ENOMEM;
      if (cudaMemcpy(t->b_hi, hi.data(), hi.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) return FFC_ECUDA;
      if (cudaMemcpy(t->b_lo, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) return FFC_ECUDA;
      t->k_pad = C::KPAD;
      t->nn_pad = C::MT * M_TILE;
    }
  }
  TcParams p{};
  p.cells = a.cells;
  p.vertices = a.vertices;
  p.n_vert = a.n_vert;
  p.coeffs = a.coeffs;
  p.a0_hi = t->b_hi;
  p.a0_lo = t->b_lo;
  p.out = static_cast<float*>(a.out);
  p.slot = a.slot;
  p.csr_val = a.csr_val;
  p.nnz = a.nnz;
  p.n_elem = a.n_elem;
  p.mu = a.f->mu;
  p.lambda = a.f->lambda;
  p.status = a.status;
  auto kern = tc_tabulate_kernel<D, FORM, Q, NPROD, ASSEMBLE>;
  static int sms = 0;
  if (sms == 0) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM)) != cudaSuccess)
      return FFC_ECUDA;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const long long n_tiles = (a.n_elem + N_CELLS - 1) / N_CELLS;
  long long grid = sms;
  if (grid > n_tiles) grid = n_tiles;
  kern<<<unsigned(grid), THREADS, C::SMEM, static_cast<cudaStream_t>(a.stream)>>>(p);
  return cudaPeekAtLastError() == cudaSuccess ? FFC_OK : FFC_ECUDA;
}

template <int D, int FORM, int Q>
int by_prec(const LaunchArgs& a, int precision, bool assemble) {
  if (precision == FFC_TF32)
    return assemble ? launch_one<D, FORM, Q, 1, true>(a) : launch_one<D, FORM, Q, 1, false>(a);
  return assemble ? launch_one<D, FORM, Q, 3, true>(a) : launch_one<D, FORM, Q, 3, false>(a);
}

}  // namespace tc

int launch_tc(const LaunchArgs& a, int precision, bool assemble) {
  const ffc_form* f = a.f;
  if (f->d != 3) return FFC_EUNSUPPORTED;
  switch (f->kind) {
    case FFC_NS_CONVECTION:
      if (f->q == 2) return tc::by_prec<3, FFC_NS_CONVECTION, 2>(a, precision, assemble);
      break;
    case FFC_ELASTICITY:
      if (f->q == 1) return tc::by_prec<3, FFC_ELASTICITY, 1>(a, precision, assemble);
      if (f->q == 2) return tc::by_prec<3, FFC_ELASTICITY, 2>(a, precision, assemble);
      if (f->q == 3) return tc::by_prec<3, FFC_ELASTICITY, 3>(a, precision, assemble);
      break;
    case FFC_POISSON:
      if (f->q == 2) return tc::by_prec<3, FFC_POISSON, 2>(a, precision, assemble);
      if (f->q == 3) return tc::by_prec<3, FFC_POISSON, 3>(a, precision, assemble);
      if (f->q == 4) return tc::by_prec<3, FFC_POISSON, 4>(a, precision, assemble);
      break;
    case FFC_MASS:
      if (f->q == 3) return tc::by_prec<3, FFC_MASS, 3>(a, precision, assemble);
      if (f->q == 4) return tc::by_prec<3, FFC_MASS, 4>(a, precision, assemble);
      break;
  }
  return FFC_EUNSUPPORTED;
}

}  // namespace ffc
