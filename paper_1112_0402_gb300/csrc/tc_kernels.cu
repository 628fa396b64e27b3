// Tensor-core (tcgen05, kind::tf32 / kind::f16 with BF16) contraction of the tensor representation
// A^K_i = A0_{i alpha} G_K^alpha (Section 3.2, eq. (tensorproduct)), batched over
// cells as one GEMM (the level-3 BLAS formulation proposed in Section 3.5):
//
//     D[i][e] = sum_alpha A0[i][alpha] * G[e][alpha]        (M = entries i, N = cells e)
//
// Orientation: the MMA's M dimension runs over element-tensor entries i (128 per
// M-tile) and N over 128 cells, so a TMEM lane holds one entry for 128 cells; a warp's
// tcgen05.ld column is 32 consecutive entries of one cell's row-major A_K block, stored
// as one coalesced 128-byte write.
//
// A0 is pre-laid-out on the host per (M-tile, K-chunk of 32) in the canonical K-major,
// no-swizzle core-matrix layout, so one 1-D bulk copy per operand part stages a chunk;
// a ring of up to 8 chunk stages in shared memory keeps several copies in flight ahead
// of the MMAs. G (operand B, 128 cells x all of K) stays resident per cell tile.
// Warp roles, the barriers and the split-precision modes are described at the kernel.
// Split-precision modes (x = sum of parts, products summed smallest first):
//   TF32     x ~ t1                     1 product   (kind::tf32, K-step 8)
//   TF32X3   x ~ t1 + t2                3 products  t2*t1, t1*t2, t1*t1
//   BF16X3   x ~ b1 + b2 + b3           6 products  b3b1, b2b2, b1b3, b2b1, b1b2, b1b1
//                                                   (kind::f16 with BF16, K-step 16)
// Every part is the round-to-nearest of the remainder left by the previous parts.
// Every mbarrier wait is bounded; on expiry the kernel sets FFC_FLAG_TIMEOUT,
// waits (bounded) for its own work in flight, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#include "ffc_internal.h"
#include "geometry.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace ffc {

namespace tc {


struct TcParams {
  const int32_t* cells;
  const double* vertices;
  long long n_vert;
  const double* coeffs;
  const void* a0_part[3];  // each [MT][128 x KPAD] in core-matrix layout
  float* out;              // A_K [n_elem][NN]
  const int32_t* slot;
  double* csr_val;
  long long nnz;
  long long n_elem;
  double mu, lambda;
  unsigned* status;
};

template <int D, int FORM, int Q, int MODE>
struct TcCfg {
  using S = Split<MODE>;
  static constexpr int N = nlocal(FORM, D, Q);
  static constexpr int NN = N * N;
  static constexpr int NA = nalpha(FORM, D, Q);
  // K per staged A0 chunk: 16 (a multiple of both MMA K steps, 8 for TF32 and 16 for
  // BF16) for forms with |alpha| <= 16 (mass 1, Poisson 4 or 9), whose K then pads to 16
  // instead of 32; 32 for the vector forms
  static constexpr int KCH = NA <= 16 ? 16 : 32;
  static constexpr int KPAD = (NA + KCH - 1) / KCH * KCH;  // a whole number of chunks
  static constexpr int KC = KPAD / S::EPC;                 // core-matrix columns of B
  static constexpr int NCH = KPAD / KCH;                   // A0 chunks per M-tile
  static constexpr int KCC = KCH / S::EPC;                 // core-matrix columns per chunk
  static constexpr int MT = (NN + M_TILE - 1) / M_TILE;
  static constexpr uint32_t CH_BYTES = M_TILE * KCH * S::ESIZE;  // one part of one chunk
  static constexpr uint32_t B_BYTES = N_CELLS * KPAD * S::ESIZE;
};

// ---------------------------------------------------------------------------------
// Warp roles:
//   warps 0..3  producers (tabulate): the geometry of the NEXT cell tile (FP64 J^{-1},
//               det, then G_K in FP32, one cell per thread) is computed into registers
//               while the MMAs of the current tile still read the B buffer; once the
//               MMA warp reports the buffer free (b_empty), the split parts are written;
//   warps 4..7  drainers (tabulate): TMEM lane quarter (warp mod 4) x all 128 cell
//               columns, stores of the element tensor entries;
//               (assembly: warps 0..7 both write B and drain, atomics being latency bound)
//   warp 8      MMA: lane 0 issues the tcgen05.mma chains, one per staged A0 chunk;
//   warp 9      TMA: lane 0 streams the A0 chunks through the stage ring.
// The accumulator is double-buffered in TMEM (2 x 128 columns) so the MMA chain of
// M-tile m+1 runs while the drainers store M-tile m. Barriers:
//   a_full[s]   bulk copy into stage s landed (expect_tx)     a_empty[s]  MMAs reading stage s done
//   acc_full[b] MMAs into TMEM buffer b done                   acc_empty[b] drainers emptied buffer b
//   b_full      B tile of the current cell tile written        b_empty     MMAs reading B done
// ---------------------------------------------------------------------------------
constexpr int EPI_WARPS = 8;                 // producers (0..3) and drainers (4..7)
constexpr int EPI_THREADS = EPI_WARPS * 32;
constexpr int ROLE_THREADS = EPI_THREADS / 2;  // 128: one producer thread per cell, one drainer per TMEM lane
constexpr int MMA_WARP = EPI_WARPS, TMA_WARP = EPI_WARPS + 1;
constexpr int WS_THREADS = EPI_THREADS + 64;
constexpr int MAX_STAGES = 8;

template <int D, int FORM, int Q, int MODE>
struct TcWsCfg {
  using Base = TcCfg<D, FORM, Q, MODE>;
  using S = Split<MODE>;
  static constexpr size_t STAGE_BYTES = size_t(S::PARTS) * Base::CH_BYTES;
  static constexpr size_t B_TOTAL = size_t(S::PARTS) * Base::B_BYTES;
  static constexpr size_t BAR_BYTES = 512;  // 2*MAX_STAGES + 6 mbarriers and the TMEM address
  static constexpr size_t BUDGET = 227 * 1024;
  static constexpr int FIT = int((BUDGET - B_TOTAL - BAR_BYTES) / STAGE_BYTES);
  static constexpr int STAGES = FIT < MAX_STAGES ? FIT : MAX_STAGES;
  static_assert(STAGES >= 2, "A0 chunk ring needs two stages");
  static constexpr size_t SMEM = STAGES * STAGE_BYTES + B_TOTAL + BAR_BYTES;
  // TMEM columns per accumulator buffer: main (+ correction) x 128 cells
  static constexpr int ACC_COLS = S::NPROD > 1 ? 2 * N_CELLS : N_CELLS;
  static constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;
};


// Writes one cell's G row (operand B row `row`) as its split parts, one 16-byte core-matrix
// row per store: a warp's 32 rows are four 128-byte core-matrix blocks, conflict free.
template <class C, int MODE>
__device__ __forceinline__ void write_b_row(unsigned char* Bs, int row, const float (&g32)[C::NA]) {
  using S = Split<MODE>;
#pragma unroll
  for (int kc = 0; kc < C::KC; ++kc) {
    uint32_t w[S::PARTS][4];
#pragma unroll
    for (int j = 0; j < S::EPC; ++j) {
      const int k = kc * S::EPC + j;
      typename S::Store parts[3];
      split_f32<MODE>(k < C::NA ? g32[k < C::NA ? k : 0] : 0.f, parts);
#pragma unroll
      for (int qq = 0; qq < S::PARTS; ++qq) {
        if constexpr (S::BF16) {
          if (j & 1) w[qq][j >> 1] |= uint32_t(parts[qq]) << 16;
          else w[qq][j >> 1] = uint32_t(parts[qq]);
        } else {
          w[qq][j] = uint32_t(parts[qq]);
        }
      }
    }
    const uint32_t o = core_offset(row, kc * S::EPC, C::KC, S::EPC) * S::ESIZE;
#pragma unroll
    for (int qq = 0; qq < S::PARTS; ++qq)
      *reinterpret_cast<uint4*>(Bs + qq * C::B_BYTES + o) = make_uint4(w[qq][0], w[qq][1], w[qq][2], w[qq][3]);
  }
}

// G_K of cell e in FP32 (zeros past the end), from the FP64 geometry.
template <class C, int D, int FORM, int Q>
__device__ __forceinline__ void cell_g32(const TcParams& p, long long e, float (&g32)[C::NA]) {
  if (e < p.n_elem) {
    float K[D][D] = {}, det;
    bool degenerate, bad_index;
    if constexpr (FORM == FFC_MASS) {  // G = |det J|: no inverse needed
      double d64;
      cell_det<D>(p.cells, p.vertices, p.n_vert, e, d64, degenerate, bad_index);
      det = float(d64);
    } else {
      cell_geometry_f32<D>(p.cells, p.vertices, p.n_vert, e, K, det, degenerate, bad_index);
    }
    if (degenerate) atomicOr(p.status, FFC_FLAG_DEGENERATE);
    if (bad_index) atomicOr(p.status, FFC_FLAG_BOUNDS);
    const double* w = FORM == FFC_NS_CONVECTION ? p.coeffs + e * C::N : nullptr;
    geometry_tensor_f32<D, FORM, Q, false>(K, det, w, p.mu, p.lambda, g32);
  } else {
#pragma unroll
    for (int a = 0; a < C::NA; ++a) g32[a] = 0.f;
  }
}

template <int D, int FORM, int Q, int MODE, bool ASSEMBLE>
__global__ void __launch_bounds__(WS_THREADS, 1) tc_ws_kernel(TcParams p) {
  using C = TcCfg<D, FORM, Q, MODE>;
  using W = TcWsCfg<D, FORM, Q, MODE>;
  using S = Split<MODE>;
  // tabulate splits the epilogue warps into producers and drainers; assembly keeps all
  // eight on both jobs (its drain is bound by atomic latency and wants every warp)
  constexpr bool SPLIT = !ASSEMBLE;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* As = smem;                                   // STAGES x PARTS x CH_BYTES
  unsigned char* Bs = smem + W::STAGES * W::STAGE_BYTES;      // PARTS x B_BYTES
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + W::STAGES * W::STAGE_BYTES + W::B_TOTAL);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 24);
  __shared__ int abort_flag;
  constexpr int BAR_A_FULL = 0, BAR_A_EMPTY = MAX_STAGES, BAR_ACC_FULL = 2 * MAX_STAGES,
                BAR_ACC_EMPTY = BAR_ACC_FULL + 2, BAR_B_FULL = BAR_ACC_EMPTY + 2, BAR_B_EMPTY = BAR_B_FULL + 1;

  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int lane = t & 31;
  auto bar = [&](int k) { return smem_u32(&bars[k]); };
  if (t == 0) {
    for (int k = 0; k < W::STAGES; ++k) {
      mbar_init(bar(BAR_A_FULL + k), 1);
      mbar_init(bar(BAR_A_EMPTY + k), 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(bar(BAR_ACC_FULL + k), 1);
      mbar_init(bar(BAR_ACC_EMPTY + k), SPLIT ? ROLE_THREADS : EPI_THREADS);
    }
    mbar_init(bar(BAR_B_FULL), SPLIT ? ROLE_THREADS : EPI_THREADS);
    mbar_init(bar(BAR_B_EMPTY), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(W::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const long long n_tiles = (p.n_elem + N_CELLS - 1) / N_CELLS;
  long long my_tiles = 0;
  if (blockIdx.x < n_tiles) my_tiles = (n_tiles - 1 - blockIdx.x) / gridDim.x + 1;
  const long long total_chunks = my_tiles * C::MT * C::NCH;  // A0 chunks this CTA consumes

  if (warp == TMA_WARP) {
    // ------------------------------------------------------------ TMA: A0 chunk ring
    if (lane == 0) {
      uint32_t ph_empty = 0;  // bit s: phase of a_empty[s]
      bool ok = true;
      for (long long g = 0; g < total_chunks && ok; ++g) {
        const int s = int(g % W::STAGES);
        if (g >= W::STAGES) {
          ok = mbar_wait_or_abort(bar(BAR_A_EMPTY + s), (ph_empty >> s) & 1u, &abort_flag);
          ph_empty ^= 1u << s;
          if (!ok) break;
        }
        const long long mc = g % (long long)(C::MT * C::NCH);  // (M-tile, chunk) of this cell tile
        mbar_expect_tx(bar(BAR_A_FULL + s), uint32_t(W::STAGE_BYTES));
#pragma unroll
        for (int q = 0; q < S::PARTS; ++q)
          bulk_g2s(smem_u32(As + s * W::STAGE_BYTES + q * C::CH_BYTES),
                   static_cast<const unsigned char*>(p.a0_part[q]) + size_t(mc) * C::CH_BYTES, C::CH_BYTES,
                   bar(BAR_A_FULL + s));
      }
      if (!ok) {
        atomicOr(p.status, FFC_FLAG_TIMEOUT);
        abort_flag = 1;
      }
    }
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      constexpr uint32_t IDESC = S::idesc(M_TILE, N_CELLS);
      constexpr uint32_t SBO_A = C::KCC * 128;  // chunk: row groups of KCC core matrices
      constexpr uint32_t SBO_B = C::KC * 128;   // B: row groups of all KC core matrices
      constexpr int KS_PER_CH = C::KCH / S::KSTEP;
      uint32_t ph_full = 0, ph_acc_empty = 0, ph_b = 0;
      bool ok = true;
      long long g = 0, gm = 0;  // chunks and M-tiles consumed
      for (long long ct = 0; ct < my_tiles && ok; ++ct) {
        ok = mbar_wait_or_abort(bar(BAR_B_FULL), ph_b, &abort_flag);
        ph_b ^= 1;
        for (int mt = 0; mt < C::MT && ok; ++mt, ++gm) {
          const int acc = int(gm & 1);
          if (gm >= 2) {
            ok = mbar_wait_or_abort(bar(BAR_ACC_EMPTY + acc), (ph_acc_empty >> acc) & 1u, &abort_flag);
            ph_acc_empty ^= 1u << acc;
            if (!ok) break;
          }
          // main product (part 0 x part 0) and the correction products accumulate
          // separately; the epilogue adds them once
          const uint32_t d_main = tmem + uint32_t(acc * W::ACC_COLS);
          const uint32_t d_corr = d_main + uint32_t(N_CELLS);
          for (int ch = 0; ch < C::NCH; ++ch, ++g) {
            const int s = int(g % W::STAGES);
            ok = mbar_wait_or_abort(bar(BAR_A_FULL + s), (ph_full >> s) & 1u, &abort_flag);
            ph_full ^= 1u << s;
            if (!ok) break;
            fence_after();
#pragma unroll
            for (int ksl = 0; ksl < KS_PER_CH; ++ksl) {
              const int ks = ch * KS_PER_CH + ksl;
#pragma unroll
              for (int k = 0; k < S::NPROD; ++k) {
                const uint64_t da =
                    smem_desc(smem_u32(As + s * W::STAGE_BYTES + S::pa(k) * C::CH_BYTES) + ksl * 256, 128, SBO_A);
                const uint64_t db = smem_desc(smem_u32(Bs + S::pb(k) * C::B_BYTES) + ks * 256, 128, SBO_B);
                if (k == S::NPROD - 1) mma<S::BF16>(d_main, da, db, IDESC, ks > 0 ? 1u : 0u);
                else mma<S::BF16>(d_corr, da, db, IDESC, (ks > 0 || k > 0) ? 1u : 0u);
              }
            }
            mma_commit(bar(BAR_A_EMPTY + s));  // the stage is free once these MMAs complete
          }
          if (!ok) break;
          mma_commit(bar(BAR_ACC_FULL + acc));
        }
        if (ok && SPLIT) mma_commit(bar(BAR_B_EMPTY));  // B free once this tile's MMAs complete
      }
      if (!ok) {
        atomicOr(p.status, FFC_FLAG_TIMEOUT);
        abort_flag = 1;
      }
      // let the last MMA chain finish before TMEM is released (bounded)
      if (g > 0) {
        const int s = int((g - 1) % W::STAGES);
        mbar_wait(bar(BAR_A_EMPTY + s), ((g - 1) / W::STAGES) & 1);
      }
    }
  } else if (SPLIT && warp < EPI_WARPS / 2) {
    // ------------------------------------------------------------ producers: G_K of each tile
    uint32_t ph_b_empty = 0;
    bool ok = true;
    for (long long ct = 0; ct < my_tiles && ok; ++ct) {
      float g32[C::NA];
      cell_g32<C, D, FORM, Q>(p, (blockIdx.x + ct * gridDim.x) * N_CELLS + t, g32);
      // the previous tile's MMAs must be done reading B before it is overwritten
      if (ct > 0) {
        ok = mbar_wait_or_abort(bar(BAR_B_EMPTY), ph_b_empty, &abort_flag);
        ph_b_empty ^= 1;
        if (!ok) break;
      }
      write_b_row<C, MODE>(Bs, t, g32);
      fence_proxy_async();
      mbar_arrive(bar(BAR_B_FULL));
    }
    if (!ok) {
      atomicOr(p.status, FFC_FLAG_TIMEOUT);
      abort_flag = 1;
    }
  } else if (SPLIT) {
    // ------------------------------------------------------------ drainers: TMEM -> HBM
    uint32_t ph_acc_full[2] = {0, 0};
    long long g = 0;
    bool ok = true;
    const int q4 = warp & 3;  // TMEM lane quarter
    for (long long ct = 0; ct < my_tiles && ok; ++ct) {
      const long long e0 = (blockIdx.x + ct * gridDim.x) * N_CELLS;
      for (int mt = 0; mt < C::MT; ++mt, ++g) {
        const int acc = int(g & 1);
        ok = mbar_wait_or_abort(bar(BAR_ACC_FULL + acc), ph_acc_full[acc], &abort_flag);
        ph_acc_full[acc] ^= 1;
        if (__any_sync(0xffffffffu, !ok)) {
          ok = false;
          break;
        }
        fence_after();
        const int i = mt * M_TILE + q4 * 32 + lane;
        const uint32_t taddr = tmem + (uint32_t(q4 * 32) << 16) + uint32_t(acc * W::ACC_COLS);
#pragma unroll 1
        for (int c = 0; c < N_CELLS / 32; ++c) {
          // 32 cell columns per step: two (four with the correction accumulator) loads in
          // flight before one wait
          uint32_t rv[32];
          float v[32];
          tmem_ld16_issue(taddr + c * 32, rv);
          tmem_ld16_issue(taddr + c * 32 + 16, rv + 16);
          if constexpr (S::NPROD > 1) {
            uint32_t rw[32];
            tmem_ld16_issue(taddr + N_CELLS + c * 32, rw);
            tmem_ld16_issue(taddr + N_CELLS + c * 32 + 16, rw + 16);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(rv[j]) + __uint_as_float(rw[j]);
          } else {
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(rv[j]);
          }
          if (i < C::NN) {
            const long long ec = e0 + c * 32;
            if constexpr (!ASSEMBLE) {
              // one base address per 32 cells; the cells' rows are constant offsets from it
              float* dst = p.out + ec * C::NN + i;
              if (ec + 32 <= p.n_elem) {
#pragma unroll
                for (int j = 0; j < 32; ++j) __stcs(dst + j * C::NN, v[j]);
              } else {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                  if (ec + j < p.n_elem) __stcs(dst + j * C::NN, v[j]);
              }
            } else {
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const long long e = ec + j;
                if (e < p.n_elem) {
                  const long long o = e * C::NN + i;
                  const int s = __ldg(p.slot + o);
                  if (s >= 0 && s < p.nnz) atomicAdd(p.csr_val + s, double(v[j]));
                  else atomicOr(p.status, FFC_FLAG_BOUNDS);
                }
              }
            }
          }
        }
        fence_before();
        mbar_arrive(bar(BAR_ACC_EMPTY + acc));
      }
    }
    if (!ok) {
      if (lane == 0) atomicOr(p.status, FFC_FLAG_TIMEOUT);
      abort_flag = 1;
    }
  } else {
    // ------------------------------------------------------------ combined epilogue (assembly)
    // warps 0..7 write the tile's B (threads 0..127, one cell each), then drain: lane
    // quarter warp mod 4, column half warp / 4
    uint32_t ph_acc_full[2] = {0, 0};
    long long g = 0;
    bool ok = true;
    const int q4 = warp & 3;
    const int half = warp >> 2;
    for (long long ct = 0; ct < my_tiles && ok; ++ct) {
      const long long e0 = (blockIdx.x + ct * gridDim.x) * N_CELLS;
      if (t < N_CELLS) {
        float g32[C::NA];
        cell_g32<C, D, FORM, Q>(p, e0 + t, g32);
        write_b_row<C, MODE>(Bs, t, g32);
        fence_proxy_async();
      }
      mbar_arrive(bar(BAR_B_FULL));
      for (int mt = 0; mt < C::MT; ++mt, ++g) {
        const int acc = int(g & 1);
        ok = mbar_wait_or_abort(bar(BAR_ACC_FULL + acc), ph_acc_full[acc], &abort_flag);
        ph_acc_full[acc] ^= 1;
        if (__any_sync(0xffffffffu, !ok)) {
          ok = false;
          break;
        }
        fence_after();
        const int i = mt * M_TILE + q4 * 32 + lane;
        const uint32_t taddr = tmem + (uint32_t(q4 * 32) << 16) + uint32_t(acc * W::ACC_COLS + half * 64);
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
          float v[16];
          tmem_ld16(taddr + c * 16, v);
          if constexpr (S::NPROD > 1) {
            float w[16];
            tmem_ld16(taddr + N_CELLS + c * 16, w);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] += w[j];
          }
          if (i < C::NN) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const long long e = e0 + half * 64 + c * 16 + j;
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
        mbar_arrive(bar(BAR_ACC_EMPTY + acc));
      }
    }
    if (!ok) {
      if (t == 0) atomicOr(p.status, FFC_FLAG_TIMEOUT);
      abort_flag = 1;
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(W::TMEM_COLS));
  }
}


template <int D, int FORM, int Q, int MODE>
int upload_parts(ffc_form* f, DeviceTensors* t) {
  using C = TcCfg<D, FORM, Q, MODE>;
  using S = Split<MODE>;
  const int fam = S::BF16 ? 1 : 0;
  std::lock_guard<std::mutex> g(f->lock);
  if (t->tc_part[fam][S::PARTS - 1] && t->tc_kpad[fam] == C::KPAD) return FFC_OK;
  const size_t per = size_t(C::MT) * M_TILE * C::KPAD;  // elements per part: [MT][NCH][128 x C::KCH] chunks
  const int nparts = S::BF16 ? 3 : 2;                    // a family uploads all its parts once
  std::vector<std::vector<typename S::Store>> parts(nparts, std::vector<typename S::Store>(per, 0));
  for (int i = 0; i < C::NN; ++i)
    for (int k = 0; k < C::NA; ++k) {
      double r = f->A0[size_t(i) * C::NA + k];
      const size_t o = (size_t(i / M_TILE) * C::NCH + k / C::KCH) * (M_TILE * C::KCH) +
                       core_offset(i % M_TILE, k % C::KCH, C::KCC, S::EPC);
      for (int q = 0; q < nparts; ++q) {
        if constexpr (S::BF16) {
          const uint16_t b = host_bf16_bits(r);
          parts[q][o] = b;
          r -= host_value(uint32_t(b) << 16);
        } else {
          const uint32_t b = host_tf32_bits(r);
          parts[q][o] = b;
          r -= host_value(b);
        }
      }
    }
  for (int q = 0; q < 3; ++q) {
    cudaFree(t->tc_part[fam][q]);
    t->tc_part[fam][q] = nullptr;
  }
  for (int q = 0; q < nparts; ++q) {
    if (cudaMalloc(&t->tc_part[fam][q], per * sizeof(typename S::Store)) != cudaSuccess) return FFC_ENOMEM;
    if (cudaMemcpy(t->tc_part[fam][q], parts[q].data(), per * sizeof(typename S::Store), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return FFC_ECUDA;
  }
  t->tc_kpad[fam] = C::KPAD;
  return FFC_OK;
}

template <int D, int FORM, int Q, int MODE, bool ASSEMBLE>
int launch_one(const LaunchArgs& a) {
  using C = TcCfg<D, FORM, Q, MODE>;
  using S = Split<MODE>;
  DeviceTensors* t = const_cast<DeviceTensors*>(a.t);
  int rc = upload_parts<D, FORM, Q, MODE>(const_cast<ffc_form*>(a.f), t);
  if (rc != FFC_OK) return rc;
  TcParams p{};
  p.cells = a.cells;
  p.vertices = a.vertices;
  p.n_vert = a.n_vert;
  p.coeffs = a.coeffs;
  for (int q = 0; q < 3; ++q) p.a0_part[q] = t->tc_part[S::BF16 ? 1 : 0][q];
  p.out = static_cast<float*>(a.out);
  p.slot = a.slot;
  p.csr_val = a.csr_val;
  p.nnz = a.nnz;
  p.n_elem = a.n_elem;
  p.mu = a.f->mu;
  p.lambda = a.f->lambda;
  p.status = a.status;
  using W = TcWsCfg<D, FORM, Q, MODE>;
  auto kern = tc_ws_kernel<D, FORM, Q, MODE, ASSEMBLE>;
  int sms = 0;
  if (launch_config(reinterpret_cast<const void*>(kern), WS_THREADS, W::SMEM, -1, &sms, nullptr) != FFC_OK)
    return FFC_ECUDA;
  const long long n_tiles = (a.n_elem + N_CELLS - 1) / N_CELLS;
  long long grid = sms;
  if (grid > n_tiles) grid = n_tiles;
  kern<<<unsigned(grid), WS_THREADS, W::SMEM, static_cast<cudaStream_t>(a.stream)>>>(p);
  (void)sizeof(C);
  return cudaPeekAtLastError() == cudaSuccess ? FFC_OK : FFC_ECUDA;
}

template <int D, int FORM, int Q>
int by_prec(const LaunchArgs& a, int precision, bool assemble) {
  switch (precision) {
    case FFC_TF32:
      return assemble ? launch_one<D, FORM, Q, MODE_TF32, true>(a) : launch_one<D, FORM, Q, MODE_TF32, false>(a);
    case FFC_TF32X3:
      return assemble ? launch_one<D, FORM, Q, MODE_TF32X3, true>(a)
                      : launch_one<D, FORM, Q, MODE_TF32X3, false>(a);
    case FFC_BF16X3:
      return assemble ? launch_one<D, FORM, Q, MODE_BF16X3, true>(a)
                      : launch_one<D, FORM, Q, MODE_BF16X3, false>(a);
  }
  return FFC_EUNSUPPORTED;
}

}  // namespace tc

// Failure-detection probe: one CTA waits, with the pipeline's bounded wait and a limit of
// `polls` tries, on an mbarrier that nothing arrives at; the wait gives up and the CTA sets
// FFC_FLAG_TIMEOUT and returns, as a pipeline role does when its partner stops.
__global__ void bounded_wait_probe_kernel(unsigned* status, uint32_t polls) {
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_u32(&bar), 1);
    abort_flag = 0;
  }
  __syncthreads();
  const bool ok = tc::mbar_wait_or_abort(tc::smem_u32(&bar), 0, &abort_flag, polls);
  if (!ok && threadIdx.x == 0) atomicOr(status, FFC_FLAG_TIMEOUT);
}

int launch_bounded_wait_probe(uint32_t polls, unsigned* status, void* stream) {
  bounded_wait_probe_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(status, polls);
  return cudaPeekAtLastError() == cudaSuccess ? FFC_OK : FFC_ECUDA;
}

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
