// Shared parts of the tensor-core (tcgen05) kernels: tile sizes, the split-precision
// modes and their operand roundings (device and host), bounded mbarrier waits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <type_traits>

#include "tc_ptx.cuh"

namespace ffc {
namespace tc {

constexpr int M_TILE = 128;   // entries per M-tile (TMEM lanes)
constexpr int N_CELLS = 128;  // cells per tile (MMA N, TMEM columns)

// Operand element handling per split mode. Core matrices are 8 rows x 16 bytes
// (4 TF32 or 8 BF16 values per row); core matrix (row_group, k_group) sits at
// ((row_group * KC) + k_group) * 128 bytes, so the leading (K) byte offset is 128 and
// the stride (row-group) byte offset KC * 128.
enum { MODE_TF32 = 1, MODE_TF32X3 = 3, MODE_BF16X3 = 6 };

template <int MODE>
struct Split {
  static constexpr bool BF16 = MODE == MODE_BF16X3;
  static constexpr int PARTS = MODE == MODE_TF32 ? 1 : (MODE == MODE_TF32X3 ? 2 : 3);
  static constexpr int EPC = BF16 ? 8 : 4;         // elements per 16-byte core row
  static constexpr int KSTEP = BF16 ? 16 : 8;      // K per MMA instruction
  static constexpr int ESIZE = BF16 ? 2 : 4;
  using Store = typename std::conditional<BF16, uint16_t, uint32_t>::type;
  // products (A part, B part), smallest first
  static constexpr int NPROD = MODE;
  __host__ __device__ static constexpr int pa(int k) {
    return MODE == MODE_TF32 ? 0 : MODE == MODE_TF32X3 ? (k == 0 ? 1 : 0)
         : (k == 0 ? 2 : k == 1 ? 1 : k == 2 ? 0 : k == 3 ? 1 : 0);
  }
  __host__ __device__ static constexpr int pb(int k) {
    return MODE == MODE_TF32 ? 0 : MODE == MODE_TF32X3 ? (k == 1 ? 1 : 0)
         : (k == 0 ? 0 : k == 1 ? 1 : k == 2 ? 2 : k == 3 ? 0 : k == 4 ? 1 : 0);
  }
  static constexpr uint32_t idesc(int m, int n) { return mma_idesc(!BF16, m, n); }
};

// Bounded wait that also gives up when another role has aborted.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t phase, volatile int* abort_flag,
                                                   uint32_t limit = WAIT_LIMIT) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, phase)) return true;
    if ((it & 1023u) == 1023u && *abort_flag) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <int MODE>
__device__ __forceinline__ void split_f32(float x, typename Split<MODE>::Store (&out)[3]) {
  float r = x;
#pragma unroll
  for (int k = 0; k < Split<MODE>::PARTS; ++k) {
    if constexpr (Split<MODE>::BF16) {
      out[k] = __bfloat16_as_ushort(__float2bfloat16_rn(r));
      r -= __uint_as_float(uint32_t(out[k]) << 16);
    } else {
      uint32_t b;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b) : "f"(r));
      out[k] = b;
      r -= __uint_as_float(b);
    }
  }
}

// Host rounding of the operand parts (the same roundings the device applies):
// TF32 = round to nearest, ties away, on the 13 dropped bits (cvt.rna.tf32.f32);
// BF16 = round to nearest even on the 16 dropped bits (__float2bfloat16_rn).
inline uint32_t host_tf32_bits(double x) {
  float f = float(x);
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (u + 0x1000u) & ~0x1FFFu;
}
inline uint16_t host_bf16_bits(double x) {
  float f = float(x);
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return uint16_t(u >> 16);
}
inline double host_value(uint32_t b) {
  float f;
  std::memcpy(&f, &b, 4);
  return f;
}

}  // namespace tc
}  // namespace ffc
