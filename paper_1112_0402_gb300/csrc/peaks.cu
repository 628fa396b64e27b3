// Measured compute ceilings of the GPU the library runs on: the denominators of the
// ALU-, tensor- and shared-atomic-bound roofline fractions that the benchmark reports.
//
//   FP64 / FP32 FMA     every thread runs eight independent fused multiply-add chains
//                       (2 flops each); 1024 resident threads per SM;
//   TF32 / BF16 MMA     one CTA per SM; one thread issues back-to-back dense
//                       tcgen05.mma (M = 128, N = 256, K = 8 for kind::tf32, 16 for
//                       kind::f16 with BF16 inputs, FP32 accumulation in TMEM) on
//                       operands resident in shared memory, then commits to an
//                       mbarrier that every thread waits on with a bounded wait;
//   shared atomics      32-bit integer atomic adds to shared memory, 32 consecutive
//                       addresses per warp instruction (no bank conflicts).
// INT8 MMA (kind::i8) is not offered: the sm_103a instruction set does not have it.
#include <cuda_runtime.h>

#include <string>

#include "ffc_internal.h"
#include "tc_ptx.cuh"

namespace ffc {
namespace {

constexpr int FMA_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe(T* out, long long iters, T x, T y) {
  T a[FMA_CHAINS];
#pragma unroll
  for (int j = 0; j < FMA_CHAINS; ++j) a[j] = T(threadIdx.x + j) * T(1e-3);
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < FMA_CHAINS; ++j) a[j] = fma(a[j], x, y);
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < FMA_CHAINS; ++j) s += a[j];
  if (s == T(-1234.5)) out[blockIdx.x] = s;  // never true; keeps the chains alive
}

__global__ void __launch_bounds__(1024) smem_atomic_probe(unsigned* out, int iters) {
  __shared__ unsigned s[4096];
  for (int i = threadIdx.x; i < 4096; i += blockDim.x) s[i] = 0;
  __syncthreads();
  const int t = threadIdx.x;
  for (int it = 0; it < iters; ++it) atomicAdd(&s[(t + it * 64) & 4095], unsigned(it));
  __syncthreads();
  if (s[t & 4095] == 0x12345678u) out[blockIdx.x] = 1;
}

constexpr int MMA_M = 128, MMA_N = 256, MMA_ROW_BYTES = 32;  // one K-step per MMA: 32 bytes of K per row

template <bool TF32>
__global__ void __launch_bounds__(128, 1) mma_probe(long long iters, unsigned* status) {
  __shared__ __align__(1024) unsigned char As[MMA_M * MMA_ROW_BYTES];
  __shared__ __align__(1024) unsigned char Bs[MMA_N * MMA_ROW_BYTES];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ uint32_t tmem_slot;
  // small finite operands (2^-7 in every element)
  const uint32_t word = TF32 ? 0x3C000000u : 0x3C003C00u;
  for (int i = threadIdx.x; i < MMA_M * MMA_ROW_BYTES / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(As)[i] = word;
  for (int i = threadIdx.x; i < MMA_N * MMA_ROW_BYTES / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(Bs)[i] = word;
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_slot)),
                 "r"(MMA_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc::fence_proxy_async();  // the operands written above are read by the tensor cores
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  if (threadIdx.x == 0) {
    // K-major, no swizzle: core matrices of 8 rows x 16 bytes, two per row group (K),
    // leading (K) offset 128 bytes, row-group stride 256 bytes
    const uint64_t da = tc::smem_desc(tc::smem_u32(As), 128, 256);
    const uint64_t db = tc::smem_desc(tc::smem_u32(Bs), 128, 256);
    constexpr uint32_t IDESC = tc::mma_idesc(TF32, MMA_M, MMA_N);
    for (long long it = 0; it < iters; ++it) tc::mma<!TF32>(tmem, da, db, IDESC, it > 0 ? 1u : 0u);
    tc::mma_commit(tc::smem_u32(&bar));
  }
  const bool ok = tc::mbar_wait(tc::smem_u32(&bar), 0);
  if (!ok && threadIdx.x == 0) atomicOr(status, FFC_FLAG_TIMEOUT);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MMA_N));
}

int cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return FFC_ECUDA;
}

}  // namespace
}  // namespace ffc

using namespace ffc;

extern "C" int ffc_diag_peak(int kind, double* rate, double* seconds, void* stream) {
  if (!rate || kind < FFC_PEAK_FP64_FMA || kind > FFC_PEAK_SMEM_ATOMIC_U32) {
    set_error("ffc_diag_peak: invalid argument");
    return FFC_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "ffc_diag_peak");
  uint32_t* st = status_word();
  if (!st) {
    set_error("status word allocation failed");
    return FFC_ECUDA;
  }
  void* scratch = nullptr;
  if ((e = cudaMallocAsync(&scratch, size_t(sms) * 16 * sizeof(double), s)) != cudaSuccess)
    return cuda_fail(e, "ffc_diag_peak: scratch");
  // work per launch, sized for some tens of milliseconds on a GB300
  long long iters = 0;
  double per_iter = 0.0;  // operations per unit of `iters`
  auto launch = [&](long long it) {
    switch (kind) {
      case FFC_PEAK_FP64_FMA:
        fma_probe<double><<<sms * 4, 256, 0, s>>>(static_cast<double*>(scratch), it, 0.999999, 1e-7);
        break;
      case FFC_PEAK_FP32_FMA:
        fma_probe<float><<<sms * 4, 256, 0, s>>>(static_cast<float*>(scratch), it, 0.999999f, 1e-7f);
        break;
      case FFC_PEAK_TF32_MMA:
        mma_probe<true><<<sms, 128, 0, s>>>(it, st);
        break;
      case FFC_PEAK_BF16_MMA:
        mma_probe<false><<<sms, 128, 0, s>>>(it, st);
        break;
      default:
        smem_atomic_probe<<<sms * 2, 1024, 0, s>>>(static_cast<unsigned*>(scratch), int(it));
        break;
    }
  };
  switch (kind) {
    case FFC_PEAK_FP64_FMA:
      iters = 1 << 15;
      per_iter = 2.0 * FMA_CHAINS * sms * 4 * 256;
      break;
    case FFC_PEAK_FP32_FMA:
      iters = 1 << 20;
      per_iter = 2.0 * FMA_CHAINS * sms * 4 * 256;
      break;
    case FFC_PEAK_TF32_MMA:
      iters = 1 << 18;
      per_iter = 2.0 * MMA_M * MMA_N * 8 * sms;
      break;
    case FFC_PEAK_BF16_MMA:
      iters = 1 << 18;
      per_iter = 2.0 * MMA_M * MMA_N * 16 * sms;
      break;
    default:
      iters = 1 << 16;
      per_iter = double(sms) * 2 * 1024;
      break;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  float ms = 0.f;
  launch(iters / 16);  // warm-up
  if ((e = cudaEventCreate(&a)) == cudaSuccess && (e = cudaEventCreate(&b)) == cudaSuccess &&
      (e = cudaEventRecord(a, s)) == cudaSuccess) {
    launch(iters);
    if ((e = cudaPeekAtLastError()) == cudaSuccess && (e = cudaEventRecord(b, s)) == cudaSuccess &&
        (e = cudaEventSynchronize(b)) == cudaSuccess)
      e = cudaEventElapsedTime(&ms, a, b);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFreeAsync(scratch, s);
  if (e != cudaSuccess) return cuda_fail(e, "ffc_diag_peak");
  uint32_t flags = 0;
  if ((e = cudaMemcpyAsync(&flags, st, sizeof(flags), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(e, "ffc_diag_peak");
  if (flags & FFC_FLAG_TIMEOUT) {
    set_error("ffc_diag_peak: the tensor-core probe's bounded wait gave up");
    return FFC_ETIMEOUT;
  }
  *rate = per_iter * double(iters) / (double(ms) * 1e-3);
  if (seconds) *seconds = double(ms) * 1e-3;
  return FFC_OK;
}
