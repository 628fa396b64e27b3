// The insertion step of Algorithm 2 (Section 2.2) on its own: precomputed element
// tensors are added into the CSR values, csr_val[slot[e][i]] += A_K[e][i], with FP64
// atomic adds. ffc_assemble fuses the same step into the contraction's epilogue; this
// kernel serves element tensors that come from elsewhere (ffc_tabulate, another code)
// and measures the insertion alone.
//
// The element tensors and slots are one flat stream of n_elem * n_entries values. At
// each step a warp takes 32 consecutive entries per atomic instruction (consecutive
// entries of an element tensor row go to one CSR row, so an instruction touches few L2
// lines), and each thread keeps four such steps in flight (four strided loads, then four
// atomics) in a grid-stride loop. Handing a thread four consecutive entries instead
// spreads one warp instruction over about four CSR rows and ran 1.7x slower.
#include <cuda_runtime.h>

#include "ffc_internal.h"

namespace ffc {
namespace {

template <typename T>
__device__ __forceinline__ void add_one(double* csr_val, long long nnz, int s, T v, unsigned* status) {
  if (s >= 0 && s < nnz) atomicAdd(csr_val + s, double(v));
  else atomicOr(status, FFC_FLAG_BOUNDS);
}

template <typename T>
__global__ void __launch_bounds__(256) scatter_add_kernel(const T* __restrict__ a, const int32_t* __restrict__ slot,
                                                          double* csr_val, long long nnz, long long total,
                                                          unsigned* status) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; k0 < total; k0 += 4 * stride) {
    int s[4];
    T v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long k = k0 + j * stride;
      s[j] = k < total ? __ldg(slot + k) : 0;
      v[j] = k < total ? __ldg(a + k) : T(0);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (k0 + j * stride < total) add_one(csr_val, nnz, s[j], v[j], status);
  }
}

template <typename T>
int run(const void* a, const int32_t* slot, double* csr_val, long long nnz, long long total, unsigned* status,
        cudaStream_t s) {
  int sms = 0;
  if (launch_config(reinterpret_cast<const void*>(scatter_add_kernel<T>), 256, 0, -1, &sms, nullptr) != FFC_OK)
    return FFC_ECUDA;
  long long grid = (total + 4 * 256 - 1) / (4 * 256);
  const long long cap = (long long)sms * 8;  // 8 CTAs of 256 threads per SM, grid-stride beyond
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  scatter_add_kernel<T><<<unsigned(grid), 256, 0, s>>>(static_cast<const T*>(a), slot, csr_val, nnz, total, status);
  return cudaPeekAtLastError() == cudaSuccess ? FFC_OK : FFC_ECUDA;
}

}  // namespace

int launch_scatter_add(const void* a, int precision, const int32_t* slot, double* csr_val, long long nnz,
                       long long total, unsigned* status, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return precision == FFC_FP64 ? run<double>(a, slot, csr_val, nnz, total, status, s)
                               : run<float>(a, slot, csr_val, nnz, total, status, s);
}

}  // namespace ffc
