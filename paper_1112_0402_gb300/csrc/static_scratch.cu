// ffc_tabulate_static: the element-tensor computation of ffc_tabulate for callers
// that must not allocate device memory.
//
// Some hosts of this library cannot call cudaMalloc after start-up: a framework that
// owns all device memory through its own pool, an application whose memory budget
// is fixed before it loads plugins, or code on a latency-critical path where an
// allocation (and the implicit synchronisation it may bring) is not allowed. The
// regular entry points allocate lazily: the device copy of the reference tensor
// A0 and the device status word. This entry point keeps both in one file-scope
// device array of fixed size instead, so the call itself allocates nothing.
//
// The array lives in every GPU that loads the library until the process exits.
// Its device address is looked up once per device (cudaGetSymbolAddress, with that
// device current) on the first call there. The call refuses to run while its stream is
// being captured into a graph. Every call shares the array and leaves its contents behind: the status
// word is cleared at the start of each call and the reference tensor is rewritten,
// so calls that overlap on the GPU (different streams, different host threads)
// race with each other and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "ffc_internal.h"

namespace ffc {
namespace {

// 2 MiB of reference-tensor storage plus one 256-byte slot for the status word.
constexpr size_t kStaticA0Bytes = size_t(2) << 20;
constexpr size_t kStatusSlot = 256;
constexpr size_t kScratchBytes = kStatusSlot + kStaticA0Bytes;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_addr_lock;
unsigned char* g_addr[64] = {nullptr};

// Fills the transposed FP64 copy and both FP32 copies from the FP64 rows.
__global__ void expand_reference_tensor(double* rows64, double* cols64, float* rows32, float* cols32, int nn, int na) {
  const long long total = (long long)nn * na;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int i = int(k / na), a = int(k % na);
    const double v = rows64[k];
    cols64[(long long)a * nn + i] = v;
    rows32[k] = float(v);
    cols32[(long long)a * nn + i] = float(v);
  }
}

__global__ void narrow_to_f32(const double* src, float* dst, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    dst[k] = float(src[k]);
}

int scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    set_error("ffc_tabulate_static: no current device");
    return FFC_ECUDA;
  }
  std::lock_guard<std::mutex> g(g_addr_lock);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return FFC_ECUDA;
    }
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return FFC_OK;
}

}  // namespace
}  // namespace ffc

using namespace ffc;

extern "C" int ffc_tabulate_static(const ffc_form* f, int64_t n_elem, const int32_t* cells, const double* vertices,
                                   int64_t n_vert, const double* coeffs, void* A_K, int precision, void* stream,
                                   uint32_t* host_flags) {
  if (!f || n_elem < 0 || n_vert < 0 || (precision != FFC_FP64 && precision != FFC_FP32)) {
    set_error("ffc_tabulate_static: invalid argument (precision must be FFC_FP64 or FFC_FP32)");
    return FFC_EINVAL;
  }
  auto align = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t nn = f->n_entries(), na = size_t(f->kernel_na()), nr = f->R.size();
  const size_t need = 2 * align(nn * na * sizeof(double)) + 2 * align(nn * na * sizeof(float)) +
                      align(nr * sizeof(double)) + align(nr * sizeof(float));
  if (need > kStaticA0Bytes) {
    set_error("ffc_tabulate_static: the reference tensor needs " + std::to_string(need) +
              " bytes, more than the fixed 2 MiB scratch");
    return FFC_EINVAL;
  }
  if (host_flags) *host_flags = 0;
  if (n_elem == 0) return FFC_OK;
  if (!cells || !vertices || n_vert == 0 || !A_K || (f->ncoeff > 0 && !coeffs) ||
      (reinterpret_cast<uintptr_t>(cells) & 15) || (reinterpret_cast<uintptr_t>(vertices) & 7) ||
      (reinterpret_cast<uintptr_t>(A_K) & 15)) {
    set_error("ffc_tabulate_static: null or misaligned pointer");
    return FFC_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the reference tensor is uploaded from the form's host copy on every call: a captured
  // copy would keep that host pointer, so capture is refused rather than recorded
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    set_error("ffc_tabulate_static: not callable while the stream is being captured");
    return FFC_EINVAL;
  }
  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != FFC_OK) return rc;
  uint32_t* status = reinterpret_cast<uint32_t*>(base);
  unsigned char* p = base + kStatusSlot;
  DeviceTensors t;
  t.a0_f64 = reinterpret_cast<double*>(p);
  p += align(nn * na * sizeof(double));
  t.a0t_f64 = reinterpret_cast<double*>(p);
  p += align(nn * na * sizeof(double));
  t.a0_f32 = reinterpret_cast<float*>(p);
  p += align(nn * na * sizeof(float));
  t.a0t_f32 = reinterpret_cast<float*>(p);
  p += align(nn * na * sizeof(float));
  if (nr > 0) {  // reduced reference tensor of the block algorithm (vector forms)
    t.r_f64 = reinterpret_cast<double*>(p);
    p += align(nr * sizeof(double));
    t.r_f32 = reinterpret_cast<float*>(p);
  }
  e = cudaMemsetAsync(status, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(t.a0_f64, f->kernel_a0().data(), nn * na * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nr > 0)
    e = cudaMemcpyAsync(t.r_f64, f->R.data(), nr * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    set_error(std::string("ffc_tabulate_static: ") + cudaGetErrorString(e));
    return FFC_ECUDA;
  }
  expand_reference_tensor<<<64, 256, 0, s>>>(t.a0_f64, t.a0t_f64, t.a0_f32, t.a0t_f32, int(nn), int(na));
  if ((e = cudaPeekAtLastError()) != cudaSuccess) {
    set_error(std::string("ffc_tabulate_static: ") + cudaGetErrorString(e));
    return FFC_ECUDA;
  }
  if (nr > 0) {  // FP32 copy of R (a host conversion would need a staging buffer)
    narrow_to_f32<<<8, 256, 0, s>>>(t.r_f64, t.r_f32, (long long)nr);
    if ((e = cudaPeekAtLastError()) != cudaSuccess) {
      set_error(std::string("ffc_tabulate_static: ") + cudaGetErrorString(e));
      return FFC_ECUDA;
    }
  }
  LaunchArgs a{f, n_elem, cells, vertices, n_vert, coeffs, A_K, nullptr, nullptr, 0, &t, status, stream};
  // the same kernel choice as ffc_tabulate for the CUDA-core precisions
  rc = FFC_EUNSUPPORTED;
  if (f->kr > 0 && f->algorithm != FFC_ALG_DENSE) rc = launch_simt_block(a, precision, false);
  if (rc == FFC_EUNSUPPORTED) rc = launch_simt_tri(a, precision, false);
  if (rc == FFC_EUNSUPPORTED) rc = launch_simt_tet_mass(a, precision, false);
  if (rc == FFC_EUNSUPPORTED) rc = launch_simt_tet_poisson(a, precision, false);
  if (rc == FFC_EUNSUPPORTED) rc = launch_simt_vector(a, precision, false);
  if (rc == FFC_EUNSUPPORTED) rc = launch_simt_source(a, precision, false);
  if (rc == FFC_EUNSUPPORTED) set_error("ffc_tabulate_static: no kernel built for this form/precision");
  if (rc == FFC_ECUDA) set_error(std::string("ffc_tabulate_static: kernel launch: ") +
                                 cudaGetErrorString(cudaGetLastError()));
  if (rc != FFC_OK) return rc;
  if (host_flags) {
    e = cudaMemcpyAsync(host_flags, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error(std::string("ffc_tabulate_static: ") + cudaGetErrorString(e));
      return FFC_ECUDA;
    }
  }
  return FFC_OK;
}
