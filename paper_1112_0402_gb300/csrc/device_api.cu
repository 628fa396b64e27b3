// Device entry points of the C ABI: argument checks, lazy upload of the reference
// tensor, the library-owned status word, and dispatch to the kernels.
#include <cuda_runtime.h>

#include <climits>
#include <map>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ffc_internal.h"

namespace ffc {

namespace {
std::mutex g_status_lock;
uint32_t* g_status[64] = {nullptr};

int cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return FFC_ECUDA;
}

template <typename T>
int upload(T** dst, const std::vector<T>& src) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), src.size() * sizeof(T));
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FFC_ENOMEM : cuda_fail(e, "cudaMalloc");
  e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? FFC_OK : cuda_fail(e, "cudaMemcpy");
}
}  // namespace

uint32_t* status_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> g(g_status_lock);
  if (!g_status[dev]) {
    uint32_t* p = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&p), sizeof(uint32_t)) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, sizeof(uint32_t)) != cudaSuccess) return nullptr;
    g_status[dev] = p;
  }
  return g_status[dev];
}

int launch_config(const void* kernel, int threads, size_t dyn_smem, int carveout, int* sms, int* blocks_per_sm) {
  struct Key {
    const void* k;
    int dev, threads, carveout;
    size_t smem;
    bool operator<(const Key& o) const {
      if (k != o.k) return k < o.k;
      if (dev != o.dev) return dev < o.dev;
      if (threads != o.threads) return threads < o.threads;
      if (carveout != o.carveout) return carveout < o.carveout;
      return smem < o.smem;
    }
  };
  static std::mutex lock;
  static std::map<Key, std::pair<int, int>> cache;
  // the dynamic shared-memory limit is a property of the kernel on a device: only raised,
  // never lowered, so every launch shape cached before stays valid
  static std::map<std::pair<const void*, int>, size_t> smem_limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  const Key key{kernel, dev, threads, carveout, dyn_smem};
  std::lock_guard<std::mutex> g(lock);
  auto it = cache.find(key);
  if (it == cache.end()) {
    int n_sm = 0, per_sm = 0;
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return cuda_fail(e, "cudaDeviceGetAttribute");
    size_t& limit = smem_limit[std::make_pair(kernel, dev)];
    if (dyn_smem > 48 * 1024 && dyn_smem > limit) {
      if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn_smem))) != cudaSuccess)
        return cuda_fail(e, "cudaFuncSetAttribute");
      limit = dyn_smem;
    }
    if (carveout >= 0 &&
        (e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, carveout)) != cudaSuccess)
      return cuda_fail(e, "cudaFuncSetAttribute");
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, dyn_smem)) != cudaSuccess)
      return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    it = cache.emplace(key, std::make_pair(n_sm, per_sm > 0 ? per_sm : 1)).first;
  }
  if (sms) *sms = it->second.first;
  if (blocks_per_sm) *blocks_per_sm = it->second.second;
  return FFC_OK;
}

int ensure_device_tensors(ffc_form* f, DeviceTensors** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> g(f->lock);
  auto it = f->dev.find(dev);
  if (it != f->dev.end()) {
    *out = &it->second;
    return FFC_OK;
  }
  const size_t nn = f->n_entries(), na = size_t(f->kernel_na());
  std::vector<double> rows(f->kernel_a0()), cols(nn * na);
  for (size_t i = 0; i < nn; ++i)
    for (size_t a = 0; a < na; ++a) cols[a * nn + i] = rows[i * na + a];
  std::vector<float> rows32(rows.begin(), rows.end()), cols32(cols.begin(), cols.end());
  DeviceTensors t;
  int rc;
  if ((rc = upload(&t.a0_f64, rows)) || (rc = upload(&t.a0t_f64, cols)) || (rc = upload(&t.a0_f32, rows32)) ||
      (rc = upload(&t.a0t_f32, cols32))) {
    cudaFree(t.a0_f64);
    cudaFree(t.a0t_f64);
    cudaFree(t.a0_f32);
    cudaFree(t.a0t_f32);
    return rc;
  }
  if (!f->R.empty()) {
    std::vector<float> r32(f->R.begin(), f->R.end());
    if ((rc = upload(&t.r_f64, f->R)) || (rc = upload(&t.r_f32, r32))) {
      cudaFree(t.a0_f64);
      cudaFree(t.a0t_f64);
      cudaFree(t.a0_f32);
      cudaFree(t.a0t_f32);
      cudaFree(t.r_f64);
      cudaFree(t.r_f32);
      return rc;
    }
  }
  if (f->rank == 2) {
    const size_t n = size_t(f->n);
    std::vector<double> soa(nn * na);
    for (size_t i1 = 0; i1 < n; ++i1)
      for (size_t a = 0; a < na; ++a)
        for (size_t i2 = 0; i2 < n; ++i2) soa[(i1 * na + a) * n + i2] = rows[(i1 * n + i2) * na + a];
    std::vector<float> soa32(soa.begin(), soa.end());
    if ((rc = upload(&t.a0s_f64, soa)) || (rc = upload(&t.a0s_f32, soa32))) {
      cudaFree(t.a0_f64);
      cudaFree(t.a0t_f64);
      cudaFree(t.a0_f32);
      cudaFree(t.a0t_f32);
      cudaFree(t.r_f64);
      cudaFree(t.r_f32);
      cudaFree(t.a0s_f64);
      cudaFree(t.a0s_f32);
      return rc;
    }
  }
  auto res = f->dev.emplace(dev, t);
  *out = &res.first->second;
  return FFC_OK;
}

void release_device_tensors(ffc_form* f) {
  std::lock_guard<std::mutex> g(f->lock);
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto& kv : f->dev) {
    cudaSetDevice(kv.first);
    DeviceTensors& t = kv.second;
    cudaFree(t.a0_f64);
    cudaFree(t.a0t_f64);
    cudaFree(t.a0_f32);
    cudaFree(t.a0t_f32);
    for (auto& fam : t.tc_part)
      for (void* q : fam) cudaFree(q);
    cudaFree(t.r_f64);
    cudaFree(t.r_f32);
    cudaFree(t.a0s_f64);
    cudaFree(t.a0s_f32);
  }
  f->dev.clear();
  cudaSetDevice(cur);
}

static int dispatch(const LaunchArgs& a, int precision, bool assemble) {
  int rc = FFC_EUNSUPPORTED;
  if (precision == FFC_FP64 || precision == FFC_FP32) {
    if (a.f->kr > 0 && a.f->algorithm != FFC_ALG_DENSE) rc = launch_simt_block(a, precision, assemble);
    if (rc == FFC_EUNSUPPORTED) rc = launch_simt_tri(a, precision, assemble);
    if (rc == FFC_EUNSUPPORTED) rc = launch_simt_tet_mass(a, precision, assemble);
    if (rc == FFC_EUNSUPPORTED) rc = launch_simt_tet_poisson(a, precision, assemble);
    if (rc == FFC_EUNSUPPORTED) rc = launch_simt_vector(a, precision, assemble);
    if (rc == FFC_EUNSUPPORTED) rc = launch_simt_source(a, precision, assemble);
  } else if (precision == FFC_TF32 || precision == FFC_TF32X3 || precision == FFC_BF16X3) {
    rc = launch_tc(a, precision, assemble);
  }
  if (rc == FFC_ECUDA) set_error(std::string("kernel launch: ") + cudaGetErrorString(cudaGetLastError()));
  if (rc == FFC_EUNSUPPORTED) set_error("no kernel built for this form/precision");
  return rc;
}

static int common_checks(const ffc_form* f, int64_t n_elem, const int32_t* cells, const double* vertices,
                         int64_t n_vert, const double* coeffs, int precision) {
  if (!f || n_elem < 0 || n_vert < 0) return FFC_EINVAL;
  if (precision < FFC_FP64 || precision > FFC_BF16X3) return FFC_EINVAL;
  if (n_elem == 0) return FFC_OK;
  if (!cells || !vertices || n_vert == 0) return FFC_EINVAL;
  if (f->ncoeff > 0 && !coeffs) return FFC_EINVAL;
  if ((reinterpret_cast<uintptr_t>(cells) & 15) || (reinterpret_cast<uintptr_t>(vertices) & 7)) return FFC_EINVAL;
  return FFC_OK;
}

}  // namespace ffc

using namespace ffc;

extern "C" {

int ffc_tabulate(const ffc_form* f, int64_t n_elem, const int32_t* cells, const double* vertices, int64_t n_vert,
                 const double* coeffs, void* A_K, int precision, void* stream) {
  int rc = common_checks(f, n_elem, cells, vertices, n_vert, coeffs, precision);
  if (rc != FFC_OK) { set_error("ffc_tabulate: invalid argument"); return rc; }
  if (n_elem == 0) return FFC_OK;
  if (!A_K || (reinterpret_cast<uintptr_t>(A_K) & 15)) { set_error("ffc_tabulate: A_K"); return FFC_EINVAL; }
  DeviceTensors* t = nullptr;
  if ((rc = ensure_device_tensors(const_cast<ffc_form*>(f), &t)) != FFC_OK) return rc;
  uint32_t* st = status_word();
  if (!st) { set_error("status word allocation failed"); return FFC_ECUDA; }
  LaunchArgs a{f, n_elem, cells, vertices, n_vert, coeffs, A_K, nullptr, nullptr, 0, t, st, stream};
  return dispatch(a, precision, false);
}

int ffc_assemble(const ffc_form* f, int64_t n_elem, const int32_t* cells, const double* vertices, int64_t n_vert,
                 const double* coeffs, const int32_t* slot, double* csr_val, int64_t nnz, int precision,
                 void* stream) {
  int rc = common_checks(f, n_elem, cells, vertices, n_vert, coeffs, precision);
  if (rc != FFC_OK) { set_error("ffc_assemble: invalid argument"); return rc; }
  if (n_elem == 0) return FFC_OK;
  if (!slot || !csr_val || nnz <= 0 || nnz > INT32_MAX) { set_error("ffc_assemble: slot/csr"); return FFC_EINVAL; }
  DeviceTensors* t = nullptr;
  if ((rc = ensure_device_tensors(const_cast<ffc_form*>(f), &t)) != FFC_OK) return rc;
  uint32_t* st = status_word();
  if (!st) { set_error("status word allocation failed"); return FFC_ECUDA; }
  LaunchArgs a{f, n_elem, cells, vertices, n_vert, coeffs, nullptr, slot, csr_val, nnz, t, st, stream};
  return dispatch(a, precision, true);
}

int ffc_assemble_pair(const ffc_form* fa, const ffc_form* fb, int64_t n_elem, const int32_t* cells,
                      const double* vertices, int64_t n_vert, const int32_t* slot, double* csr_val_a,
                      double* csr_val_b, int64_t nnz, int precision, void* stream) {
  if (!fa || !fb || fa->rank != 2 || fb->rank != 2 || fa->d != fb->d || fa->q != fb->q || fa->n != fb->n ||
      csr_val_a == csr_val_b) {
    set_error("ffc_assemble_pair: two bilinear forms on one space, two distinct matrices");
    return FFC_EINVAL;
  }
  if (fa->ncoeff > 0 || fb->ncoeff > 0) {
    set_error("ffc_assemble_pair: forms with coefficients are assembled with ffc_assemble");
    return FFC_EUNSUPPORTED;
  }
  int rc = common_checks(fa, n_elem, cells, vertices, n_vert, nullptr, precision);
  if (rc != FFC_OK) { set_error("ffc_assemble_pair: invalid argument"); return rc; }
  if (n_elem == 0) return FFC_OK;
  if (!slot || !csr_val_a || !csr_val_b || nnz <= 0 || nnz > INT32_MAX) {
    set_error("ffc_assemble_pair: slot/csr");
    return FFC_EINVAL;
  }
  const bool mp = fa->kind == FFC_MASS && fb->kind == FFC_POISSON;
  const bool pm = fa->kind == FFC_POISSON && fb->kind == FFC_MASS;
  if ((mp || pm) && precision == FFC_FP32) {
    DeviceTensors *ta = nullptr, *tb = nullptr;
    if ((rc = ensure_device_tensors(const_cast<ffc_form*>(fa), &ta)) != FFC_OK ||
        (rc = ensure_device_tensors(const_cast<ffc_form*>(fb), &tb)) != FFC_OK)
      return rc;
    uint32_t* st = status_word();
    if (!st) { set_error("status word allocation failed"); return FFC_ECUDA; }
    LaunchArgs a{fa, n_elem, cells, vertices, n_vert, nullptr, nullptr, slot, nullptr, nnz, ta, st, stream};
    rc = mp ? launch_simt_pair(a, ta, tb, csr_val_a, csr_val_b) : launch_simt_pair(a, tb, ta, csr_val_b, csr_val_a);
    if (rc == FFC_ECUDA) set_error(std::string("kernel launch: ") + cudaGetErrorString(cudaGetLastError()));
    return rc;
  }
  // any other pair: the two assemblies one after the other
  if ((rc = ffc_assemble(fa, n_elem, cells, vertices, n_vert, nullptr, slot, csr_val_a, nnz, precision, stream)))
    return rc;
  return ffc_assemble(fb, n_elem, cells, vertices, n_vert, nullptr, slot, csr_val_b, nnz, precision, stream);
}

int ffc_scatter_add(int64_t n_elem, int n_entries, const void* A_K, int precision, const int32_t* slot,
                    double* csr_val, int64_t nnz, void* stream) {
  if (n_elem < 0 || n_entries <= 0 || (precision != FFC_FP64 && precision != FFC_FP32) || nnz < 0 ||
      nnz > INT32_MAX) {
    set_error("ffc_scatter_add: invalid argument");
    return FFC_EINVAL;
  }
  if (n_elem == 0) return FFC_OK;
  if (!A_K || !slot || !csr_val || nnz == 0) {
    set_error("ffc_scatter_add: null pointer or empty CSR");
    return FFC_EINVAL;
  }
  const size_t esize = precision == FFC_FP64 ? 8 : 4;
  if ((reinterpret_cast<uintptr_t>(A_K) % esize) || (reinterpret_cast<uintptr_t>(slot) % 4) ||
      (reinterpret_cast<uintptr_t>(csr_val) % 8)) {
    set_error("ffc_scatter_add: misaligned pointer");
    return FFC_EINVAL;
  }
  uint32_t* st = status_word();
  if (!st) { set_error("status word allocation failed"); return FFC_ECUDA; }
  return launch_scatter_add(A_K, precision, slot, csr_val, nnz, n_elem * (long long)n_entries, st, stream);
}

int ffc_tabulate_adjoint(const ffc_form* f, int64_t n_elem, const int32_t* cells, const double* vertices,
                         int64_t n_vert, const double* dA_K, double* dvertices, void* stream) {
  int rc = common_checks(f, n_elem, cells, vertices, n_vert, nullptr, FFC_FP64);
  if (rc != FFC_OK) { set_error("ffc_tabulate_adjoint: invalid argument"); return rc; }
  if (f->kind != FFC_POISSON) { set_error("adjoint: Poisson forms only"); return FFC_EUNSUPPORTED; }
  if (n_elem == 0) return FFC_OK;
  if (!dA_K || !dvertices) return FFC_EINVAL;
  DeviceTensors* t = nullptr;
  if ((rc = ensure_device_tensors(const_cast<ffc_form*>(f), &t)) != FFC_OK) return rc;
  uint32_t* st = status_word();
  if (!st) return FFC_ECUDA;
  LaunchArgs a{f, n_elem, cells, vertices, n_vert, nullptr, nullptr, nullptr, nullptr, 0, t, st, stream};
  return launch_adjoint(a, dA_K, dvertices);
}

int ffc_diag_bounded_wait(uint32_t polls, void* stream) {
  if (polls > (1u << 20)) {
    set_error("ffc_diag_bounded_wait: at most 2^20 polls");
    return FFC_EINVAL;
  }
  uint32_t* st = status_word();
  if (!st) { set_error("status word allocation failed"); return FFC_ECUDA; }
  return launch_bounded_wait_probe(polls, st, stream);
}

int ffc_status_poll(void* stream, uint32_t* flags) {
  if (!flags) return FFC_EINVAL;
  uint32_t* st = status_word();
  if (!st) return FFC_ECUDA;
  // read and clear in the order of `stream`, then wait for that stream only: work queued
  // on other streams keeps running (bits it sets later appear at the next poll)
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, st, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync status");
  e = cudaMemsetAsync(st, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync status");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  *flags = v;
  return FFC_OK;
}

}  // extern "C"
