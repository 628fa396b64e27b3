// Batched heterogeneous assembly: many (mesh, form, degree) problems in one
// persistent launch (Algorithm 2 of Section 2.2 with the tensor representation of
// Section 3.2, applied to a list of independent problems).
//
// The host flattens every problem into tiles of E cells (E depends on the form and
// on the tile variant) and uploads a work table sorted by first tile. Each CTA of
// the persistent kernel takes the next tile index from one global atomic counter
// (no CTA ever waits for another), finds its problem by binary search over the
// tables' first-tile indices, loads that form's reference-tensor rows and runs the
// shared CUDA-core tile body: FP64 geometry, FP32 contraction, FP64 atomic scatter
// (elasticity through the block-structured contraction, the other forms densely).
//
// The tile variant (256 threads per block, or 416 with registers bounded for one or two
// resident blocks; x 16, 32, 64 or 128 cells per thread group and tile) is chosen by
// timing all twelve on the caller's data (ffc_batch_tune). A run can be captured
// once into a CUDA graph (queue reset, optional CSR zeroing, kernel) and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <new>
#include <string>
#include <vector>

#include "ffc_internal.h"
#include "simt_block.cuh"
#include "simt_kernels.cuh"

namespace ffc {
namespace {

// Tile variants the autotuner times: block size x cells per thread group and tile x
// resident blocks per SM the registers are bounded for.
constexpr int N_VARIANTS = 12;
// 416 threads: 400 pairs of elasticity P3, 4 x 100 of elasticity P2 and Poisson P2;
// 416 x 2 resident blocks caps the registers at 72 (a few spills, twice the warps)
constexpr int VARIANT_BLOCK[N_VARIANTS] = {256, 256, 256, 256, 416, 416, 416, 416, 416, 416, 416, 416};
constexpr int VARIANT_KE[N_VARIANTS] = {16, 32, 64, 128, 16, 32, 64, 128, 16, 32, 64, 128};
constexpr int VARIANT_MINB[N_VARIANTS] = {2, 2, 2, 2, 1, 1, 1, 1, 2, 2, 2, 2};

// Forms the batched kernel carries, by code.
enum : int { CODE_ELAST_P1 = 0, CODE_ELAST_P2, CODE_ELAST_P3, CODE_POISSON_P1, CODE_POISSON_P2, CODE_MASS_P1,
             N_CODES };

template <int CODE>
struct CodeForm;
template <> struct CodeForm<CODE_ELAST_P1> { static constexpr int FORM = FFC_ELASTICITY, Q = 1; };
template <> struct CodeForm<CODE_ELAST_P2> { static constexpr int FORM = FFC_ELASTICITY, Q = 2; };
template <> struct CodeForm<CODE_ELAST_P3> { static constexpr int FORM = FFC_ELASTICITY, Q = 3; };
template <> struct CodeForm<CODE_POISSON_P1> { static constexpr int FORM = FFC_POISSON, Q = 1; };
template <> struct CodeForm<CODE_POISSON_P2> { static constexpr int FORM = FFC_POISSON, Q = 2; };
template <> struct CodeForm<CODE_MASS_P1> { static constexpr int FORM = FFC_MASS, Q = 1; };

template <int CODE, int BLK, int KE>
using CfgOf = SimtCfg<3, CodeForm<CODE>::FORM, CodeForm<CODE>::Q, float, BLK, KE>;
template <int CODE, int BLK, int KE>
using BlockCfgOf = BlockCfg<3, CodeForm<CODE>::FORM, CodeForm<CODE>::Q, float, BLK, KE>;
template <int CODE>
constexpr bool kBlock = CodeForm<CODE>::FORM == FFC_ELASTICITY;

struct WorkItem {
  int code;
  int pad;
  long long tile_begin;
  SimtParams p;
};

template <int CODE, int BLK, int KE>
__device__ __forceinline__ void run_tile(const SimtParams& p, long long tile, unsigned char* smem) {
  constexpr int FORM = CodeForm<CODE>::FORM, Q = CodeForm<CODE>::Q;
  if constexpr (kBlock<CODE>) {
    using C = BlockCfgOf<CODE, BLK, KE>;
    BlockRows<C, float> rows;
    block_rows_init<C, 3, FORM, float>(p.a0, rows, smem);
    block_tile<C, 3, FORM, Q, float, true>(p, tile, smem, rows);
  } else {
    using C = CfgOf<CODE, BLK, KE>;
    float a0r[C::REG_A0 ? C::R : 1][C::REG_A0 ? C::NA : 1];
    load_a0_rows<C, float>(p.a0, threadIdx.x, a0r);
    simt_tile<C, 3, FORM, Q, float, true>(p, tile, smem, a0r);
  }
}

template <int BLK, int KE, int MINB>
__global__ void __launch_bounds__(BLK, MINB)
    batch_assemble_kernel(const WorkItem* __restrict__ items, int n_items, long long total_tiles,
                          unsigned long long* queue) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(queue, 1ull);
    __syncthreads();
    const long long tile = s_tile;
    __syncthreads();
    if (tile >= total_tiles) break;
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].tile_begin <= tile) lo = mid;
      else hi = mid - 1;
    }
    const WorkItem& w = items[lo];
    const SimtParams p = w.p;
    const long long local = tile - w.tile_begin;
    switch (w.code) {
      case CODE_ELAST_P1: run_tile<CODE_ELAST_P1, BLK, KE>(p, local, smem); break;
      case CODE_ELAST_P2: run_tile<CODE_ELAST_P2, BLK, KE>(p, local, smem); break;
      case CODE_ELAST_P3: run_tile<CODE_ELAST_P3, BLK, KE>(p, local, smem); break;
      case CODE_POISSON_P1: run_tile<CODE_POISSON_P1, BLK, KE>(p, local, smem); break;
      case CODE_POISSON_P2: run_tile<CODE_POISSON_P2, BLK, KE>(p, local, smem); break;
      case CODE_MASS_P1: run_tile<CODE_MASS_P1, BLK, KE>(p, local, smem); break;
      default: break;
    }
  }
}

// Host view of the per-code configuration for a tile variant.
struct CodeInfo {
  int cells_per_tile;
  size_t smem;
  bool reg_a0;
  bool block;  // reads the reduced reference tensor
};

template <int CODE, int BLK, int KE>
CodeInfo info_of() {
  if constexpr (kBlock<CODE>) {
    using C = BlockCfgOf<CODE, BLK, KE>;
    return {C::E, C::SMEM, false, true};
  } else {
    using C = CfgOf<CODE, BLK, KE>;
    return {C::E, C::SMEM, C::REG_A0, false};
  }
}

template <int V>
CodeInfo code_info(int code) {
  constexpr int BLK = VARIANT_BLOCK[V], KE = VARIANT_KE[V];
  switch (code) {
    case CODE_ELAST_P1: return info_of<CODE_ELAST_P1, BLK, KE>();
    case CODE_ELAST_P2: return info_of<CODE_ELAST_P2, BLK, KE>();
    case CODE_ELAST_P3: return info_of<CODE_ELAST_P3, BLK, KE>();
    case CODE_POISSON_P1: return info_of<CODE_POISSON_P1, BLK, KE>();
    case CODE_POISSON_P2: return info_of<CODE_POISSON_P2, BLK, KE>();
    default: return info_of<CODE_MASS_P1, BLK, KE>();
  }
}

CodeInfo code_info_variant(int variant, int code) {
  switch (variant) {
    case 0: return code_info<0>(code);
    case 1: return code_info<1>(code);
    case 2: return code_info<2>(code);
    case 3: return code_info<3>(code);
    case 4: return code_info<4>(code);
    case 5: return code_info<5>(code);
    case 6: return code_info<6>(code);
    case 7: return code_info<7>(code);
    case 8: return code_info<8>(code);
    case 9: return code_info<9>(code);
    case 10: return code_info<10>(code);
    default: return code_info<11>(code);
  }
}

int code_for(const ffc_form* f) {
  if (f->d != 3) return -1;
  if (f->kind == FFC_ELASTICITY && f->q >= 1 && f->q <= 3) return CODE_ELAST_P1 + (f->q - 1);
  if (f->kind == FFC_POISSON && f->q == 1) return CODE_POISSON_P1;
  if (f->kind == FFC_POISSON && f->q == 2) return CODE_POISSON_P2;
  if (f->kind == FFC_MASS && f->q == 1) return CODE_MASS_P1;
  return -1;
}

}  // namespace
}  // namespace ffc

struct ffc_batch {
  std::vector<ffc_batch_item> items;
  std::vector<int> codes;
  std::vector<ffc::DeviceTensors*> tensors;
  int zero_csr = 1;
  int variant = 1;
  int sms = 0;
  int grid[ffc::N_VARIANTS] = {};
  ffc::WorkItem* d_items[ffc::N_VARIANTS] = {};
  long long total_tiles[ffc::N_VARIANTS] = {};
  size_t smem[ffc::N_VARIANTS] = {};
  unsigned long long* d_queue = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_variant = -1;
  cudaStream_t capture = nullptr;  // private stream the graph is captured on
};

using namespace ffc;

namespace {

int build_table(ffc_batch* b, int variant) {
  std::vector<WorkItem> w(b->items.size());
  long long begin = 0;
  size_t smem = 0;
  uint32_t* status = status_word();
  if (!status) return FFC_ECUDA;
  for (size_t k = 0; k < b->items.size(); ++k) {
    const ffc_batch_item& it = b->items[k];
    const CodeInfo ci = code_info_variant(variant, b->codes[k]);
    WorkItem& x = w[k];
    x.code = b->codes[k];
    x.tile_begin = begin;
    SimtParams& p = x.p;
    p = SimtParams{};
    p.cells = it.cells;
    p.vertices = it.vertices;
    p.n_vert = it.n_vert;
    p.coeffs = it.coeffs;
    p.a0 = ci.block ? (const void*)b->tensors[k]->r_f32
                    : ci.reg_a0 ? (const void*)b->tensors[k]->a0_f32 : (const void*)b->tensors[k]->a0t_f32;
    p.out = nullptr;
    p.slot = it.slot;
    p.csr_val = it.csr_val;
    p.nnz = it.nnz;
    p.n_elem = it.n_elem;
    p.mu = it.form->mu;
    p.lambda = it.form->lambda;
    p.status = status;
    begin += (it.n_elem + ci.cells_per_tile - 1) / ci.cells_per_tile;
    smem = std::max(smem, ci.smem);
  }
  cudaFree(b->d_items[variant]);
  b->d_items[variant] = nullptr;
  if (cudaMalloc(&b->d_items[variant], w.size() * sizeof(WorkItem)) != cudaSuccess) return FFC_ENOMEM;
  if (cudaMemcpy(b->d_items[variant], w.data(), w.size() * sizeof(WorkItem), cudaMemcpyHostToDevice) != cudaSuccess)
    return FFC_ECUDA;
  b->total_tiles[variant] = begin;
  b->smem[variant] = smem;
  return FFC_OK;
}

template <int V>
int launch_variant(ffc_batch* b, cudaStream_t s) {
  constexpr int variant = V, BLK = VARIANT_BLOCK[V], KE = VARIANT_KE[V], MINB = VARIANT_MINB[V];
  auto kern = batch_assemble_kernel<BLK, KE, MINB>;
  if (b->smem[variant] > 96 * 1024) return FFC_EUNSUPPORTED;
  int sms = 0, per_sm = 1;
  if (launch_config(reinterpret_cast<const void*>(kern), BLK, b->smem[variant], -1, &sms, &per_sm) != FFC_OK)
    return FFC_ECUDA;
  b->grid[variant] = sms * std::max(1, per_sm);
  kern<<<b->grid[variant], BLK, b->smem[variant], s>>>(b->d_items[variant], int(b->items.size()),
                                                                  b->total_tiles[variant], b->d_queue);
  const cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) set_error(std::string("batch kernel launch: ") + cudaGetErrorString(e));
  return e == cudaSuccess ? FFC_OK : FFC_ECUDA;
}

int enqueue(ffc_batch* b, int variant, cudaStream_t s) {
  if (b->zero_csr)
    for (const auto& it : b->items)
      if (cudaMemsetAsync(it.csr_val, 0, size_t(it.nnz) * sizeof(double), s) != cudaSuccess) return FFC_ECUDA;
  if (cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), s) != cudaSuccess) return FFC_ECUDA;
  switch (variant) {
    case 0: return launch_variant<0>(b, s);
    case 1: return launch_variant<1>(b, s);
    case 2: return launch_variant<2>(b, s);
    case 3: return launch_variant<3>(b, s);
    case 4: return launch_variant<4>(b, s);
    case 5: return launch_variant<5>(b, s);
    case 6: return launch_variant<6>(b, s);
    case 7: return launch_variant<7>(b, s);
    case 8: return launch_variant<8>(b, s);
    case 9: return launch_variant<9>(b, s);
    case 10: return launch_variant<10>(b, s);
    default: return launch_variant<11>(b, s);
  }
}

void drop_graph(ffc_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_variant = -1;
}

}  // namespace

extern "C" {

int ffc_batch_create(const ffc_batch_item* items, int n_items, int zero_csr, ffc_batch** out) {
  if (!out || !items || n_items <= 0) return FFC_EINVAL;
  *out = nullptr;
  ffc_batch* b = new (std::nothrow) ffc_batch();
  if (!b) return FFC_ENOMEM;
  b->zero_csr = zero_csr ? 1 : 0;
  for (int k = 0; k < n_items; ++k) {
    const ffc_batch_item& it = items[k];
    const int code = it.form ? code_for(it.form) : -1;
    if (code < 0) {
      set_error("ffc_batch_create: item " + std::to_string(k) + " has a form the batched kernel does not carry");
      delete b;
      return it.form ? FFC_EUNSUPPORTED : FFC_EINVAL;
    }
    if (it.n_elem <= 0 || !it.cells || !it.vertices || it.n_vert <= 0 || !it.slot || !it.csr_val || it.nnz <= 0 ||
        it.nnz > INT32_MAX || (reinterpret_cast<uintptr_t>(it.cells) & 15)) {
      set_error("ffc_batch_create: item " + std::to_string(k) + " has an invalid pointer or size");
      delete b;
      return FFC_EINVAL;
    }
    DeviceTensors* t = nullptr;
    int rc = ensure_device_tensors(const_cast<ffc_form*>(it.form), &t);
    if (rc != FFC_OK) {
      delete b;
      return rc;
    }
    b->items.push_back(it);
    b->codes.push_back(code);
    b->tensors.push_back(t);
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMalloc(&b->d_queue, sizeof(unsigned long long)) != cudaSuccess) {
    delete b;
    return FFC_ENOMEM;
  }
  for (int v = 0; v < N_VARIANTS; ++v) {
    int rc = build_table(b, v);
    if (rc != FFC_OK) {
      ffc_batch_destroy(b);
      return rc;
    }
  }
  *out = b;
  return FFC_OK;
}

int ffc_batch_tune(ffc_batch* b, void* stream, int* cells_per_tile_group, int* threads_per_block) {
  if (!b) return FFC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return FFC_ECUDA;
  float best = 1e30f;
  int best_v = b->variant;
  for (int v = 0; v < N_VARIANTS; ++v) {
    int rc = enqueue(b, v, s);  // warm-up
    if (rc != FFC_OK) continue;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3 && rc == FFC_OK; ++r) rc = enqueue(b, v, s);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = FFC_ECUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rc == FFC_OK && ms < best) {
      best = ms;
      best_v = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_v != b->variant) drop_graph(b);
  b->variant = best_v;
  // leave the matrices zeroed: tuning accumulated into them
  for (const auto& it : b->items)
    if (cudaMemsetAsync(it.csr_val, 0, size_t(it.nnz) * sizeof(double), s) != cudaSuccess) return FFC_ECUDA;
  if (cells_per_tile_group) *cells_per_tile_group = VARIANT_KE[b->variant];
  if (threads_per_block) *threads_per_block = VARIANT_BLOCK[b->variant];
  return cudaStreamSynchronize(s) == cudaSuccess ? FFC_OK : FFC_ECUDA;
}

int ffc_batch_run(ffc_batch* b, int use_graph, void* stream) {
  if (!b) return FFC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!use_graph) return enqueue(b, b->variant, s);
  if (!b->graph || b->graph_variant != b->variant) {
    // capture on the batch's own stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph then runs on the caller's stream
    drop_graph(b);
    if (!b->capture && cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess)
      return FFC_ECUDA;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      set_error(std::string("ffc_batch_run: begin capture: ") + cudaGetErrorString(e));
      cudaGetLastError();
      return FFC_ECUDA;
    }
    int rc = enqueue(b, b->variant, b->capture);
    e = cudaStreamEndCapture(b->capture, &g);
    if (rc != FFC_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      set_error(std::string("ffc_batch_run: capture: ") + cudaGetErrorString(e));
      cudaGetLastError();
      return FFC_ECUDA;
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      set_error(std::string("ffc_batch_run: instantiate: ") + cudaGetErrorString(e));
      cudaGetLastError();
      return FFC_ECUDA;
    }
    b->graph_variant = b->variant;
  }
  cudaError_t e = cudaGraphLaunch(b->graph, s);
  if (e != cudaSuccess) set_error(std::string("ffc_batch_run: graph launch: ") + cudaGetErrorString(e));
  return e == cudaSuccess ? FFC_OK : FFC_ECUDA;
}

int ffc_batch_info(const ffc_batch* b, int* n_items, long long* total_tiles, int* cells_per_tile_group,
                   int* threads_per_block) {
  if (!b) return FFC_EINVAL;
  if (n_items) *n_items = int(b->items.size());
  if (total_tiles) *total_tiles = b->total_tiles[b->variant];
  if (cells_per_tile_group) *cells_per_tile_group = VARIANT_KE[b->variant];
  if (threads_per_block) *threads_per_block = VARIANT_BLOCK[b->variant];
  return FFC_OK;
}

void ffc_batch_destroy(ffc_batch* b) {
  if (!b) return;
  drop_graph(b);
  if (b->capture) cudaStreamDestroy(b->capture);
  for (auto& d : b->d_items) cudaFree(d);
  cudaFree(b->d_queue);
  delete b;
}

}  // extern "C"
