// CUDA-core kernel of the linear source form L(v) = int v f dx (Section 2.1), whose
// tensor representation is rank 1 (Section 3.2): b^K_i = A0[i][t] G_K[t] with
// A0[i][t] = int_{K0} Psi_i Psi_t and G_K[t] = |det J| f_t, evaluated here as
// b^K_i = |det J| * sum_t A0[i][t] f_t. With ASSEMBLE the element vector is added into
// the global vector through the dof map (Section 2.2, Algorithm 2 for a vector).
//
// A CTA takes tiles of TC consecutive cells (persistent grid-stride loop):
//   load      the tile's f values are one contiguous block of TC*n doubles: coalesced
//             loads into shared memory as T, rows padded to NP for 16-byte vector reads;
//   geometry  one thread per cell computes |det J| in FP64 (no J^{-1}: the form needs
//             none, which on GB300's narrow FP64 pipe is most of the geometry cost);
//   contract  thread t < G*n owns the local index i = t mod n, with A0 row i in
//             registers, and the cells c = t div n + k*G: at step k the G thread groups
//             cover G consecutive cells, so a warp's stores (or dof-map loads) touch
//             consecutive addresses. The dof of the next cell is loaded while this
//             cell's atomic add issues.
#include <cuda_runtime.h>

#include <type_traits>

#include "ffc_internal.h"
#include "geometry.cuh"

namespace ffc {
namespace {

struct SourceParams {
  const int32_t* cells;
  const double* vertices;
  long long n_vert;
  const double* f;         // [n_elem][n] f on each cell
  const void* a0;          // [n][n] reference tensor rows, in T
  void* out;               // [n_elem][n] element vectors (tabulate)
  const int32_t* dofmap;   // [n_elem][n] (assemble)
  double* b;               // [n_dof] global vector (assemble)
  long long n_dof;
  long long n_elem;
  unsigned* status;
};

template <int D, int Q, typename T>
struct SourceCfg {
  static constexpr int N = nscalar(D, Q);
  static constexpr int NT = 256;
  static constexpr int G = NT / N;                         // cells contracted side by side
  static constexpr int TC = sizeof(T) == 4 ? 256 : 128;    // cells per tile
  static constexpr int VEC = 16 / int(sizeof(T));
  static constexpr int NP = (N + VEC - 1) / VEC * VEC;     // padded row of f in shared memory
  static constexpr size_t SMEM = size_t(TC) * NP * sizeof(T) + size_t(TC) * sizeof(T);
};

// four resident CTAs per SM for FP32 (64 registers), two for FP64
template <int D, int Q, typename T, bool ASSEMBLE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) source_kernel(SourceParams p) {
  using C = SourceCfg<D, Q, T>;
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int N = C::N, NP = C::NP, TC = C::TC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* fs = reinterpret_cast<T*>(smem_raw);  // [TC][NP]
  T* ds = fs + TC * NP;                    // [TC]
  const int t = threadIdx.x;
  const int i = t % N;
  const int g = t / N;
  const bool active = g < C::G;
  T a0r[N];
  {
    const T* A0 = static_cast<const T*>(p.a0);
#pragma unroll
    for (int s = 0; s < N; ++s) a0r[s] = active ? A0[i * N + s] : T(0);
  }
  // the padding columns are never written by the tile loader: zero them once
  if constexpr (NP > N) {
    for (int k = t; k < TC * (NP - N); k += C::NT) fs[(k / (NP - N)) * NP + N + k % (NP - N)] = T(0);
  }
  const long long n_tiles = (p.n_elem + TC - 1) / TC;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long long e0 = tile * TC;
    const int nc = int(p.n_elem - e0 < TC ? p.n_elem - e0 : TC);
    const double* src = p.f + e0 * N;
    for (int k = t; k < nc * N; k += C::NT) {
      const int c = k / N;
      fs[c * NP + (k - c * N)] = T(__ldg(src + k));
    }
    for (int c = t; c < nc; c += C::NT) {
      double det;
      bool degenerate, bad_index;
      cell_det<D>(p.cells, p.vertices, p.n_vert, e0 + c, det, degenerate, bad_index);
      if (degenerate) atomicOr(p.status, FFC_FLAG_DEGENERATE);
      if (bad_index) atomicOr(p.status, FFC_FLAG_BOUNDS);
      ds[c] = T(det);
    }
    __syncthreads();
    if (active) {
      int dof_next = -1;
      if constexpr (ASSEMBLE) dof_next = (g < nc) ? __ldg(p.dofmap + (e0 + g) * N + i) : -1;
#pragma unroll 1
      for (int c = g; c < nc; c += C::G) {
        int dof = -1;
        if constexpr (ASSEMBLE) {
          dof = dof_next;
          const int cn = c + C::G;
          dof_next = (cn < nc) ? __ldg(p.dofmap + (e0 + cn) * N + i) : -1;
        }
        const T* fr = fs + c * NP;
        T acc = T(0);
#pragma unroll
        for (int s0 = 0; s0 < NP; s0 += C::VEC) {
          const V v = *reinterpret_cast<const V*>(fr + s0);
          if constexpr (sizeof(T) == 4) {
            if (s0 + 0 < N) acc = fma(v.x, a0r[s0 + 0 < N ? s0 + 0 : 0], acc);
            if (s0 + 1 < N) acc = fma(v.y, a0r[s0 + 1 < N ? s0 + 1 : 0], acc);
            if (s0 + 2 < N) acc = fma(v.z, a0r[s0 + 2 < N ? s0 + 2 : 0], acc);
            if (s0 + 3 < N) acc = fma(v.w, a0r[s0 + 3 < N ? s0 + 3 : 0], acc);
          } else {
            if (s0 + 0 < N) acc = fma(v.x, a0r[s0 + 0 < N ? s0 + 0 : 0], acc);
            if (s0 + 1 < N) acc = fma(v.y, a0r[s0 + 1 < N ? s0 + 1 : 0], acc);
          }
        }
        const T val = acc * ds[c];
        if constexpr (ASSEMBLE) {
          if (dof >= 0 && dof < p.n_dof) atomicAdd(p.b + dof, double(val));
          else atomicOr(p.status, FFC_FLAG_BOUNDS);
        } else {
          __stcs(static_cast<T*>(p.out) + (e0 + c) * N + i, val);
        }
      }
    }
    __syncthreads();
  }
}

template <int D, int Q, typename T, bool ASSEMBLE>
int launch_source_one(const SourceParams& p, cudaStream_t stream) {
  using C = SourceCfg<D, Q, T>;
  auto kern = source_kernel<D, Q, T, ASSEMBLE>;
  int sms = 0, blocks_per_sm = 1;
  if (launch_config(reinterpret_cast<const void*>(kern), C::NT, C::SMEM, -1, &sms, &blocks_per_sm) != FFC_OK)
    return FFC_ECUDA;
  const long long n_tiles = (p.n_elem + C::TC - 1) / C::TC;
  long long grid = (long long)sms * blocks_per_sm;
  if (grid > n_tiles) grid = n_tiles;
  if (grid < 1) grid = 1;
  kern<<<unsigned(grid), C::NT, C::SMEM, stream>>>(p);
  return cudaPeekAtLastError() == cudaSuccess ? FFC_OK : FFC_ECUDA;
}

template <int D, int Q, typename T>
int source_run(const LaunchArgs& a, bool assemble) {
  SourceParams p{};
  p.cells = a.cells;
  p.vertices = a.vertices;
  p.n_vert = a.n_vert;
  p.f = a.coeffs;
  p.a0 = std::is_same<T, double>::value ? (const void*)a.t->a0_f64 : (const void*)a.t->a0_f32;
  p.out = a.out;
  p.dofmap = a.slot;
  p.b = a.csr_val;
  p.n_dof = a.nnz;
  p.n_elem = a.n_elem;
  p.status = a.status;
  cudaStream_t s = static_cast<cudaStream_t>(a.stream);
  return assemble ? launch_source_one<D, Q, T, true>(p, s) : launch_source_one<D, Q, T, false>(p, s);
}

template <int D, typename T>
int source_by_degree(const LaunchArgs& a, bool assemble) {
  switch (a.f->q) {
    case 1: return source_run<D, 1, T>(a, assemble);
    case 2: return source_run<D, 2, T>(a, assemble);
    case 3: return source_run<D, 3, T>(a, assemble);
    case 4: return source_run<D, 4, T>(a, assemble);
  }
  return FFC_EUNSUPPORTED;
}

template <int D>
int source_by_precision(const LaunchArgs& a, int precision, bool assemble) {
  if (precision == FFC_FP64) return source_by_degree<D, double>(a, assemble);
  if (precision == FFC_FP32) return source_by_degree<D, float>(a, assemble);
  return FFC_EUNSUPPORTED;
}

}  // namespace

int launch_simt_source(const LaunchArgs& a, int precision, bool assemble) {
  if (a.f->kind != FFC_SOURCE) return FFC_EUNSUPPORTED;
  return a.f->d == 2 ? source_by_precision<2>(a, precision, assemble) : source_by_precision<3>(a, precision, assemble);
}

}  // namespace ffc
