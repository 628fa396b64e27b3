// Host-only entry points of the C ABI: form handles, the CSR pattern builder,
// status strings. Device entry points live in device_api.cu.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstring>
#include <new>
#include <sched.h>
#include <string>
#include <thread>
#include <vector>

#include "ffc_internal.h"

namespace ffc {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

static int host_threads() {
  cpu_set_t set;
  if (sched_getaffinity(0, sizeof(set), &set) == 0) {
    int c = CPU_COUNT(&set);
    if (c > 0) return c;
  }
  unsigned h = std::thread::hardware_concurrency();
  return h ? int(h) : 1;
}

template <typename F>
static void parallel_for(int64_t n, F&& fn) {
  int nt = int(std::min<int64_t>(host_threads(), std::max<int64_t>(1, n / 1024)));
  if (nt <= 1) {
    fn(int64_t(0), n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    int64_t lo = t * chunk, hi = std::min(n, lo + chunk);
    if (lo >= hi) break;
    th.emplace_back([&, lo, hi] { fn(lo, hi); });
  }
  for (auto& x : th) x.join();
}

}  // namespace ffc

using namespace ffc;

extern "C" {

const char* ffc_last_error(void) { return g_last_error.c_str(); }

const char* ffc_status_string(int s) {
  switch (s) {
    case FFC_OK: return "FFC_OK";
    case FFC_EINVAL: return "FFC_EINVAL: invalid argument";
    case FFC_ENOMEM: return "FFC_ENOMEM: allocation failed";
    case FFC_ECUDA: return "FFC_ECUDA: CUDA runtime error";
    case FFC_EDEGENERATE: return "FFC_EDEGENERATE: degenerate cell";
    case FFC_EUNSUPPORTED: return "FFC_EUNSUPPORTED: combination not built";
    case FFC_EBOUNDS: return "FFC_EBOUNDS: index out of range";
    case FFC_ETIMEOUT: return "FFC_ETIMEOUT: bounded wait expired";
    default: return "unknown ffc status";
  }
}

int ffc_form_create(int form, int cell, int degree, double mu, double lambda, ffc_form** out) {
  if (!out) return FFC_EINVAL;
  *out = nullptr;
  if (form < FFC_MASS || form > FFC_SOURCE) { set_error("unknown form"); return FFC_EINVAL; }
  if (cell != FFC_TRIANGLE && cell != FFC_TETRAHEDRON) { set_error("unknown cell"); return FFC_EINVAL; }
  if (degree < 1 || degree > 4) { set_error("degree must be 1..4"); return FFC_EINVAL; }
  if (form == FFC_NS_CONVECTION && (cell != FFC_TETRAHEDRON || degree > 2)) {
    set_error("convection: tetrahedra, degree 1..2");
    return FFC_EUNSUPPORTED;
  }
  if (form == FFC_ELASTICITY && (cell != FFC_TETRAHEDRON || degree > 3)) {
    set_error("elasticity: tetrahedra, degree 1..3");
    return FFC_EUNSUPPORTED;
  }
  ffc_form* f = new (std::nothrow) ffc_form();
  if (!f) return FFC_ENOMEM;
  f->kind = form;
  f->d = cell;
  f->q = degree;
  f->ns = n_scalar_local(f->d, f->q);
  bool vec = (form == FFC_NS_CONVECTION || form == FFC_ELASTICITY);
  f->n = vec ? f->d * f->ns : f->ns;
  switch (form) {
    case FFC_MASS: f->na = 1; break;
    case FFC_POISSON: f->na = f->d * f->d; break;
    case FFC_NS_CONVECTION: f->na = f->n * f->d; break;
    case FFC_ELASTICITY: f->na = f->d * f->d * f->d * f->d; break;
    case FFC_SOURCE: f->na = f->n; break;
  }
  f->ncoeff = (form == FFC_NS_CONVECTION || form == FFC_SOURCE) ? f->n : 0;
  f->rank = (form == FFC_SOURCE) ? 1 : 2;
  f->mu = mu;
  f->lambda = lambda;
  int rc;
  try {
    rc = compile_reference_tensor(f);
  } catch (const std::bad_alloc&) {
    rc = FFC_ENOMEM;
  }
  if (rc != FFC_OK) {
    delete f;
    return rc;
  }
  *out = f;
  return FFC_OK;
}

int ffc_form_info(const ffc_form* f, int* n_local, int* n_alpha, int* n_coeff) {
  if (!f) return FFC_EINVAL;
  if (n_local) *n_local = f->n;
  if (n_alpha) *n_alpha = f->na;
  if (n_coeff) *n_coeff = f->ncoeff;
  return FFC_OK;
}

int ffc_form_rank(const ffc_form* f, int* rank) {
  if (!f || !rank) return FFC_EINVAL;
  *rank = f->rank;
  return FFC_OK;
}

int ffc_form_reference_tensor(const ffc_form* f, double* host_out) {
  if (!f || !host_out) return FFC_EINVAL;
  std::memcpy(host_out, f->A0.data(), f->A0.size() * sizeof(double));
  return FFC_OK;
}

int ffc_form_set_algorithm(ffc_form* f, int algorithm) {
  if (!f || algorithm < FFC_ALG_AUTO || algorithm > FFC_ALG_BLOCK) return FFC_EINVAL;
  f->algorithm = algorithm;
  return FFC_OK;
}

void ffc_form_destroy(ffc_form* f) {
  if (!f) return;
  release_device_tensors(f);
  delete f;
}

int ffc_csr_pattern(int64_t n_elem, int n_local, const int32_t* dofmap, int64_t n_dof, int64_t* row_ptr,
                    int64_t* nnz, int32_t* col, int64_t col_capacity, int32_t* slot) {
  if (n_elem < 0 || n_local <= 0 || n_dof <= 0 || !row_ptr || !nnz || (n_elem > 0 && !dofmap)) {
    set_error("ffc_csr_pattern: bad arguments");
    return FFC_EINVAL;
  }
  if (n_dof > INT32_MAX) { set_error("n_dof exceeds int32"); return FFC_EINVAL; }
  const int n = n_local;
  // range check
  std::atomic<bool> bad{false};
  parallel_for(n_elem * n, [&](int64_t lo, int64_t hi) {
    for (int64_t k = lo; k < hi; ++k)
      if (dofmap[k] < 0 || dofmap[k] >= n_dof) { bad = true; return; }
  });
  if (bad) { set_error("dof id out of range"); return FFC_EBOUNDS; }
  try {
    // dof -> cells adjacency
    std::vector<int64_t> adj_ptr(n_dof + 1, 0);
    for (int64_t k = 0; k < n_elem * n; ++k) adj_ptr[dofmap[k] + 1]++;
    for (int64_t r = 0; r < n_dof; ++r) adj_ptr[r + 1] += adj_ptr[r];
    std::vector<int64_t> adj(adj_ptr[n_dof]);
    {
      std::vector<int64_t> fill(adj_ptr.begin(), adj_ptr.end() - 1);
      for (int64_t e = 0; e < n_elem; ++e)
        for (int i = 0; i < n; ++i) adj[fill[dofmap[e * n + i]]++] = e;
    }
    // per-row sorted unique columns (count pass, then fill pass)
    auto row_cols = [&](int64_t r, std::vector<int32_t>& buf) {
      buf.clear();
      for (int64_t k = adj_ptr[r]; k < adj_ptr[r + 1]; ++k) {
        const int32_t* dm = dofmap + adj[k] * n;
        buf.insert(buf.end(), dm, dm + n);
      }
      std::sort(buf.begin(), buf.end());
      buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
    };
    row_ptr[0] = 0;
    parallel_for(n_dof, [&](int64_t lo, int64_t hi) {
      std::vector<int32_t> buf;
      for (int64_t r = lo; r < hi; ++r) {
        row_cols(r, buf);
        row_ptr[r + 1] = int64_t(buf.size());
      }
    });
    for (int64_t r = 0; r < n_dof; ++r) row_ptr[r + 1] += row_ptr[r];
    *nnz = row_ptr[n_dof];
    if (!col || col_capacity < *nnz) return FFC_OK;
    if (slot && *nnz > INT32_MAX) { set_error("nnz exceeds int32 slots"); return FFC_EINVAL; }
    parallel_for(n_dof, [&](int64_t lo, int64_t hi) {
      std::vector<int32_t> buf;
      for (int64_t r = lo; r < hi; ++r) {
        row_cols(r, buf);
        std::copy(buf.begin(), buf.end(), col + row_ptr[r]);
      }
    });
    if (slot) {
      parallel_for(n_elem, [&](int64_t lo, int64_t hi) {
        for (int64_t e = lo; e < hi; ++e) {
          const int32_t* dm = dofmap + e * n;
          for (int i1 = 0; i1 < n; ++i1) {
            const int32_t* b = col + row_ptr[dm[i1]];
            const int32_t* en = col + row_ptr[dm[i1] + 1];
            for (int i2 = 0; i2 < n; ++i2) {
              const int32_t* p = std::lower_bound(b, en, dm[i2]);
              slot[(e * n + i1) * n + i2] = int32_t(p - col);
            }
          }
        }
      });
    }
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed in ffc_csr_pattern");
    return FFC_ENOMEM;
  }
  return FFC_OK;
}

}  // extern "C"
