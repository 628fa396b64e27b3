// Internal declarations shared by the host and device translation units of the
// library. Nothing here is part of the C ABI.
#pragma once

#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ffc_gb300.h"

namespace ffc {

// Device copies of a reference tensor, created lazily per device.
struct DeviceTensors {
  double* a0_f64 = nullptr;   // [nn][na]  row i holds A0[i][alpha]
  double* a0t_f64 = nullptr;  // [na][nn]  transposed (coalesced over i)
  float* a0_f32 = nullptr;    // [nn][na]
  float* a0t_f32 = nullptr;   // [na][nn]
  // bilinear forms: rows of A0 by i1, then alpha, then i2 ([n][na][n]; the row-owner kernels,
  // whose lanes take consecutive columns i2 of one row i1)
  double* a0s_f64 = nullptr;
  float* a0s_f32 = nullptr;
  // tcgen05 operands: A0 split into TF32 (family 0: 2 parts) or BF16 (family 1: 3 parts),
  // each part laid out per 128-entry M-tile in the core-matrix layout
  void* tc_part[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  int tc_kpad[2] = {0, 0};
  double* r_f64 = nullptr;    // reduced reference tensor [ns*ns][kr]
  float* r_f32 = nullptr;
};

}  // namespace ffc

struct ffc_form {
  int kind = 0;        // ffc_form_kind
  int d = 0;           // spatial dimension
  int q = 0;           // polynomial degree
  int ns = 0;          // scalar local dofs
  int n = 0;           // local dofs (ns or d*ns)
  int na = 0;          // |alpha|
  int ncoeff = 0;      // per-cell coefficients
  int rank = 2;        // 2: element matrix [n][n]; 1: element vector [n]
  double mu = 1.0, lambda = 1.25;
  std::vector<double> A0;  // [n*n][na]
  // the CUDA-core kernels' layout of A0 where it differs (the Poisson form: G_K is
  // symmetric, so A0 is stored once per pair a1 <= a2 with the (a1, a2) and (a2, a1)
  // columns summed, nak = d(d+1)/2); empty otherwise
  std::vector<double> A0k;
  int nak = 0;
  // Cartesian-product structure of the vector forms (Section 3.5): reduced reference
  // tensor R[ns*ns][kr] and nb geometry blocks per cell (0 when the form has none)
  std::vector<double> R;
  int kr = 0, nb = 0;
  int algorithm = 0;  // ffc_algorithm
  std::mutex lock;
  std::map<int, ffc::DeviceTensors> dev;
  // entries of one element tensor (rows of A0)
  size_t n_entries() const { return rank == 2 ? size_t(n) * n : size_t(n); }
  const std::vector<double>& kernel_a0() const { return A0k.empty() ? A0 : A0k; }
  int kernel_na() const { return A0k.empty() ? na : nak; }
};

namespace ffc {

// Host form compiler (reference tensor by collapsed Gauss-Jacobi quadrature).
int compile_reference_tensor(ffc_form* f);
int n_scalar_local(int d, int q);
// The collapsed Gauss-Jacobi rule on the reference simplex exact for degree p (points
// X [N][d], weights summing to 1/d!), and the reference Lagrange P_q basis at points X:
// values psi [N][ns] and gradients dpsi [N][ns][d], in the local dof order.
void reference_rule(int d, int p, std::vector<double>& X, std::vector<double>& W);
void reference_basis(int d, int q, const std::vector<double>& X, std::vector<double>& psi, std::vector<double>& dpsi);
// column of the symmetric pair (a, b) in the Poisson kernel layout: diagonal pairs
// 0..d-1, then (0,1) [, (0,2), (1,2)]; the device code uses the same numbering
int sym_pair(int d, int a, int b);

// Error text for ffc_last_error.
void set_error(const std::string& msg);

// Device side (defined in .cu files).
int ensure_device_tensors(ffc_form* f, DeviceTensors** out);
void release_device_tensors(ffc_form* f);
uint32_t* status_word();  // library-owned device status word of the current device

// Launch shape of one kernel on the current device: the device's SM count and how many
// CTAs of `threads` threads with `dyn_smem` bytes of dynamic shared memory are resident
// per SM. The first call for a (kernel, device, threads, dyn_smem) tuple raises the
// kernel's dynamic shared-memory limit on that device when dyn_smem exceeds 48 KiB (and
// sets its shared-memory carveout when carveout >= 0); the answers are cached per device
// under a lock, so several host threads and several devices are served correctly.
// Returns FFC_OK or FFC_ECUDA (message via ffc_last_error).
int launch_config(const void* kernel, int threads, size_t dyn_smem, int carveout, int* sms, int* blocks_per_sm);

struct LaunchArgs {
  const ffc_form* f;
  int64_t n_elem;
  const int32_t* cells;
  const double* vertices;
  int64_t n_vert;
  const double* coeffs;
  void* out;              // A_K (tabulate)
  const int32_t* slot;    // assemble
  double* csr_val;        // assemble
  int64_t nnz;            // assemble
  const DeviceTensors* t;
  uint32_t* status;
  void* stream;
};

// Each returns FFC_EUNSUPPORTED when it has no instantiation for the form.
int launch_simt_tri(const LaunchArgs& a, int precision, bool assemble);
int launch_simt_tet_mass(const LaunchArgs& a, int precision, bool assemble);
int launch_simt_tet_poisson(const LaunchArgs& a, int precision, bool assemble);
int launch_simt_vector(const LaunchArgs& a, int precision, bool assemble);
int launch_simt_source(const LaunchArgs& a, int precision, bool assemble);
int launch_tc(const LaunchArgs& a, int precision, bool assemble);
int launch_simt_block(const LaunchArgs& a, int precision, bool assemble);
int launch_adjoint(const LaunchArgs& a, const double* dA, double* dvert);
int launch_bounded_wait_probe(uint32_t polls, unsigned* status, void* stream);
// the mass + Poisson pair in one launch (FP32 contraction); a.f is either form of the pair
int launch_simt_pair(const LaunchArgs& a, const DeviceTensors* t_mass, const DeviceTensors* t_poisson,
                     double* val_mass, double* val_poisson);
int launch_scatter_add(const void* a, int precision, const int32_t* slot, double* csr_val, long long nnz,
                       long long total, unsigned* status, void* stream);

}  // namespace ffc
