// Host form compiler: the reference tensor A0 of each supported form, computed
// once per (form, cell, degree) in FP64 (Section 3.2: A0 is independent of the
// cell and precomputed; Section 5.3: its entries are integrals over the reference
// simplex by a quadrature rule matched to the integrand degree; Section 6: the
// rules are the collapsed-coordinate Gauss-Jacobi rules of Karniadakis & Sherwin).
//
// Reference simplex K0: vertices 0, e_1, ..., e_d; barycentric coordinates
// lambda_0 = 1 - sum X, lambda_j = X_j. Lagrange basis on the lattice of step 1/q
// through Silvester's product formula; reference gradients
// dPsi/dX_a = dPsi/dlambda_{a+1} - dPsi/dlambda_0.
//
// Index layouts of A0[i][alpha] (i = i1*n + i2; alpha as below) and the matching
// geometry tensors G_K computed on the device (K = J^{-1}, det = |det J|):
//   mass        alpha = 0                     A0 = int Psi_i1 Psi_i2             G = det
//   Poisson     alpha = a1*d + a2             A0 = int d_a1 Psi_i1 d_a2 Psi_i2   G = det sum_b K[a1][b] K[a2][b]
//               (the CUDA-core kernels use the symmetry of G, Section 3.5: one column per
//               pair a1 <= a2, diagonal pairs first, the two off-diagonal columns summed)
//   convection  alpha = t*d + a  (t = coefficient dof, component c(t))
//               A0 = int Phi_i1[b] Phi_t[c(t)] d_a Phi_i2[b]                     G = det K[a][c(t)] w_t
//               (eq. (navierstokes) with alpha_1 = c(alpha_2) for a component-blocked basis)
//   source      (rank 1, i = test index) alpha = t (coefficient dof)
//               A0 = int Psi_i Psi_t                                             G = det f_t
//   elasticity  alpha = ((b1*d + b2)*d + a1)*d + a2
//               A0 = delta(c(i1), b1) delta(c(i2), b2) int d_a1 Psi_s1 d_a2 Psi_s2
//               G  = det (mu delta(b1,b2) (K K^T)[a1][a2] + mu K[a1][b2] K[a2][b1]
//                         + lambda K[a1][b1] K[a2][b2])
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <vector>

#include "ffc_internal.h"

namespace ffc {

int sym_pair(int d, int a, int b) {
  if (a > b) std::swap(a, b);
  if (a == b) return a;
  return d == 2 ? 2 : (a == 0 ? (b == 1 ? 3 : 4) : 5);
}

int n_scalar_local(int d, int q) {
  int num = 1;
  for (int j = 1; j <= d; ++j) num = num * (q + j) / j;
  return num;
}

namespace {

// Lattice multi-indices in the local dof order (see ffc_gb300.h).
std::vector<std::vector<int>> local_lattice(int d, int q) {
  std::vector<std::vector<int>> all;
  std::vector<int> k(d + 1, 0);
  // enumerate all k with |k| = q
  std::function<void(int, int)> rec = [&](int j, int left) {
    if (j == d) {
      k[d] = left;
      all.push_back(k);
      return;
    }
    for (int v = 0; v <= left; ++v) {
      k[j] = v;
      rec(j + 1, left - v);
    }
  };
  rec(0, q);
  std::vector<std::vector<int>> out;
  for (int m = 0; m <= d; ++m) {
    // vertex subsets of size m+1 in lexicographic order
    std::vector<int> sub(m + 1);
    for (int i = 0; i <= m; ++i) sub[i] = i;
    while (true) {
      std::vector<std::vector<int>> pts;
      for (auto& kk : all) {
        bool ok = true;
        for (int j = 0, s = 0; j <= d; ++j) {
          bool in = (s <= m && sub[s] == j);
          if (in) ++s;
          if (in != (kk[j] > 0)) { ok = false; break; }
        }
        if (ok) pts.push_back(kk);
      }
      std::sort(pts.begin(), pts.end(), [](const std::vector<int>& a, const std::vector<int>& b) {
        return a > b;  // descending lexicographic
      });
      out.insert(out.end(), pts.begin(), pts.end());
      // next subset
      int i = m;
      while (i >= 0 && sub[i] == d - m + i) --i;
      if (i < 0) break;
      ++sub[i];
      for (int j = i + 1; j <= m; ++j) sub[j] = sub[j - 1] + 1;
    }
  }
  return out;
}

// Jacobi polynomial P_n^{(a,b)}(x) and its derivative by the three-term recurrence.
void jacobi(int n, double a, double b, double x, double* p, double* dp) {
  auto eval = [&](int nn, double aa, double bb) {
    if (nn == 0) return 1.0;
    double p0 = 1.0;
    double p1 = 0.5 * (aa - bb + (aa + bb + 2.0) * x);
    for (int k = 2; k <= nn; ++k) {
      double c = 2.0 * k + aa + bb;
      double a1 = 2.0 * k * (k + aa + bb) * (c - 2.0);
      double a2 = (c - 1.0) * (aa * aa - bb * bb);
      double a3 = (c - 2.0) * (c - 1.0) * c;
      double a4 = 2.0 * (k + aa - 1.0) * (k + bb - 1.0) * c;
      double p2 = ((a2 + a3 * x) * p1 - a4 * p0) / a1;
      p0 = p1;
      p1 = p2;
    }
    return p1;
  };
  *p = eval(n, a, b);
  *dp = n == 0 ? 0.0 : 0.5 * (n + a + b + 1.0) * eval(n - 1, a + 1.0, b + 1.0);
}

// Gauss-Jacobi rule with weight (1-x)^a (1+x)^b on [-1,1], mapped to [0,1]
// (weight (1-u)^a u^b): Newton iteration with deflation from Chebyshev guesses.
void gauss_jacobi01(int m, double a, double b, std::vector<double>& u, std::vector<double>& w) {
  std::vector<double> x(m);
  for (int k = 0; k < m; ++k) {
    double r = -std::cos((2.0 * k + 1.0) * M_PI / (2.0 * m));
    if (k > 0) r = 0.5 * (r + x[k - 1]);
    for (int it = 0; it < 200; ++it) {
      double p, dp;
      jacobi(m, a, b, r, &p, &dp);
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += 1.0 / (r - x[j]);
      double delta = -p / (dp - s * p);
      r += delta;
      if (std::fabs(delta) < 1e-17) break;
    }
    x[k] = r;
  }
  std::sort(x.begin(), x.end());
  // w_k = 2^{a+b+1} G(m+a+1) G(m+b+1) / (G(m+a+b+1) m!) / ((1-x^2) P'(x)^2)
  double lc = (a + b + 1.0) * std::log(2.0) + std::lgamma(m + a + 1.0) + std::lgamma(m + b + 1.0) -
              std::lgamma(m + a + b + 1.0) - std::lgamma(m + 1.0);
  double c = std::exp(lc);
  u.resize(m);
  w.resize(m);
  for (int k = 0; k < m; ++k) {
    double p, dp;
    jacobi(m, a, b, x[k], &p, &dp);
    double wx = c / ((1.0 - x[k] * x[k]) * dp * dp);
    u[k] = 0.5 * (1.0 + x[k]);
    w[k] = wx / std::pow(2.0, a + b + 1.0);
  }
}

// Collapsed rule on K0 exact for degree p: points X [N][d], weights summing to 1/d!.
void collapsed_rule(int d, int p, std::vector<double>& X, std::vector<double>& W) {
  int m = std::max(1, (p + 2) / 2);  // ceil((p+1)/2)
  std::vector<std::vector<double>> u(d), w(d);
  for (int k = 0; k < d; ++k) gauss_jacobi01(m, double(k), 0.0, u[k], w[k]);
  int N = 1;
  for (int k = 0; k < d; ++k) N *= m;
  X.assign(size_t(N) * d, 0.0);
  W.assign(N, 0.0);
  for (int idx = 0; idx < N; ++idx) {
    int r = idx;
    std::vector<int> ix(d);
    for (int k = d - 1; k >= 0; --k) { ix[k] = r % m; r /= m; }
    double wt = 1.0;
    for (int k = 0; k < d; ++k) wt *= w[k][ix[k]];
    // X_k = u_k prod_{l>k} (1 - u_l)
    for (int k = 0; k < d; ++k) {
      double v = u[k][ix[k]];
      for (int l = k + 1; l < d; ++l) v *= 1.0 - u[l][ix[l]];
      X[size_t(idx) * d + k] = v;
    }
    W[idx] = wt;
  }
}

// Silvester basis value and barycentric partial derivatives at one point.
void silvester(int d, int q, const std::vector<int>& k, const double* lam, double* val, double* dlam) {
  std::vector<double> f(d + 1), df(d + 1);
  for (int j = 0; j <= d; ++j) {
    double prod = 1.0, der = 0.0;
    for (int m = 0; m < k[j]; ++m) {
      double fac = (q * lam[j] - m) / (m + 1);
      der = der * fac + prod * (double(q) / (m + 1));
      prod *= fac;
    }
    f[j] = prod;
    df[j] = der;
  }
  double v = 1.0;
  for (int j = 0; j <= d; ++j) v *= f[j];
  *val = v;
  for (int j = 0; j <= d; ++j) {
    double t = df[j];
    for (int l = 0; l <= d; ++l)
      if (l != j) t *= f[l];
    dlam[j] = t;
  }
}

}  // namespace

void reference_rule(int d, int p, std::vector<double>& X, std::vector<double>& W) { collapsed_rule(d, p, X, W); }

void reference_basis(int d, int q, const std::vector<double>& X, std::vector<double>& psi, std::vector<double>& dpsi) {
  auto lat = local_lattice(d, q);
  const int ns = int(lat.size()), N = int(X.size()) / d;
  psi.assign(size_t(N) * ns, 0.0);
  dpsi.assign(size_t(N) * ns * d, 0.0);
  std::vector<double> lam(d + 1), dl(d + 1);
  for (int iq = 0; iq < N; ++iq) {
    double s = 0.0;
    for (int a = 0; a < d; ++a) { lam[a + 1] = X[size_t(iq) * d + a]; s += lam[a + 1]; }
    lam[0] = 1.0 - s;
    for (int i = 0; i < ns; ++i) {
      double v;
      silvester(d, q, lat[i], lam.data(), &v, dl.data());
      psi[size_t(iq) * ns + i] = v;
      for (int a = 0; a < d; ++a) dpsi[(size_t(iq) * ns + i) * d + a] = dl[a + 1] - dl[0];
    }
  }
}

int compile_reference_tensor(ffc_form* f) {
  const int d = f->d, q = f->q, ns = f->ns, n = f->n;
  auto lat = local_lattice(d, q);
  if (int(lat.size()) != ns) return FFC_EINVAL;
  int p;
  switch (f->kind) {
    case FFC_MASS:
    case FFC_SOURCE: p = 2 * q; break;
    case FFC_POISSON:
    case FFC_ELASTICITY: p = std::max(0, 2 * q - 2); break;
    case FFC_NS_CONVECTION: p = 3 * q - 1; break;
    default: return FFC_EINVAL;
  }
  std::vector<double> X, W;
  collapsed_rule(d, p, X, W);
  const int N = int(W.size());
  // tabulate Psi and dPsi/dX on the rule
  std::vector<double> psi(size_t(N) * ns), dpsi(size_t(N) * ns * d);
  std::vector<double> lam(d + 1), dl(d + 1);
  for (int iq = 0; iq < N; ++iq) {
    double s = 0.0;
    for (int a = 0; a < d; ++a) { lam[a + 1] = X[size_t(iq) * d + a]; s += lam[a + 1]; }
    lam[0] = 1.0 - s;
    for (int i = 0; i < ns; ++i) {
      double v;
      silvester(d, q, lat[i], lam.data(), &v, dl.data());
      psi[size_t(iq) * ns + i] = v;
      for (int a = 0; a < d; ++a) dpsi[(size_t(iq) * ns + i) * d + a] = dl[a + 1] - dl[0];
    }
  }
  const int na = f->na;
  f->A0.assign(f->n_entries() * na, 0.0);
  if (f->kind == FFC_SOURCE) {
    for (int i = 0; i < ns; ++i)
      for (int t = 0; t < ns; ++t) {
        double s = 0.0;
        for (int iq = 0; iq < N; ++iq) s += W[iq] * psi[size_t(iq) * ns + i] * psi[size_t(iq) * ns + t];
        f->A0[size_t(i) * na + t] = s;
      }
    return FFC_OK;
  }
  auto A0 = [&](int i1, int i2, int alpha) -> double& { return f->A0[(size_t(i1) * n + i2) * na + alpha]; };
  // reduced reference tensors of the vector forms (component-blocked Cartesian basis)
  if (f->kind == FFC_ELASTICITY) {
    f->kr = d * d;
    f->nb = d * d;
  } else if (f->kind == FFC_NS_CONVECTION) {
    f->kr = ns * d;
    f->nb = 1;
  }
  if (f->kr > 0) f->R.assign(size_t(ns) * ns * f->kr, 0.0);
  if (f->kind == FFC_MASS) {
    for (int i1 = 0; i1 < ns; ++i1)
      for (int i2 = 0; i2 < ns; ++i2) {
        double s = 0.0;
        for (int iq = 0; iq < N; ++iq) s += W[iq] * psi[size_t(iq) * ns + i1] * psi[size_t(iq) * ns + i2];
        A0(i1, i2, 0) = s;
      }
  } else if (f->kind == FFC_POISSON || f->kind == FFC_ELASTICITY) {
    // scalar stiffness blocks S[s1][s2][a1][a2]
    std::vector<double> S(size_t(ns) * ns * d * d, 0.0);
    for (int s1 = 0; s1 < ns; ++s1)
      for (int s2 = 0; s2 < ns; ++s2)
        for (int a1 = 0; a1 < d; ++a1)
          for (int a2 = 0; a2 < d; ++a2) {
            double s = 0.0;
            for (int iq = 0; iq < N; ++iq)
              s += W[iq] * dpsi[(size_t(iq) * ns + s1) * d + a1] * dpsi[(size_t(iq) * ns + s2) * d + a2];
            S[((size_t(s1) * ns + s2) * d + a1) * d + a2] = s;
          }
    if (f->kind == FFC_POISSON) {
      for (int s1 = 0; s1 < ns; ++s1)
        for (int s2 = 0; s2 < ns; ++s2)
          for (int a = 0; a < d * d; ++a) A0(s1, s2, a) = S[(size_t(s1) * ns + s2) * d * d + a];
      f->nak = d * (d + 1) / 2;
      f->A0k.assign(size_t(n) * n * f->nak, 0.0);
      for (size_t i = 0; i < size_t(n) * n; ++i)
        for (int a1 = 0; a1 < d; ++a1)
          for (int a2 = a1; a2 < d; ++a2) {
            const double* row = &f->A0[i * na];
            const double v = (a1 == a2) ? row[a1 * d + a1] : row[a1 * d + a2] + row[a2 * d + a1];
            f->A0k[i * f->nak + sym_pair(d, a1, a2)] = v;
          }
    } else {
      for (int c1 = 0; c1 < d; ++c1)
        for (int s1 = 0; s1 < ns; ++s1)
          for (int c2 = 0; c2 < d; ++c2)
            for (int s2 = 0; s2 < ns; ++s2)
              for (int a1 = 0; a1 < d; ++a1)
                for (int a2 = 0; a2 < d; ++a2) {
                  int alpha = ((c1 * d + c2) * d + a1) * d + a2;
                  A0(c1 * ns + s1, c2 * ns + s2, alpha) = S[((size_t(s1) * ns + s2) * d + a1) * d + a2];
                }
      f->R = S;  // R[(s1,s2)][(a1,a2)]: the scalar stiffness blocks
    }
  } else {  // convection
    for (int s1 = 0; s1 < ns; ++s1)
      for (int s2 = 0; s2 < ns; ++s2)
        for (int st = 0; st < ns; ++st)
          for (int a = 0; a < d; ++a) {
            double s = 0.0;
            for (int iq = 0; iq < N; ++iq)
              s += W[iq] * psi[size_t(iq) * ns + s1] * psi[size_t(iq) * ns + st] *
                   dpsi[(size_t(iq) * ns + s2) * d + a];
            for (int c = 0; c < d; ++c)          // test/trial component (delta(c1, c2))
              for (int ct = 0; ct < d; ++ct)     // coefficient component c(t)
                A0(c * ns + s1, c * ns + s2, (ct * ns + st) * d + a) = s;
            f->R[(size_t(s1) * ns + s2) * f->kr + st * d + a] = s;
          }
  }
  return FFC_OK;
}

}  // namespace ffc
