"""Exact rational element tensors and reference tensors (test-only).

An independent route to the same integrals as the oracle and the form compiler:
* the Lagrange basis on the reference simplex is obtained by inverting the
  monomial Vandermonde matrix at the lattice nodes exactly, in ``fractions``
  (no Silvester product, no quadrature);
* integrals use the simplex moment formula
  int_{K0} X_1^a_1 ... X_d^a_d dX = a_1! ... a_d! / (a_1 + ... + a_d + d)!;
* on a physical element with rational vertices, the change of variables of
  Section 3.2 (affine F_K, J = [x_1 - x_0, ..., x_d - x_0]) pulls each integral
  back to K0 exactly: physical gradients are J^{-T} times reference gradients
  and dx = |det J| dX.

Small degrees only (cost grows fast with q).
"""
from __future__ import annotations

import itertools
from fractions import Fraction
from functools import lru_cache
from math import factorial

from synthetic.dofmap import local_lattice


def monomials(d: int, q: int):
    return [a for a in itertools.product(range(q + 1), repeat=d) if sum(a) <= q]


def moment(a) -> Fraction:
    d = len(a)
    num = 1
    for x in a:
        num *= factorial(x)
    return Fraction(num, factorial(sum(a) + d))


def _solve_identity(V):
    n = len(V)
    M = [list(row) + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(V)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [x / pv for x in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [x - f * y for x, y in zip(M[r], M[col])]
    return [row[n:] for row in M]


@lru_cache(maxsize=None)
def nodal_basis(d: int, q: int):
    """Basis polynomials as dicts {exponent: Fraction}, in the local dof order."""
    mons = monomials(d, q)
    nodes = [tuple(Fraction(int(k[j + 1]), q) for j in range(d)) for k in local_lattice(d, q)]
    V = []
    for X in nodes:
        row = []
        for a in mons:
            v = Fraction(1)
            for x, e in zip(X, a):
                v *= x**e
            row.append(v)
        V.append(row)
    Vinv = _solve_identity(V)  # coefficient of monomial m in basis s: Vinv[m][s]
    out = []
    for s in range(len(nodes)):
        out.append({a: Vinv[m][s] for m, a in enumerate(mons) if Vinv[m][s] != 0})
    return tuple(tuple(sorted(p.items())) for p in out)


def padd(p, r, scale=Fraction(1)):
    out = dict(p)
    for k, v in r.items():
        out[k] = out.get(k, Fraction(0)) + scale * v
    return out


def pmul(p, r):
    out = {}
    for a, x in p.items():
        for b, y in r.items():
            k = tuple(i + j for i, j in zip(a, b))
            out[k] = out.get(k, Fraction(0)) + x * y
    return out


def pdiff(p, axis):
    out = {}
    for a, x in p.items():
        if a[axis] > 0:
            k = list(a)
            k[axis] -= 1
            out[tuple(k)] = out.get(tuple(k), Fraction(0)) + x * a[axis]
    return out


def pint(p) -> Fraction:
    return sum((x * moment(a) for a, x in p.items()), Fraction(0))


def _basis(d, q):
    return [dict(b) for b in nodal_basis(d, q)]


def _affine(verts):
    """J (d x d, columns x_j - x_0), K = J^{-1}, |det J| in Fractions."""
    d = len(verts) - 1
    J = [[Fraction(verts[c + 1][r]) - Fraction(verts[0][r]) for c in range(d)] for r in range(d)]
    Kinv = _solve_identity(J)  # rows of J^{-1}
    det = Fraction(1)
    # determinant by elimination
    M = [row[:] for row in J]
    for col in range(d):
        piv = next(r for r in range(col, d) if M[r][col] != 0)
        if piv != col:
            M[col], M[piv] = M[piv], M[col]
            det = -det
        det *= M[col][col]
        for r in range(col + 1, d):
            f = M[r][col] / M[col][col]
            M[r] = [x - f * y for x, y in zip(M[r], M[col])]
    return J, Kinv, abs(det)


def _phys_grad(ref_polys, Kinv, d):
    """grad_x psi = J^{-T} grad_X psi: component beta = sum_a K[a][beta] d_a psi."""
    out = []
    for p in ref_polys:
        dp = [pdiff(p, a) for a in range(d)]
        g = []
        for beta in range(d):
            acc = {}
            for a in range(d):
                if Kinv[a][beta] != 0:
                    acc = padd(acc, dp[a], Kinv[a][beta])
            g.append(acc)
        out.append(g)
    return out


def element_tensor(form: int, verts, q: int, w=None, mu=Fraction(1), lmbda=Fraction(5, 4)):
    """Exact element tensor (list of lists of Fraction). form ids: 0 mass, 1 Poisson,
    2 convection (vector P_q, w = per-cell coefficients, component blocked), 3 elasticity."""
    d = len(verts) - 1
    _, Kinv, det = _affine(verts)
    psi = _basis(d, q)
    ns = len(psi)
    if form == 0:
        return [[det * pint(pmul(psi[i], psi[j])) for j in range(ns)] for i in range(ns)]
    g = _phys_grad(psi, Kinv, d)
    if form == 1:
        return [[det * sum(pint(pmul(g[i][b], g[j][b])) for b in range(d)) for j in range(ns)]
                for i in range(ns)]
    n = d * ns
    A = [[Fraction(0)] * n for _ in range(n)]
    if form == 2:
        wc = [{} for _ in range(d)]  # w as a polynomial per component
        for c in range(d):
            for s in range(ns):
                wc[c] = padd(wc[c], psi[s], Fraction(w[c * ns + s]))
        for s2 in range(ns):
            conv = {}
            for b in range(d):
                conv = padd(conv, pmul(wc[b], g[s2][b]))
            for s1 in range(ns):
                val = det * pint(pmul(psi[s1], conv))
                for c in range(d):
                    A[c * ns + s1][c * ns + s2] = val
        return A
    if form == 3:
        for c1 in range(d):
            for s1 in range(ns):
                for c2 in range(d):
                    for s2 in range(ns):
                        val = Fraction(0)
                        if c1 == c2:
                            val += mu * sum(pint(pmul(g[s1][b], g[s2][b])) for b in range(d))
                        val += mu * pint(pmul(g[s1][c2], g[s2][c1]))
                        val += lmbda * pint(pmul(g[s1][c1], g[s2][c2]))
                        A[c1 * ns + s1][c2 * ns + s2] = det * val
        return A
    raise ValueError(form)


def load_vector(verts, q: int, f):
    """Exact b^K_i = int_K psi_i f with f = sum_t f_t psi_t (rational vertices and f_t)."""
    d = len(verts) - 1
    _, _, det = _affine(verts)
    psi = _basis(d, q)
    fp = {}
    for t, ft in enumerate(f):
        fp = padd(fp, psi[t], Fraction(ft))
    return [det * pint(pmul(p, fp)) for p in psi]


def reference_tensor_poisson(d: int, q: int):
    """A0[i1][i2][a1][a2] = int_{K0} d_a1 Psi_i1 d_a2 Psi_i2 dX, exact."""
    psi = _basis(d, q)
    dp = [[pdiff(p, a) for a in range(d)] for p in psi]
    n = len(psi)
    return [[[[pint(pmul(dp[i][a1], dp[j][a2])) for a2 in range(d)] for a1 in range(d)]
             for j in range(n)] for i in range(n)]


def reference_tensor_mass(d: int, q: int):
    psi = _basis(d, q)
    n = len(psi)
    return [[pint(pmul(psi[i], psi[j])) for j in range(n)] for i in range(n)]


def reference_tensor_convection(d: int, q: int):
    """S[s1][s2][st][a] = int_{K0} Psi_s1 Psi_st d_a Psi_s2 dX (scalar block, exact)."""
    psi = _basis(d, q)
    n = len(psi)
    dp = [[pdiff(p, a) for a in range(d)] for p in psi]
    prod = [[pmul(psi[s1], psi[st]) for st in range(n)] for s1 in range(n)]
    return [[[[pint(pmul(prod[s1][st], dp[s2][a])) for a in range(d)] for st in range(n)]
             for s2 in range(n)] for s1 in range(n)]
