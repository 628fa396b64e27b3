"""The oracle's pins catch plausible mistakes: each test plants one mistake in the
oracle (on the CPU, through monkeypatching) and checks that an independent pin
(exact rational values, printed values, closed forms) then fails."""
from fractions import Fraction

import numpy as np

import exact_forms as X
from oracle import basis, element, quadrature
from oracle.element import ELASTICITY, MASS, NS_CONVECTION, POISSON

TET = [(Fraction(1, 3), 0, 0), (Fraction(1, 2), Fraction(1, 10), 0), (Fraction(1, 5), Fraction(3, 5), Fraction(1, 7)),
       (Fraction(1, 9), Fraction(1, 4), Fraction(2, 3))]
TET_NEG = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (Fraction(1, 2), Fraction(1, 2), Fraction(-3, 4))]
W = [Fraction((7 * i) % 11 - 5, 3) for i in range(30)]


def _exact_pins_hold(form, q, verts=TET, w=None):
    vf = np.array([[float(c) for c in v] for v in verts])[None]
    ref = np.array(X.element_tensor(form, [tuple(Fraction(c) for c in v) for v in verts], q, w=w), dtype=float)
    coeffs = None if w is None else np.array([[float(x) for x in w]])
    A = element.element_tensors(form, vf, q, coeffs=coeffs)[0]
    return np.abs(A - ref).max() <= 1e-13 * np.abs(ref).max()


def _printed_p3_pin_holds():
    v = np.array([[[0, 0], [1, 0], [1, 1]]], float)
    A = element.element_tensors(POISSON, v, 3)[0]
    return np.allclose([A[0, 0], A[0, 1], A[0, 2], A[9, 9]], [0.425, -0.0875, 0.0, 8.1], atol=1e-13)


def test_unmutated_oracle_passes_the_pins():
    assert _exact_pins_hold(NS_CONVECTION, 2, w=W)
    assert _exact_pins_hold(ELASTICITY, 2)
    assert _exact_pins_hold(MASS, 3, TET_NEG)
    assert _printed_p3_pin_holds()


def test_transposed_convection_operands_are_caught(monkeypatch):
    orig = element.element_tensors

    def mutated(form, verts, q, coeffs=None, **kw):
        A = orig(form, verts, q, coeffs=coeffs, **kw)
        return np.swapaxes(A, 1, 2) if form == NS_CONVECTION else A  # v and u exchanged

    monkeypatch.setattr(element, "element_tensors", mutated)
    assert not _exact_pins_hold(NS_CONVECTION, 2, w=W)


def test_dropped_lambda_term_is_caught(monkeypatch):
    orig = element.element_tensors
    monkeypatch.setattr(element, "element_tensors",
                        lambda form, verts, q, coeffs=None, **kw: orig(form, verts, q, coeffs=coeffs, lmbda=0.0))
    assert not _exact_pins_hold(ELASTICITY, 2)


def test_dropped_symmetric_strain_half_is_caught(monkeypatch):
    orig = element.element_tensors

    def mutated(form, verts, q, coeffs=None, **kw):
        # grad-grad instead of eps:eps: 2 mu grad:grad + lambda div div differs from the pin
        if form != ELASTICITY:
            return orig(form, verts, q, coeffs=coeffs, **kw)
        P = orig(POISSON, verts, q)
        out = orig(form, verts, q, coeffs=coeffs, **kw)
        ns = P.shape[1]
        for c in range(verts.shape[2]):
            out[:, c * ns:(c + 1) * ns, c * ns:(c + 1) * ns] = 2 * P
        return out

    monkeypatch.setattr(element, "element_tensors", mutated)
    assert not _exact_pins_hold(ELASTICITY, 2)


def test_signed_determinant_is_caught(monkeypatch):
    orig = element.barycentric_geometry

    def mutated(verts):
        g, vol = orig(verts)
        E, dp1, d = verts.shape
        M = np.concatenate([np.ones((E, dp1, 1)), verts], axis=2)
        return g, np.linalg.det(M) / (2 if d == 2 else 6)

    monkeypatch.setattr(element, "barycentric_geometry", mutated)
    assert not _exact_pins_hold(MASS, 3, TET_NEG)


def test_underintegration_is_caught(monkeypatch):
    orig = element.integrand_degree
    monkeypatch.setattr(element, "integrand_degree", lambda form, q: max(0, orig(form, q) - 2))
    assert not _exact_pins_hold(MASS, 3)


def test_wrong_gradient_sign_in_basis_is_caught(monkeypatch):
    orig = basis.bary_derivatives
    monkeypatch.setattr(basis, "bary_derivatives", lambda d, q, lam: -orig(d, q, lam) if q == 2 else orig(d, q, lam))
    # Poisson is quadratic in gradients; the convection form is linear in them
    assert not _exact_pins_hold(NS_CONVECTION, 2, w=W)


def test_swapped_local_order_is_caught(monkeypatch):
    orig = basis.lattice

    def mutated(d, q):
        ks = orig(d, q)
        if d == 2 and q == 3:
            ks[0], ks[1] = ks[1], ks[0]
        return ks

    monkeypatch.setattr(basis, "lattice", mutated)
    assert not _printed_p3_pin_holds()


def test_wrong_quadrature_weights_are_caught(monkeypatch):
    orig = quadrature.simplex_rule

    def mutated(d, p, extra=0):
        lam, w = orig(d, p, extra)
        w = w.copy()
        w[0] *= 1.01
        return lam, w / w.sum()

    monkeypatch.setattr(quadrature, "simplex_rule", mutated)
    assert not _exact_pins_hold(POISSON, 2)
