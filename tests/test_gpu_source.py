"""Parity of the linear source form (b^K_i = int_K phi_i f, rank-1 element tensors)
and of its assembly into a global vector with the oracle, on triangles and tetrahedra
P1-P4; edge cases; and the full 48^3 x 6 tetrahedral mesh at P4 checked by sampled
cells and by global integrals that hold at any size.

FP32 bound per entry: the kernel rounds A0 and f to FP32, sums n products with FMAs
and multiplies by |det J| rounded to FP32, n + 4 roundings in all, so
|b_i - ref_i| <= (n + 4) 2^-24 (|M_K| |f|)_i, where M_K is the element mass matrix and
|.| is taken entrywise."""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import element as OE
from synthetic import mesh as M
from synthetic import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-6


@pytest.fixture(scope="module")
def F():
    import torch

    from paper_1112_0402_gb300 import build as B

    B.build()
    import paper_1112_0402_gb300 as F

    assert torch.cuda.is_available()
    return F


def _dev(x, dtype=None):
    import torch

    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype).cuda()


def _case(d, n, q, seed=17):
    m = M.unit_square_triangles(n, 0.2, seed) if d == 2 else M.unit_cube_tets(n, 0.2, seed)
    return W.make_problem(m, W.SOURCE, q, seed=seed)


def _inputs(p):
    import torch

    return (_dev(p.mesh.cells, torch.int32), _dev(p.mesh.vertices, torch.float64),
            _dev(p.coeffs, torch.float64), _dev(p.dofmap, torch.int32))


def _entry_bound(p, V):
    Mk = OE.element_tensors(W.MASS, V, p.degree)
    return (p.n_local + 4) * 2.0**-24 * np.einsum("eij,ej->ei", np.abs(Mk), np.abs(p.coeffs))


CASES = [(2, 7, 1), (2, 5, 2), (2, 5, 3), (2, 4, 4), (3, 4, 1), (3, 3, 2), (3, 3, 3), (3, 2, 4)]


@pytest.mark.parametrize("d,n,q", CASES)
def test_source_tabulate_matches_oracle(F, d, n, q):
    p = _case(d, n, q)
    V = M.gather_cell_vertices(p.mesh)
    ref = OE.element_tensors(W.SOURCE, V, q, coeffs=p.coeffs)
    form = F.Form(F.SOURCE, d, q)
    assert form.rank == 1 and form.tensor_shape == (p.n_local,)
    cells, verts, coeffs, _ = _inputs(p)
    b64 = F.tabulate(form, cells, verts, coeffs=coeffs, precision="fp64")
    b32 = F.tabulate(form, cells, verts, coeffs=coeffs, precision="fp32")
    assert F.status_poll() == 0
    assert tuple(b64.shape) == (p.n_elem, p.n_local)
    assert OE.frobenius_rel_error(b64.cpu().numpy(), ref).max() <= FP64_TOL
    g32 = b32.double().cpu().numpy()
    assert OE.frobenius_rel_error(g32, ref).max() <= FP32_TOL
    assert np.all(np.abs(g32 - ref) <= _entry_bound(p, V))


@pytest.mark.parametrize("d,n,q", CASES)
def test_source_assembly_matches_oracle_vector(F, d, n, q):
    import torch

    p = _case(d, n, q)
    V = M.gather_cell_vertices(p.mesh)
    ref = OA.assemble_vector(OE.element_tensors(W.SOURCE, V, q, coeffs=p.coeffs), p.dofmap, p.n_dof)
    form = F.Form(F.SOURCE, d, q)
    cells, verts, coeffs, dm = _inputs(p)
    for prec, tol in (("fp64", FP64_TOL), ("fp32", FP32_TOL)):
        b = torch.zeros(p.n_dof, dtype=torch.float64, device="cuda")
        F.assemble(form, cells, verts, dm, b, coeffs=coeffs, precision=prec)
        assert F.status_poll() == 0
        got = b.cpu().numpy()
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), prec
    # the global bound: each entry sums at most valence element entries, each within its bound
    bnd = np.zeros(p.n_dof)
    np.add.at(bnd, p.dofmap.reshape(-1), _entry_bound(p, V).reshape(-1))
    assert np.all(np.abs(got - ref) <= bnd + 1e-300)


def test_source_edge_cases(F):
    import torch

    form = F.Form(F.SOURCE, F.TETRAHEDRON, 2)
    # empty input launches nothing
    e = torch.empty((0, 4), dtype=torch.int32, device="cuda")
    v = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    out = F.tabulate(form, e, v, coeffs=torch.empty((0, 10), dtype=torch.float64, device="cuda"))
    assert out.shape == (0, 10)
    # one reference cell with f = 1: b_i = int Psi_i; P2 on a tet: lambda(2 lambda - 1)
    # integrates to -|K|/20 = -1/120, 4 lambda_a lambda_b to |K|/5 = 1/30
    c1 = torch.tensor([[0, 1, 2, 3]], dtype=torch.int32, device="cuda")
    v1 = torch.tensor([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=torch.float64, device="cuda")
    b = F.tabulate(form, c1, v1, coeffs=torch.ones((1, 10), dtype=torch.float64, device="cuda"))
    assert F.status_poll() == 0
    want = np.array([-1.0 / 120] * 4 + [1.0 / 30] * 6)
    assert np.abs(b.cpu().numpy()[0] - want).max() < 1e-16
    # a linear form has no tensor-core path; coefficients are required
    with pytest.raises(F.FFCError) as ex:
        F.tabulate(form, c1, v1, coeffs=torch.ones((1, 10), dtype=torch.float64, device="cuda"),
                   precision="bf16x3")
    assert ex.value.code == -5
    L = __import__("paper_1112_0402_gb300._capi", fromlist=["lib"]).lib()
    assert L.ffc_tabulate(form.handle, 1, c1.data_ptr(), v1.data_ptr(), 4, None, b.data_ptr(), 0, None) == -1
    # a dof id outside the vector is skipped and reported
    bad = torch.tensor([[0, 1, 2, 3, 4, 5, 6, 7, 8, 99]], dtype=torch.int32, device="cuda")
    vec = torch.zeros(10, dtype=torch.float64, device="cuda")
    F.assemble(form, c1, v1, bad, vec, coeffs=torch.ones((1, 10), dtype=torch.float64, device="cuda"))
    assert F.status_poll() == F.FLAG_BOUNDS
    assert abs(vec.sum().item() - 4 / 30) < 1e-16


def test_source_static_entry_matches_tabulate(F):
    import ctypes

    import torch

    from paper_1112_0402_gb300 import _capi

    p = _case(3, 3, 3)
    form = F.Form(F.SOURCE, 3, 3)
    cells, verts, coeffs, _ = _inputs(p)
    ref = F.tabulate(form, cells, verts, coeffs=coeffs)
    out = torch.empty_like(ref)
    flags = ctypes.c_uint32(7)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    rc = _capi.lib().ffc_tabulate_static(form.handle, p.n_elem, vp(cells), vp(verts), verts.shape[0], vp(coeffs),
                                        vp(out), 0, None, ctypes.byref(flags))
    assert rc == 0 and flags.value == 0
    assert torch.equal(out, ref)


def test_source_full_size_p4(F):
    """48^3 x 6 tets (663,552 cells), P4, FP32 contraction with FP64 accumulation: the
    sampled element vectors agree with the oracle, and the assembled vector integrates
    interpolated polynomials exactly (b . 1 = int f, b . X = int x f)."""
    import torch

    m = W.tet_scalar_mesh(48)
    p = W.make_problem(m, W.SOURCE, 4, seed=2)
    form = F.Form(F.SOURCE, 3, 4)
    cells, verts, coeffs, dm = _inputs(p)
    b32 = F.tabulate(form, cells, verts, coeffs=coeffs, precision="fp32")
    assert F.status_poll() == 0
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(p.n_elem, size=2000, replace=False))
    sel[-1] = p.n_elem - 1
    V = M.gather_cell_vertices(m)[sel]
    ref = OE.element_tensors(W.SOURCE, V, 4, coeffs=p.coeffs[sel])
    got = b32[torch.as_tensor(sel, device="cuda")].double().cpu().numpy()
    assert OE.frobenius_rel_error(got, ref).max() <= FP32_TOL
    # global integrals with f = 1 and f = x (interpolated exactly by P4)
    from synthetic.dofmap import local_lattice

    lam = local_lattice(3, 4).astype(float) / 4
    X = np.zeros(p.n_dof)
    X[p.dofmap.reshape(-1)] = np.einsum("kj,ejx->ekx", lam, M.gather_cell_vertices(m))[..., 0].reshape(-1)
    Xd = _dev(X, torch.float64)
    # |sum_i (b_i - ref_i) u_i| <= (n + 4) 2^-24 sum_K 1^T |M_K| 1 for |f|, |u| <= 1, and
    # sum_K 1^T |M_K| 1 = |Omega| sum|M0| / |K0| with M0 the reference mass matrix
    M0 = OE.element_tensors(W.MASS, np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]]]), 4)[0]
    tol = (35 + 4) * 2.0**-24 * np.abs(M0).sum() * 6.0 + 1e-12
    for f_nodal, int_f, int_xf in ((np.ones(p.n_dof), 1.0, 0.5), (X, 0.5, 1.0 / 3.0)):
        fK = _dev(f_nodal[p.dofmap], torch.float64)
        b = torch.zeros(p.n_dof, dtype=torch.float64, device="cuda")
        F.assemble(form, cells, verts, dm, b, coeffs=fK, precision="fp32")
        assert F.status_poll() == 0
        assert abs(b.sum().item() - int_f) <= tol
        assert abs((b @ Xd).item() - int_xf) <= tol


def _conversion_cases():
    """Doubles that exercise FP64 -> FP32 round-to-nearest-even: a wide exponent range
    (normal, subnormal and overflowing FP32 results), exact ties with even and odd kept
    fractions, one unit either side of a tie, the largest finite FP32 value and its
    rounding boundary, signed zeros, infinities, NaN."""
    rng = np.random.default_rng(7)
    xs = list(rng.standard_normal(3000) * 10.0 ** rng.uniform(-50, 50, 3000))
    for _ in range(400):
        e = int(rng.integers(897, 1151))
        frac = int(rng.integers(0, 1 << 23))
        for low in (0x10000000, 0x10000001, 0x0FFFFFFF, 0, 0x1FFFFFFF):
            bits = (int(rng.integers(0, 2)) << 63) | (e << 52) | (frac << 29) | low
            xs.append(np.array([bits], dtype=np.uint64).view(np.float64)[0])
    fmax = float(np.finfo(np.float32).max)
    half_ulp = 2.0 ** (127 - 24)
    xs += [fmax, -fmax, fmax + half_ulp, fmax + half_ulp * (1 - 2 ** -30), 2.0 ** -126, 2.0 ** -126 * (1 - 2 ** -40),
           2.0 ** -149, 2.0 ** -150, 3e-46, 0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 1e300, -1e-300]
    return np.array(xs, dtype=np.float64)


def test_fp32_source_arithmetic_is_exact_ieee(F):
    """The FP32 source kernel rounds f to FP32, multiplies in FP32 and accumulates in FP64.
    On the reference tetrahedron (det J = 1) with f = (x, 0, 0, 0) and one cell per dof
    block, b[4c] = f64(RN32(RN32(x) * RN32(A0[0][0]))) for every x, ties, overflow,
    subnormal results, signed zeros, infinities and NaN included, which numpy reproduces
    exactly in IEEE float32 arithmetic."""
    import torch

    xs = _conversion_cases()
    n = xs.size
    form = F.Form(F.SOURCE, F.TETRAHEDRON, 1)
    a00 = np.float32(form.reference_tensor()[0, 0])
    cells = torch.zeros((n, 4), dtype=torch.int32, device="cuda") + torch.arange(4, dtype=torch.int32, device="cuda")
    verts = _dev(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float), torch.float64)
    f = np.zeros((n, 4))
    f[:, 0] = xs
    dm = _dev(np.arange(4 * n, dtype=np.int32).reshape(n, 4), torch.int32)
    b = torch.zeros(4 * n, dtype=torch.float64, device="cuda")
    with np.errstate(over="ignore", invalid="ignore"):
        want = (xs.astype(np.float32) * a00).astype(np.float64)
    F.assemble(form, cells, verts, dm, b, coeffs=_dev(f, torch.float64), precision="fp32")
    bt = F.tabulate(form, cells, verts, coeffs=_dev(f, torch.float64), precision="fp32")
    F.status_poll()
    got = b.cpu().numpy()[0::4]
    assert np.array_equal(got, want, equal_nan=True)
    with np.errstate(over="ignore", invalid="ignore"):
        assert np.array_equal(bt.cpu().numpy()[:, 0], want.astype(np.float32), equal_nan=True)
