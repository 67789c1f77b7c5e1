"""Pins of the oracle's mesh and assembly (oracle/mesh.py, oracle/assembly.py).

P2 elements reproduce quadratics, so for u interpolating a global quadratic p the
assembled forms must equal exact polynomial integrals over the box [0, L]^d
(Section 3: M, K, N(psi) and the load (psi^3, phi)).  The exact integrals are
computed here from monomial coefficients, independently of any quadrature.
"""
import numpy as np
import pytest
import scipy.signal

import synth
from oracle import assembly
from oracle.mesh import structured_mesh


def _rand_quadratic(dim, seed):
    c = np.zeros((3,) * dim)
    u = synth.random_vector(3 ** dim, seed).reshape(c.shape)
    for idx in np.ndindex(c.shape):
        if sum(idx) <= 2:
            c[idx] = u[idx]
    return c


def _peval(c, x):
    out = np.zeros(x.shape[0])
    for idx in np.ndindex(c.shape):
        if c[idx] != 0.0:
            out += c[idx] * np.prod(x ** np.array(idx), axis=1)
    return out


def _pmul(a, b):
    return scipy.signal.convolve(a, b, method="direct")


def _pint(c, L):
    tot = 0.0
    for idx in np.ndindex(c.shape):
        tot += c[idx] * np.prod([L ** (k + 1) / (k + 1) for k in idx])
    return tot


def _pdiff(c, axis):
    d = np.zeros_like(c)
    for idx in np.ndindex(c.shape):
        if idx[axis] > 0:
            j = list(idx)
            j[axis] -= 1
            d[tuple(j)] += idx[axis] * c[idx]
    return d


CASES = [(2, 1, 1.0), (2, 3, 4.5), (2, 5, 5.0), (3, 1, 1.0), (3, 2, 3.0)]


@pytest.fixture(scope="module", params=CASES, ids=[f"{d}d-s{s}" for d, s, _ in CASES])
def fem(request):
    dim, side, L = request.param
    mesh = structured_mesh(dim, side, L)
    ref = assembly.Reference(dim)
    return mesh, ref, assembly.mass_matrix(mesh, ref), assembly.stiffness_matrix(mesh, ref), L


def test_dof_and_nnz_counts():
    for s in (1, 2, 3, 5, 8):
        m = structured_mesh(2, s, 1.0)
        assert m.n == (2 * s + 1) ** 2
        assert assembly.pattern_nnz(m) == 46 * s * s + 16 * s + 1
    for s in (1, 2, 3):
        m = structured_mesh(3, s, 1.0)
        assert m.n == (2 * s + 1) ** 3
        assert assembly.pattern_nnz(m) == 230 * s ** 3 + 138 * s ** 2 + 24 * s + 1


def test_mass_sum_is_volume_and_stiffness_kills_constants(fem):
    mesh, _, M, K, L = fem
    one = np.ones(mesh.n)
    assert one @ (M @ one) == pytest.approx(L ** mesh.dim, rel=1e-13)
    assert np.abs(K @ one).max() < 1e-12 * abs(K).max()
    assert abs(M - M.T).max() < 1e-15 * abs(M).max()
    assert abs(K - K.T).max() < 1e-14 * abs(K).max()


def test_quadratic_reproduction(fem):
    mesh, ref, M, K, L = fem
    dim = mesh.dim
    p = _rand_quadratic(dim, 11)
    q = _rand_quadratic(dim, 12)
    u, v = _peval(p, mesh.coords), _peval(q, mesh.coords)
    # (p, q) and (grad p, grad q)
    assert u @ (M @ v) == pytest.approx(_pint(_pmul(p, q), L), rel=1e-12)
    gg = sum(_pmul(_pdiff(p, k), _pdiff(q, k)) for k in range(dim))
    assert u @ (K @ v) == pytest.approx(_pint(gg, L), rel=1e-12)
    # load (p^3, phi): tested against 1 and against q
    l3 = assembly.load_cubed(mesh, u, ref)
    p3 = _pmul(_pmul(p, p), p)
    assert l3.sum() == pytest.approx(_pint(p3, L), rel=1e-12)
    assert l3 @ v == pytest.approx(_pint(_pmul(p3, q), L), rel=1e-12)
    # N(p) = ((-3 p^2 phi_j, phi_i)):  v^T N w = -3 int p^2 q s
    s = _rand_quadratic(dim, 13)
    w = _peval(s, mesh.coords)
    N = assembly.nonlinear_mass(mesh, u, ref)
    want = -3.0 * _pint(_pmul(_pmul(_pmul(p, p), q), s), L)
    assert v @ (N @ w) == pytest.approx(want, rel=1e-12)


def test_nonlinear_mass_of_constant(fem):
    mesh, ref, M, _, _ = fem
    c = -0.37
    N = assembly.nonlinear_mass(mesh, np.full(mesh.n, c), ref)
    assert abs(N - (-3.0 * c * c) * M).max() < 1e-14 * abs(M).max()


def test_two_exact_rules_agree(fem):
    mesh, _, _, _, _ = fem
    psi = synth.initial_psi(mesh.dim, mesh.side, -0.3, 0.2, 7)
    r5, r7 = assembly.Reference(mesh.dim, 5), assembly.Reference(mesh.dim, 7)
    N5 = assembly.nonlinear_mass(mesh, psi, r5)
    N7 = assembly.nonlinear_mass(mesh, psi, r7)
    assert abs(N5 - N7).max() < 1e-13 * abs(N5).max()
    l5, l7 = assembly.load_cubed(mesh, psi, r5), assembly.load_cubed(mesh, psi, r7)
    assert np.abs(l5 - l7).max() < 1e-13 * np.abs(l5).max()
    # a rule that is too coarse (degree 5) must differ: the integrand has degree 8
    r3 = assembly.Reference(mesh.dim, 3)
    assert abs(assembly.nonlinear_mass(mesh, psi, r3) - N5).max() > 1e-10 * abs(N5).max()


def test_mass_positive_definite_and_stiffness_semidefinite():
    mesh = structured_mesh(2, 3, 3.0)
    M = assembly.mass_matrix(mesh).toarray()
    K = assembly.stiffness_matrix(mesh).toarray()
    assert np.linalg.eigvalsh(M).min() > 0
    ev = np.linalg.eigvalsh(K)
    assert ev.min() > -1e-12 and np.sum(np.abs(ev) < 1e-10) == 1   # only constants in the kernel


@pytest.mark.parametrize("dim,side,lengths", [
    # parity class (x, y[, z] mod 2, x fastest) -> nonzeros of a row with all its elements
    (2, 12, [19, 9, 9, 9]),
    (3, 6, [65, 27, 27, 19, 27, 19, 19, 27]),
])
def test_interior_row_lengths_per_lattice_parity_class(dim, side, lengths):
    # P2 dofs are the half-spacing lattice (Section 2); a row couples the nodes of the
    # elements around it, so rows with every element present have one length per
    # parity class of the lattice point: vertices (all even) the longest.  The
    # structured stencils are one table per class, and a warp over 32 consecutive rows
    # runs to the longest one among them.
    mesh = structured_mesh(dim, side, float(side))
    lens = np.diff(assembly.mass_matrix(mesh).tocsr().indptr)
    m = 2 * side + 1
    coords = np.stack(np.unravel_index(np.arange(m ** dim), (m,) * dim, order="F"), axis=1)
    interior = np.all((coords >= 2) & (coords <= m - 3), axis=1)
    cls = (coords % 2) @ (2 ** np.arange(dim))
    for c, want in enumerate(lengths):
        assert set(lens[interior & (cls == c)].tolist()) == {want}
    if dim == 2:
        # along an even lattice line classes 0 and 1 alternate, along an odd one 2 and 3:
        # a 32-row warp loops to the longer stencil rounded up to the table's multiple of 4
        def pad(k):
            return (k + 3) // 4 * 4

        issued = 32 * pad(max(lengths[0], lengths[1])) + 32 * pad(max(lengths[2], lengths[3]))
        useful = 16 * sum(lengths)
        assert issued / useful == pytest.approx(1024 / 736)


@pytest.mark.parametrize("dim,side,ratio", [(2, 512, 1.403), (3, 64, 1.418)])
def test_warp_uniform_stencil_loop_padding_on_the_benchmark_meshes(dim, side, ratio):
    # Gathers a 32-row warp issues when every lane loops to the longest interior stencil
    # among its rows (rounded up to a multiple of 4), against the gathers the rows need,
    # on the 2D 512^2 and 3D 64^3 meshes.  Interior: the row's incident-element count is
    # the largest of its parity class (every element around it exists); the lengths per
    # class are the ones pinned above.
    lengths = {2: [19, 9, 9, 9], 3: [65, 27, 27, 19, 27, 19, 19, 27]}[dim]
    mesh = structured_mesh(dim, side, float(side))
    m = 2 * side + 1
    n = m ** dim
    inc = np.bincount(mesh.elem_dofs.ravel(), minlength=n)
    coords = np.stack(np.unravel_index(np.arange(n), (m,) * dim, order="F"), axis=1)
    cls = (coords % 2) @ (2 ** np.arange(dim))
    interior = np.zeros(n, dtype=bool)
    for c in range(2 ** dim):
        sel = cls == c
        interior[sel] = inc[sel] == inc[sel].max()
    per_row = np.zeros((n + 31) // 32 * 32, dtype=np.int64)
    per_row[:n] = np.where(interior, np.asarray(lengths)[cls], 0)
    per_row = per_row.reshape(-1, 32)
    nmax = per_row.max(axis=1)
    issued = int(((nmax + 3) // 4 * 4 * 32)[nmax > 0].sum())
    assert issued / int(per_row.sum()) == pytest.approx(ratio, abs=1e-3)
