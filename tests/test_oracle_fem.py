"""Pins of the oracle's discretisation (Section 2, Eqs. 1-3) against facts that
do not come from the oracle itself: exact integer identities, closed forms,
a textbook 1-D finite-element solve, geometry, and polynomial completeness."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import fem


# --------------------------------------------------------------------------
# numbering and orientation
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [2, 3])
def test_edge_count_and_geometry(dim):
    n = 4
    mesh = (W.structured_mesh_2d(n, n, relabel=True, rotate_cells=True) if dim == 2
            else W.structured_mesh_3d(n, relabel=True, rotate_cells=True))
    d = fem.number_dofs(mesh.cells, dim, 1)
    expect = 2 * n * (n + 1) if dim == 2 else 3 * n * (n + 1) ** 2
    assert d.n_edge == expect
    # lexicographic order of (lo, hi) and lo < hi
    assert np.all(d.edges[:, 0] < d.edges[:, 1])
    key = d.edges[:, 0] * mesh.n_vert + d.edges[:, 1]
    assert np.all(np.diff(key) > 0)
    # every edge joins grid neighbours: length exactly h
    L = np.linalg.norm(mesh.coords[d.edges[:, 1]] - mesh.coords[d.edges[:, 0]], axis=1)
    assert np.allclose(L, 1.0 / n, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_orientation_signs_brute_force(dim):
    """sign * (x_hi - x_lo) must equal the local edge vector (x_b - x_a)."""
    mesh = (W.structured_mesh_2d(3, 3, relabel=True, rotate_cells=True) if dim == 2
            else W.structured_mesh_3d(2, relabel=True, rotate_cells=True))
    d = fem.number_dofs(mesh.cells, dim, 1)
    X = mesh.coords
    for c in range(mesh.n_cell):
        for k, (a, b) in enumerate(fem.LOCAL_EDGES[dim]):
            va, vb = mesh.cells[c, a], mesh.cells[c, b]
            e = d.edge_of_cell[c, k]
            lo, hi = d.edges[e]
            assert {lo, hi} == {va, vb}
            assert np.array_equal(d.edge_sign[c, k] * (X[hi] - X[lo]), X[vb] - X[va])


def test_order2_numbering_layout():
    mesh = W.structured_mesh_2d(3, 2, relabel=True, rotate_cells=True)
    d1 = fem.number_dofs(mesh.cells, 2, 1)
    d2 = fem.number_dofs(mesh.cells, 2, 2)
    E = d1.n_edge
    assert d2.n_dof == 2 * E + 4 * mesh.n_cell
    assert np.array_equal(d2.cell_dofs[:, 0:8:2], 2 * d1.cell_dofs)
    assert np.array_equal(d2.cell_dofs[:, 1:8:2], 2 * d1.cell_dofs + 1)
    assert np.array_equal(d2.cell_signs[:, 0:8:2], d1.cell_signs)
    assert np.all(d2.cell_signs[:, 1:] [:, 0::2] == 1)
    assert np.array_equal(d2.cell_dofs[:, 8:], 2 * E + 4 * np.arange(mesh.n_cell)[:, None] + np.arange(4))
    # every DOF used, each interior DOF once
    assert np.array_equal(np.unique(d2.cell_dofs), np.arange(d2.n_dof))


# --------------------------------------------------------------------------
# element matrices
# --------------------------------------------------------------------------
def test_quad_order1_closed_form():
    a, b = 0.25, 0.5
    A, M = fem.element_matrices(2, 1, np.diag([a, b]))
    c = np.array([1, -1, -1, 1.0])
    assert np.allclose(A, np.outer(c, c) / (a * b), rtol=1e-14, atol=0)
    Mx = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    ref = np.zeros((4, 4))
    ref[:2, :2] = b / a * Mx
    ref[2:, 2:] = a / b * Mx
    assert np.allclose(M, ref, rtol=1e-14, atol=1e-16)


def test_hex_order1_mass_closed_form():
    h = 0.5
    A, M = fem.element_matrices(3, 1, h * np.eye(3))
    # parallel edges of one direction: self h/9, face-adjacent h/18, diagonal h/36
    blk = h * np.array([[4, 2, 2, 1], [2, 4, 1, 2], [2, 1, 4, 2], [1, 2, 2, 4]]) / 36
    for k in range(3):
        assert np.allclose(M[4 * k:4 * k + 4, 4 * k:4 * k + 4], blk, rtol=1e-14)
    off = M.copy()
    for k in range(3):
        off[4 * k:4 * k + 4, 4 * k:4 * k + 4] = 0
    assert np.abs(off).max() < 1e-16
    assert np.allclose(A, A.T) and np.linalg.eigvalsh(A).min() > -1e-13


def test_order2_mass_exact_symbolic():
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    q = lambda t: t * (1 - t)
    dq = lambda t: 1 - 2 * t
    W_ = [(1 - y, 0), (y, 0), (0, 1 - x), (0, x)]
    G = [(dq(x) * (1 - y), -q(x)), (dq(x) * y, q(x)), (-q(y), dq(y) * (1 - x)), (q(y), dq(y) * x)]
    B = [(q(y) * (1 - x), 0), (q(y) * x, 0), (0, q(x) * (1 - y)), (0, q(x) * y)]
    funcs = []
    for k in range(4):
        funcs += [W_[k], G[k]]
    funcs += B
    curl = [sympy.diff(f[1], x) - sympy.diff(f[0], y) for f in funcs]
    n = len(funcs)
    Mex = np.array([[float(sympy.integrate(funcs[i][0] * funcs[j][0] + funcs[i][1] * funcs[j][1],
                                           (x, 0, 1), (y, 0, 1))) for j in range(n)] for i in range(n)])
    Aex = np.array([[float(sympy.integrate(curl[i] * curl[j], (x, 0, 1), (y, 0, 1))) for j in range(n)]
                    for i in range(n)])
    A, M = fem.element_matrices(2, 2, np.eye(2))
    assert np.allclose(M, Mex, rtol=0, atol=1e-15)
    assert np.allclose(A, Aex, rtol=0, atol=1e-14)


def test_order2_basis_spans_Q12xQ21():
    rng = np.random.default_rng(1)
    p = rng.random((40, 2))
    V, _ = fem.ref_basis_2d(2, p[:, 0], p[:, 1])        # [40, 12, 2]
    basis = V.transpose(1, 0, 2).reshape(12, -1)
    mono = []
    for i in range(2):
        for j in range(3):
            mono.append(np.stack([p[:, 0] ** i * p[:, 1] ** j, 0 * p[:, 0]], 1).ravel())
            mono.append(np.stack([0 * p[:, 0], p[:, 0] ** j * p[:, 1] ** i], 1).ravel())
    mono = np.array(mono)
    assert np.linalg.matrix_rank(basis) == 12
    assert np.linalg.matrix_rank(np.vstack([basis, mono])) == 12


# --------------------------------------------------------------------------
# discrete de Rham: curl o grad = 0 (exact: h a power of two)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,order", [(2, 1), (2, 2), (3, 1)])
def test_curl_grad_zero(dim, order):
    if dim == 2:
        P = W.square_problem(8, 1, order, 3.0, relabel=True, rotate_cells=True)
    else:
        P = W.cube_problem(4, 1, 3.0, relabel=True, rotate_cells=True)
    S = fem.assemble(P)
    d1 = fem.number_dofs(P.mesh.cells, dim, 1)
    E, nv = d1.n_edge, P.mesh.n_vert
    G = np.zeros((S.dofs.n_dof, nv))
    stride = 1 if order == 1 else 2
    G[stride * np.arange(E), d1.edges[:, 1]] = 1.0
    G[stride * np.arange(E), d1.edges[:, 0]] = -1.0
    AG = S.A @ G
    # quadrature weights are not dyadic, so the oracle meets the identity to
    # rounding; 2-D curls are constants per term and come out exact
    tol = 0.0 if dim == 2 else 1e-13 * abs(S.A).max()
    assert np.abs(AG).max() <= tol
    if order == 2:
        assert abs(S.A[:, 1:2 * E:2]).max() == 0.0      # gradient functions are curl-free


@pytest.mark.parametrize("order", [1, 2])
def test_symmetry(order):
    """K^T = K (complex symmetric, not Hermitian); the oracle's quadrature
    products are not commutative in rounding, so this holds to 1 ulp-scale."""
    P = W.square_problem(6, 2, order, 7.0, mu_inv=W.mu_inv_lognormal(36, 0.3, "sym"), relabel=True,
                         rotate_cells=True)
    S = fem.assemble(P)
    D = (S.K - S.K.T).tocoo()
    assert (abs(D.data).max() if D.nnz else 0.0) <= 4e-16 * abs(S.K).max()
    assert abs(S.K - S.K.conj().T).max() > 0      # not Hermitian: boundary term is i*k*w*M


# --------------------------------------------------------------------------
# Dirichlet moments
# --------------------------------------------------------------------------
def test_edge_moments_linear_trace_exact():
    mesh = W.structured_mesh_2d(2, 2)
    d = fem.number_dofs(mesh.cells, 2, 2)
    # E = pol * exp(-i w d.x) with w*d small is not linear; use a tiny omega and
    # compare with the projection of the first-order Taylor expansion
    e = 0
    lo, hi = d.edges[e]
    t = mesh.coords[hi] - mesh.coords[lo]
    ell = np.linalg.norm(t)
    pol = np.array([0.3 + 0.1j, -0.7j])
    dirv = np.array([0.6, 0.8])
    om = 1e-3
    m = fem.edge_moments(d, mesh.coords, e, om, pol, dirv)
    # E_t(s) ~ alpha + beta s,  alpha = pol.t/ell e^{-iw d.x_lo},  beta = alpha*(-i w d.t)
    alpha = (pol @ t / ell) * np.exp(-1j * om * dirv @ mesh.coords[lo])
    beta = alpha * (-1j * om * dirv @ t)
    assert abs(m[0] - ell * (alpha + beta / 2)) < 1e-8 * ell
    assert abs(m[1] - (-beta * ell / 2)) < 1e-8 * ell


# --------------------------------------------------------------------------
# plane waves: the discrete 2-D/3-D solution is exactly one-dimensional
# --------------------------------------------------------------------------
def _robin_1d_p1(n, omega, kappa=1.0):
    """Vertex values of the 1-D P1 FE solution of v'' + w^2 v = 0, v(0)=1,
    v'(1) = -i k w v(1), in closed form: v_j = a e^{-i th j} + b e^{i th j}."""
    h = 1.0 / n
    th = np.arccos((6 - 2 * (omega * h) ** 2) / (6 + (omega * h) ** 2))
    d = lambda j, a, b: a * np.exp(-1j * th * j) + b * np.exp(1j * th * j)
    rob = lambda a, b: ((d(n, a, b) - d(n - 1, a, b)) / h ** 2 - omega ** 2 / 6 * (2 * d(n, a, b) + d(n - 1, a, b))
                        + 1j * kappa * omega * d(n, a, b) / h)
    Mx = np.array([[1, 1], [rob(1, 0), rob(0, 1)]])
    a, b = np.linalg.solve(Mx, [1, 0])
    return lambda x: (lambda j: d(np.floor(j), a, b) * (1 - (j - np.floor(j))) + d(np.floor(j) + 1, a, b) * (j - np.floor(j)))(np.minimum(x / h, n - 1e-12))


def _robin_1d_p2(n, omega, kappa=1.0):
    """Textbook 1-D quadratic Lagrange FE for the same problem (dense solve)."""
    h = 1.0 / n
    N = 2 * n + 1
    K = np.zeros((N, N), np.complex128)
    Ke = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / (3 * h)
    Me = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) * h / 30
    for e in range(n):
        idx = [2 * e, 2 * e + 1, 2 * e + 2]
        K[np.ix_(idx, idx)] += Ke - omega ** 2 * Me
    K[N - 1, N - 1] += 1j * kappa * omega
    rhs = -K[:, 0] * 1.0
    v = np.zeros(N, np.complex128)
    v[0] = 1.0
    v[1:] = np.linalg.solve(K[1:, 1:], rhs[1:])

    def ev(x):
        j = np.minimum(np.floor(x / h).astype(int), n - 1)
        t = x / h - j
        return (v[2 * j] * 2 * (t - 0.5) * (t - 1) + v[2 * j + 1] * (-4) * t * (t - 1)
                + v[2 * j + 2] * 2 * t * (t - 0.5))
    return ev


@pytest.mark.parametrize("order,swap", [(1, False), (2, False), (2, True)])
def test_plane_wave_2d_exact(order, swap):
    n, omega = 8, 5.0
    P = W.square_problem(n, 1, order, omega, bc="planewave", relabel=True, rotate_cells=True)
    k = 0   # propagation axis
    if swap:   # reflect the geometry across the diagonal: wave along +y, E along x
        P.mesh.coords = P.mesh.coords[:, ::-1].copy()
        P.pol = np.array([1.0, 0.0], np.complex128)
        P.direction = np.array([0.0, 1.0])
        k = 1
    S = fem.assemble(P)
    u = fem.solve_monolithic(S)
    v = _robin_1d_p1(n, omega) if order == 1 else _robin_1d_p2(n, omega)
    rng = np.random.default_rng(3)
    worst = 0.0
    for c in range(P.mesh.n_cell):
        xi = rng.random((3, 2))
        E = fem.evaluate_field(P.mesh, S.dofs, u, c, xi)
        X = fem.physical_point(P.mesh, c, xi)
        ex = v(X[:, k])
        worst = max(worst, np.abs(E[:, 1 - k] - ex).max(), np.abs(E[:, k]).max())
    assert worst < 1e-12


def test_plane_wave_3d_exact():
    n, omega = 4, 4.0
    P = W.cube_problem(n, 1, omega, bc="planewave", relabel=True, rotate_cells=True)
    S = fem.assemble(P)
    u = fem.solve_monolithic(S)
    v = _robin_1d_p1(n, omega)
    rng = np.random.default_rng(4)
    worst = 0.0
    for c in range(P.mesh.n_cell):
        xi = rng.random((2, 3))
        E = fem.evaluate_field(P.mesh, S.dofs, u, c, xi)
        X = fem.physical_point(P.mesh, c, xi)
        worst = max(worst, np.abs(E[:, 1] - v(X[:, 0])).max(), np.abs(E[:, [0, 2]]).max())
    assert worst < 1e-12


@pytest.mark.parametrize("order,rate", [(1, 2), (2, 4)])
def test_plane_wave_convergence_to_continuum(order, rate):
    """Against the exact continuum solution e^{-i w x} (first-order impedance
    with kappa=1 is exact for normal incidence): nodal/phase error O(h^{2p})."""
    omega = 6.0
    errs = []
    for n in (8, 16):
        P = W.square_problem(n, 1, order, omega, bc="planewave")
        S = fem.assemble(P)
        u = fem.solve_monolithic(S)
        c = n - 1        # cell touching x = 1 at the bottom row
        X = fem.physical_point(P.mesh, c, np.array([[1.0, 0.5]]))
        E = fem.evaluate_field(P.mesh, S.dofs, u, c, np.array([[1.0, 0.5]]))
        errs.append(abs(E[0, 1] - np.exp(-1j * omega * X[0, 0])))
    assert errs[0] / errs[1] > 0.8 * 2 ** rate


def test_residual_of_direct_solve():
    P = W.config("square32_p1")
    S = fem.assemble(P)
    u = fem.solve_monolithic(S)
    assert fem.residual(S, u) < 1e-12
    assert S.dofs.n_dof == 2112


def test_subdomain_blocks_balanced_when_side_does_not_divide():
    """s = ceil(n/32) blocks per side of a side-n square (the batch workload):
    block sizes differ by at most one cell, and a dividing s gives equal blocks."""
    for n, s in [(57, 2), (100, 4), (33, 2), (64, 2), (97, 4)]:
        mesh = W.structured_mesh_2d(n, n, s, s)
        counts = np.bincount(mesh.cell_sub, minlength=s * s)
        assert counts.size == s * s and counts.min() > 0
        assert max(counts) - min(counts) <= 2 * int(np.ceil(n / s)) + 1
        rows = np.bincount((np.arange(n) * s // n), minlength=s)
        assert rows.max() - rows.min() <= 1
        if n % s == 0:
            assert counts.min() == counts.max() == (n // s) ** 2
    probs = W.batch_problems(16)
    for P in probs:
        n = P.mesh.shape[0]
        assert P.mesh.n_sub == int(np.ceil(n / 32)) ** 2


def test_given_dirichlet_values_superpose_and_reproduce_the_plane_wave():
    """fem.with_dirichlet: Dirichlet values given as DOF values.  With the
    plane wave's own moments it is the plane-wave problem (same solution);
    the solution is linear in the data (superposition of two random data
    sets), and its Dirichlet entries are the data."""
    P = W.square_problem(6, 2, 2, 7.0, mu_inv=W.mu_inv_lognormal(36, 0.3, "given"), relabel=True,
                         rotate_cells=True)
    S = fem.assemble(P)
    dd = np.flatnonzero(S.is_dir)
    u_pw = fem.solve_monolithic(S)
    u_same = fem.solve_monolithic(fem.with_dirichlet(S, S.uD[dd]))
    assert np.linalg.norm(u_same - u_pw) <= 1e-12 * np.linalg.norm(u_pw)
    r = np.random.default_rng(3)
    d1 = r.standard_normal(len(dd)) + 1j * r.standard_normal(len(dd))
    d2 = r.standard_normal(len(dd)) + 1j * r.standard_normal(len(dd))
    u1 = fem.solve_monolithic(fem.with_dirichlet(S, d1))
    u2 = fem.solve_monolithic(fem.with_dirichlet(S, d2))
    u12 = fem.solve_monolithic(fem.with_dirichlet(S, 2.0 * d1 - 0.5j * d2))
    assert np.linalg.norm(u12 - (2.0 * u1 - 0.5j * u2)) <= 1e-11 * np.linalg.norm(u12)
    assert np.array_equal(u1[dd], d1)


# --------------------------------------------------------------------------
# permittivity per cell (eps weights the mass term)
# --------------------------------------------------------------------------
def _robin_1d_p2_layered(n, omega, eps_e, kappa=1.0):
    """Textbook 1-D quadratic Lagrange FE for v'' + w^2 eps(x) v = 0 with eps
    constant per element, v(0) = 1, v'(1) = -i k w v(1) (dense solve)."""
    h = 1.0 / n
    N = 2 * n + 1
    K = np.zeros((N, N), np.complex128)
    Ke = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / (3 * h)
    Me = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) * h / 30
    for e in range(n):
        idx = [2 * e, 2 * e + 1, 2 * e + 2]
        K[np.ix_(idx, idx)] += Ke - omega ** 2 * eps_e[e] * Me
    K[N - 1, N - 1] += 1j * kappa * omega
    v = np.zeros(N, np.complex128)
    v[0] = 1.0
    v[1:] = np.linalg.solve(K[1:, 1:], -K[1:, 0])

    def ev(x):
        j = np.minimum(np.floor(x / h).astype(int), n - 1)
        t = x / h - j
        return (v[2 * j] * 2 * (t - 0.5) * (t - 1) + v[2 * j + 1] * (-4) * t * (t - 1)
                + v[2 * j + 2] * 2 * t * (t - 0.5))
    return ev


def _max_plane_wave_error(P, S, u, v, seed):
    rng = np.random.default_rng(seed)
    worst = 0.0
    for c in range(P.mesh.n_cell):
        xi = rng.random((3, 2))
        E = fem.evaluate_field(P.mesh, S.dofs, u, c, xi)
        X = fem.physical_point(P.mesh, c, xi)
        worst = max(worst, np.abs(E[:, 1] - v(X[:, 0])).max(), np.abs(E[:, 0]).max())
    return worst


def test_constant_eps_is_the_closed_form_with_scaled_wavenumber():
    """eps = n^2 everywhere: omega^2 eps M is the mass term of wavenumber
    omega n, while the impedance row keeps i kappa omega = i (kappa/n)(omega n):
    the 1-D closed form with (omega n, kappa / n)."""
    n, omega, ref = 8, 4.0, 1.5
    P = W.square_problem(n, 1, 1, omega, bc="planewave", relabel=True, rotate_cells=True)
    P.eps = np.full(P.mesh.n_cell, ref ** 2)
    S = fem.assemble(P)
    u = fem.solve_monolithic(S)
    assert _max_plane_wave_error(P, S, u, _robin_1d_p1(n, omega * ref, kappa=1.0 / ref), 5) < 1e-12


def test_layered_eps_matches_a_1d_solve():
    """eps constant on each column of cells (layers across the propagation
    direction, refractive index 1.516 in some): the 2-D order-2 solution is
    the 1-D quadratic FE solution with per-element eps."""
    n, omega = 8, 6.0
    P = W.square_problem(n, 1, 2, omega, bc="planewave", relabel=True, rotate_cells=True)
    col_eps = np.where(np.arange(n) % 3 == 1, 1.516 ** 2, 1.0)
    X = P.mesh.coords[P.mesh.cells].mean(1)
    P.eps = col_eps[np.floor(X[:, 0] * n).astype(int)]
    S = fem.assemble(P)
    u = fem.solve_monolithic(S)
    assert _max_plane_wave_error(P, S, u, _robin_1d_p2_layered(n, omega, col_eps), 6) < 1e-12
