"""Pins of the oracle's Krylov solver and DDM (Section 3, Eqs. 4-8) against the
monolithic direct solve, dense linear algebra, and the structure of Eq. 7."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import ddm, fem
from oracle.krylov import gmres


def test_gmres_matches_dense_solve():
    rng = np.random.default_rng(0)
    n = 40
    # spectrum in a disc of radius ~4.5 around 10: restarted GMRES converges
    A = np.eye(n) * 10 + 0.5 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, it, hist = gmres(lambda v: A @ v, b, tol=1e-13, restart=15, maxiter=400)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-11 * np.linalg.norm(x)
    assert hist[-1] <= 1e-13 * 1.01
    # exact right preconditioner -> one step
    Ainv = np.linalg.inv(A)
    x1, it1, _ = gmres(lambda v: A @ v, b, precond=lambda v: Ainv @ v, tol=1e-12)
    assert it1 == 1 and np.linalg.norm(A @ x1 - b) <= 1e-11 * np.linalg.norm(b)
    # without restart GMRES terminates in <= n steps
    _, itn, _ = gmres(lambda v: A @ v, b, tol=1e-12, restart=n, maxiter=n)
    assert itn <= n


CASES = [
    ("2d_p1_2x2", lambda: W.square_problem(8, 2, 1, 9.0, relabel=True, rotate_cells=True)),
    ("2d_p1_3x3", lambda: W.square_problem(9, 3, 1, 7.0, mu_inv=W.mu_inv_lognormal(81, 0.3, "d3"))),
    ("2d_p2_2x2", lambda: W.square_problem(8, 2, 2, 11.0, mu_inv=W.mu_inv_lognormal(64, 0.3, "d2"),
                                           relabel=True, rotate_cells=True)),
    ("3d_p1_2x2x2", lambda: W.cube_problem(4, 2, 5.0, relabel=True, rotate_cells=True)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_ddm_fixed_point_equals_monolithic(name, make):
    P = make()
    S = fem.assemble(P)
    u0 = fem.solve_monolithic(S)
    u, info = ddm.solve(P, inner="direct", outer_tol=1e-13)
    assert np.linalg.norm(u - u0) <= 1e-10 * np.linalg.norm(u0)
    assert info["outer_iters"] >= 1
    # continuity across every interface at the fixed point
    D = info["ddm"]
    for p in D.pairs:
        ui = info["us"][p.i][np.searchsorted(D.subs[p.i].dofs, p.dofs)]
        uj = info["us"][p.j][np.searchsorted(D.subs[p.j].dofs, p.dofs)]
        assert np.linalg.norm(p.M @ (ui - uj)) <= 1e-10 * abs(p.M).max() * np.linalg.norm(u0)


def test_single_subdomain_is_monolithic():
    P = W.square_problem(8, 1, 2, 9.0)
    S = fem.assemble(P)
    u, info = ddm.solve(P, inner="direct")
    assert info["ddm"].n_iface == 0
    assert np.linalg.norm(u - fem.solve_monolithic(S)) <= 1e-12 * np.linalg.norm(u)


def test_block_preconditioned_inner_gmres_matches_direct():
    P = W.square_problem(8, 2, 2, 11.0, mu_inv=W.mu_inv_lognormal(64, 0.3, "bp"))
    D = ddm.setup(P)
    ud, infod = ddm.solve(D, inner="direct", outer_tol=1e-12)
    ug, infog = ddm.solve(D, inner="block_gmres", inner_tol=1e-13, outer_tol=1e-12)
    assert np.linalg.norm(ud - ug) <= 1e-10 * np.linalg.norm(ud)
    assert abs(infod["outer_iters"] - infog["outer_iters"]) <= 1
    assert len(infog["inner_iters"]) > 0


def test_block_preconditioner_spectrum():
    """With the exact P of Eq. 7, P^{-1}(P + iB) = I + i P^{-1}B: every
    eigenvalue has real part 1 and at most rank(B) of them differ from 1."""
    P = W.square_problem(4, 2, 1, 6.0)
    D = ddm.setup(P)
    for s in D.subs:
        T = s.Tff.toarray()
        Pm = s.P.toarray()
        Bm = T.imag
        lam = np.linalg.eigvals(np.linalg.solve(Pm, T))
        assert np.allclose(lam.real, 1.0, atol=1e-9)
        r = np.linalg.matrix_rank(Bm)
        assert np.sum(np.abs(lam - 1) > 1e-8) <= r
        assert np.allclose(Pm, Pm.T) and np.abs(T - T.T).max() < 1e-14


def test_jacobi_and_gmres_outer_agree():
    """Eq. 8 by its Jacobi fixed point and by GMRES: same solution, GMRES in
    far fewer sweeps (two strips, no cross points, so Jacobi contracts)."""
    mesh = W.structured_mesh_2d(8, 8, 2, 1)
    pol, d = W.plane_wave_y(2)
    P = W.Problem("strips", mesh, 1, np.ones(mesh.n_cell), 8.0, 1.0, pol, d)
    D = ddm.setup(P)
    ug, ig = ddm.solve(D, outer="gmres", outer_tol=1e-12)
    uj, ij = ddm.solve(D, outer="jacobi", outer_tol=1e-11, outer_maxiter=2000)
    assert np.linalg.norm(ug - uj) <= 1e-8 * np.linalg.norm(ug)
    assert ij["outer_iters"] > ig["outer_iters"]


def test_interface_sizes_small_config():
    D = ddm.setup(W.config("square32_p1"))
    assert D.n_iface == 128                           # 4 interfaces x 2 directions x 16 edges
    assert [len(s.dofs) for s in D.subs] == [544] * 4


def _jacobi_map(D):
    """The sweep map g -> A g of Eq. 8 (zero sources) as a dense matrix."""
    n = D.n_iface
    sv = ddm.subdomain_solver(D, "direct")
    A = np.zeros((n, n), np.complex128)
    for k in range(n):
        e = np.zeros(n, np.complex128)
        e[k] = 1.0
        A[:, k] = ddm.sweep(D, e, None, False, sv)[0]
    return A


def test_fixed_point_is_monolithic_for_other_interface_coefficients():
    """The argument that the DDM fixed point is the monolithic solution does
    not use the value of the interface coefficient: real Robin and a
    Dirichlet-like penalty give the same answer (solved by GMRES on Eq. 8)."""
    P = W.square_problem(8, 2, 1, 9.0, mu_inv=W.mu_inv_lognormal(64, 0.3, "tr"))
    u0 = fem.solve_monolithic(fem.assemble(P))
    for c in (1.0, 50.0, 2.0 + 1.0j):
        D = ddm.setup(P, transmission=c)
        u, _ = ddm.solve(D, inner="direct", outer_tol=1e-13, outer_restart=400, outer_maxiter=400)
        assert np.linalg.norm(u - u0) <= 1e-9 * np.linalg.norm(u0), c


def test_dirichlet_like_interface_conditions_do_not_converge_for_large_omega():
    """Section 3.1: the classical Schwarz decomposition with Dirichlet-like
    interface conditions cannot be expected to converge for large omega,
    while the impedance condition (S = 1) can.  Two strips (no cross points),
    many wavelengths along the interface: the Jacobi map of Eq. 8 contracts
    with the impedance coefficient i kappa omega and has spectral radius >= 1
    with a real coefficient (Robin with a real parameter, or a large real
    penalty: the Dirichlet-like limit)."""
    mesh = W.structured_mesh_2d(16, 8, 2, 1)
    pol, d = W.plane_wave_y(2)
    P = W.Problem("strips", mesh, 1, np.ones(mesh.n_cell), 20.0, 1.0, pol, d)
    rho = {}
    for c in (1j, 1.0, 100.0):
        lam = np.linalg.eigvals(_jacobi_map(ddm.setup(P, transmission=c)))
        rho[c] = np.abs(lam).max()
    assert rho[1j] < 1.0
    assert rho[1.0] >= 1.0 - 1e-9 and rho[100.0] >= 1.0 - 1e-9
    # and the plain fixed-point iteration: converges with impedance, not with the penalty
    _, ij = ddm.solve(ddm.setup(P, transmission=1j), outer="jacobi", outer_tol=1e-8, outer_maxiter=3000)
    _, idl = ddm.solve(ddm.setup(P, transmission=100.0), outer="jacobi", outer_tol=1e-8, outer_maxiter=300)
    assert ij["hist"][-1] < 1e-8
    assert idl["hist"][-1] > 1e-2


def test_full_block_preconditioner_variant():
    """Section 3.2's alternative preconditioner, the full 2x2 block operator.
    With the signs of Eq. 3 its exact inverse is T_ff^{-1}: GMRES stops after
    one step in every subdomain and the DDM reaches the monolithic solution.
    With the off-diagonal signs as printed ([[P, -B], [-B, P]]) it is a
    different real symmetric matrix: GMRES still reaches the same solution,
    in more steps than one."""
    P = W.square_problem(8, 2, 2, 11.0, mu_inv=W.mu_inv_lognormal(64, 0.3, "fb"))
    D = ddm.setup(P)
    u0 = fem.solve_monolithic(D.sys)
    uf, info_f = ddm.solve(D, inner="full_block", inner_tol=1e-12, outer_tol=1e-12)
    assert np.linalg.norm(uf - u0) <= 1e-10 * np.linalg.norm(u0)
    assert {it for _, it in info_f["inner_iters"]} == {1}
    up, info_p = ddm.solve(D, inner="full_block_printed", inner_tol=1e-12, outer_tol=1e-12)
    assert np.linalg.norm(up - u0) <= 1e-9 * np.linalg.norm(u0)
    assert max(it for _, it in info_p["inner_iters"]) > 1
