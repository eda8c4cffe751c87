"""Pins of the oracle adjoint: central finite differences through the
monolithic solve, and the scaling invariant of K."""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as adj
from oracle import fem


def _problem(order, dirichlet_phase=False):
    P = W.square_problem(6, 2, order, 7.0, mu_inv=W.mu_inv_lognormal(36, 0.3, "adj"), relabel=True,
                         rotate_cells=True)
    if dirichlet_phase:      # oblique incidence: the Dirichlet data depend on omega
        P.direction = np.array([0.6, 0.8])
    return P


@pytest.mark.parametrize("order,phase", [(1, False), (2, False), (1, True)])
def test_adjoint_matches_central_differences(order, phase):
    P = _problem(order, phase)
    S = fem.assemble(P)
    u = fem.solve_monolithic(S)
    X = P.mesh.coords[P.mesh.cells].mean(1)
    region = np.flatnonzero((X[:, 0] > 0.3) & (X[:, 0] < 0.7) & (X[:, 1] > 0.3) & (X[:, 1] < 0.7))
    MR = adj.region_mass(P, S, region)
    a = MR @ np.conj(u)
    g_mu, g_w, _ = adj.adjoint_gradients(P, S, u, a)
    rng = np.random.default_rng(0)
    cells = rng.choice(P.mesh.n_cell, 6, replace=False)
    fd = adj.gradients_by_fd(P, MR, cells, h=1e-5)
    scale = np.abs(g_mu).max()
    for c in cells:
        assert abs(g_mu[c] - fd[int(c)]) <= 1e-6 * scale + 1e-7 * abs(fd[int(c)])
    assert abs(g_w - fd["omega"]) <= 1e-6 * max(abs(fd["omega"]), scale)


def test_scaling_invariant():
    """K(s mu, sqrt(s) w, sqrt(s) k) = s K(mu, w, k): u is unchanged, so
    sum_c mu_c dL/dmu_c + (w/2) dL/dw + (k/2) dL/dk = 0.  With kappa=1 fixed
    and the Dirichlet data at x=0 independent of omega this pins the relative
    weights of the curl-curl, mass and boundary terms in the gradient."""
    P = W.square_problem(6, 2, 1, 7.0, mu_inv=W.mu_inv_lognormal(36, 0.3, "inv"))
    S = fem.assemble(P)
    u = fem.solve_monolithic(S)
    MR = adj.region_mass(P, S, np.arange(0, 36, 3))
    a = MR @ np.conj(u)
    g_mu, g_w, lam = adj.adjoint_gradients(P, S, u, a)
    g_k = adj.kappa_gradient(P, S, u, lam)
    total = np.sum(P.mu_inv * g_mu) + 0.5 * P.omega * g_w + 0.5 * P.kappa * g_k
    assert abs(total) <= 1e-9 * (np.abs(P.mu_inv * g_mu).sum() + abs(P.omega * g_w))


def test_adjoint_3d_matches_central_differences():
    """3-D hexes, oblique incidence: the Dirichlet data depend on omega, and
    impedance faces share edges with the Dirichlet face, so the face term of
    dK/domega meets Dirichlet columns (the path a 2-D mesh never exercises)."""
    P = W.cube_problem(3, 1, 5.0, mu_inv=W.mu_inv_lognormal(27, 0.3, "adj3"), relabel=True, rotate_cells=True)
    P.direction = np.array([0.6, 0.8, 0.0])
    S = fem.assemble(P)
    u = fem.solve_monolithic(S)
    X = P.mesh.coords[P.mesh.cells].mean(1)
    region = np.flatnonzero(np.all((X > 0.3) & (X < 0.7), axis=1))
    MR = adj.region_mass(P, S, region)
    g_mu, g_w, _ = adj.adjoint_gradients(P, S, u, MR @ np.conj(u))
    cells = np.array([0, 7, 13, 26])
    fd = adj.gradients_by_fd(P, MR, cells, h=1e-5)
    scale = np.abs(g_mu).max()
    for c in cells:
        assert abs(g_mu[c] - fd[int(c)]) <= 1e-6 * scale + 1e-7 * abs(fd[int(c)])
    assert abs(g_w - fd["omega"]) <= 1e-6 * max(abs(fd["omega"]), scale)


def test_kappa_gradient_matches_central_differences():
    """dL/dkappa from the adjoint against central differences in kappa
    through the monolithic solve (oblique incidence, order 2)."""
    P = _problem(2, True)
    S = fem.assemble(P)
    u = fem.solve_monolithic(S)
    MR = adj.region_mass(P, S, np.arange(0, 36, 2))
    _, _, lam = adj.adjoint_gradients(P, S, u, MR @ np.conj(u))
    g_k = adj.kappa_gradient(P, S, u, lam)

    def L_of(kappa):
        Q = copy.copy(P)
        Q.kappa = kappa
        return adj.loss(fem.solve_monolithic(fem.assemble(Q)), MR)

    h = 1e-5
    fd = (L_of(P.kappa + h) - L_of(P.kappa - h)) / (2 * h)
    assert abs(g_k - fd) <= 1e-6 * abs(fd)
