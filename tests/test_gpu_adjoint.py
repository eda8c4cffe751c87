"""GPU adjoint (thm_adjoint and the autograd wrapper) against the FP64 oracle
adjoint and central finite differences through the GPU solve."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as adj
from oracle import fem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2105_11993_gb300 import build
    build.build()


def _setup(order, oblique=False):
    P = W.square_problem(8, 2, order, 9.0, mu_inv=W.mu_inv_lognormal(64, 0.3, "gadj"), relabel=True,
                         rotate_cells=True)
    if oblique:
        P.direction = np.array([0.6, 0.8])
    S = fem.assemble(P)
    X = P.mesh.coords[P.mesh.cells].mean(1)
    region = np.flatnonzero((X[:, 0] > 0.3) & (X[:, 0] < 0.7) & (X[:, 1] > 0.3) & (X[:, 1] < 0.7))
    MR = adj.region_mass(P, S, region)
    return P, S, MR


@pytest.mark.parametrize("order,oblique", [(1, False), (2, False), (1, True)])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_adjoint_matches_oracle_adjoint(order, oblique, mode):
    import paper_2105_11993_gb300 as thm
    P, S, MR = _setup(order, oblique)
    mesh = thm.Mesh.from_workload(P.mesh, P.order)
    sysg = thm.System(mesh, P.mu_inv, P.omega, P.kappa, P.pol, P.direction)
    u, _ = sysg.solve(mode=mode, rtol=1e-12 if mode == "fp64" else 1e-11)
    uh = u.cpu().numpy()
    a = MR @ np.conj(uh)
    g_mu, g_w, st = sysg.adjoint(u, torch.tensor(a, device="cuda"), mode=mode, rtol=1e-12 if mode == "fp64" else 1e-11)
    g_ref, gw_ref, _ = adj.adjoint_gradients(P, S, fem.solve_monolithic(S), MR @ np.conj(fem.solve_monolithic(S)))
    g_mu = g_mu.cpu().numpy()
    assert np.linalg.norm(g_mu - g_ref) <= 1e-8 * np.linalg.norm(g_ref)
    assert abs(g_w - gw_ref) <= 1e-8 * abs(gw_ref)


def test_adjoint_vs_central_differences_and_autograd():
    """Gradient check: dL/dmu^{-1} and dL/domega against central differences
    (h = 1e-4) of the GPU solve itself, to 1e-5 relative."""
    import paper_2105_11993_gb300 as thm
    from paper_2105_11993_gb300 import autograd as ag
    P, S, MR = _setup(2)
    mesh = thm.Mesh.from_workload(P.mesh, P.order)
    MRt = torch.tensor(MR.toarray(), dtype=torch.complex128, device="cuda")
    mu = torch.tensor(P.mu_inv, device="cuda", requires_grad=True)
    om = torch.tensor(P.omega, dtype=torch.float64, requires_grad=True)

    def L_of(mu_t, omega):
        u = ag.solve(mesh, mu_t, omega, P.kappa, P.pol, P.direction, rtol=1e-13)
        return torch.real(torch.vdot(u, MRt @ u))

    L = L_of(mu, om)
    L.backward()
    g_mu = mu.grad.cpu().numpy()
    g_w = float(om.grad)
    rng = np.random.default_rng(5)
    h = 1e-4
    scale = np.abs(g_mu).max()
    with torch.no_grad():
        for c in rng.choice(P.mesh.n_cell, 5, replace=False):
            mp = mu.detach().clone(); mp[c] += h
            mm = mu.detach().clone(); mm[c] -= h
            fd = (float(L_of(mp, P.omega)) - float(L_of(mm, P.omega))) / (2 * h)
            assert abs(g_mu[c] - fd) <= 1e-5 * max(abs(fd), 1e-3 * scale)
        fdw = (float(L_of(mu.detach(), P.omega + h)) - float(L_of(mu.detach(), P.omega - h))) / (2 * h)
        assert abs(g_w - fdw) <= 1e-5 * abs(fdw)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_adjoint_3d_matches_oracle_adjoint(mode):
    """3-D hexes over 2x2x2 subdomains, oblique incidence (omega-dependent
    Dirichlet data on a face that borders impedance faces)."""
    import paper_2105_11993_gb300 as thm
    P = W.cube_problem(4, 2, 6.0, mu_inv=W.mu_inv_lognormal(64, 0.3, "gadj3"), relabel=True, rotate_cells=True)
    P.direction = np.array([0.6, 0.8, 0.0])
    S = fem.assemble(P)
    X = P.mesh.coords[P.mesh.cells].mean(1)
    region = np.flatnonzero(np.all((X > 0.2) & (X < 0.8), axis=1))
    MR = adj.region_mass(P, S, region)
    mesh = thm.Mesh.from_workload(P.mesh, P.order)
    sysg = thm.System(mesh, P.mu_inv, P.omega, P.kappa, P.pol, P.direction)
    tol = 1e-12 if mode == "fp64" else 1e-11
    u, _ = sysg.solve(mode=mode, rtol=tol)
    a = MR @ np.conj(u.cpu().numpy())
    g_mu, g_w, _ = sysg.adjoint(u, torch.tensor(a, device="cuda"), mode=mode, rtol=tol)
    u0 = fem.solve_monolithic(S)
    g_ref, gw_ref, _ = adj.adjoint_gradients(P, S, u0, MR @ np.conj(u0))
    assert np.linalg.norm(g_mu.cpu().numpy() - g_ref) <= 1e-8 * np.linalg.norm(g_ref)
    assert abs(g_w - gw_ref) <= 1e-8 * abs(gw_ref)


def _cube12():
    """The 12^3 copy of the 48^3 differentiation workload: 3x3x3 subdomains,
    smooth random mu^{-1} (the same generator), oblique incidence, the loss
    over the central 2^3 cells (the 8^3 of 48^3 scaled)."""
    n = 12
    mu = W.mu_inv_smooth_3d(n, 0.3, 3.0, "adj12/mu")
    P = W.cube_problem(n, 3, 3 * np.pi, mu_inv=mu)
    P.direction = np.array([0.6, 0.8, 0.0])
    X = P.mesh.coords[P.mesh.cells].mean(1)
    region = np.flatnonzero(np.all((X >= 5 / n) & (X < 7 / n), axis=1))
    return P, region


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_adjoint_12cube_matches_oracle_adjoint(mode):
    """The 12^3 copy of the differentiation workload: every dL/dmu^{-1}, dL/domega
    and dL/dkappa against the FP64 CPU oracle adjoint."""
    import paper_2105_11993_gb300 as thm
    P, region = _cube12()
    S = fem.assemble(P)
    MR = adj.region_mass(P, S, region)
    mesh = thm.Mesh.from_workload(P.mesh, P.order)
    sysg = thm.System(mesh, P.mu_inv, P.omega, P.kappa, P.pol, P.direction)
    tol = 1e-12 if mode == "fp64" else 1e-11
    u, _ = sysg.solve(mode=mode, rtol=tol)
    a = MR @ np.conj(u.cpu().numpy())
    g_mu, g_w, g_k, _ = sysg.adjoint(u, torch.tensor(a, device="cuda"), mode=mode, rtol=tol, with_kappa=True)
    u0 = fem.solve_monolithic(S)
    g_ref, gw_ref, lam = adj.adjoint_gradients(P, S, u0, MR @ np.conj(u0))
    gk_ref = adj.kappa_gradient(P, S, u0, lam)
    assert np.linalg.norm(g_mu.cpu().numpy() - g_ref) <= 1e-8 * np.linalg.norm(g_ref)
    assert abs(g_w - gw_ref) <= 1e-8 * abs(gw_ref)
    assert abs(g_k - gk_ref) <= 1e-8 * abs(gk_ref)


def test_adjoint_3d_vs_central_differences():
    """3-D (12^3 hexes, 3x3x3 subdomains, smooth random mu^{-1} as in the
    48^3 differentiation workload, oblique incidence): gradients from one
    adjoint solve against central differences (h = 1e-4) of the GPU solve
    itself, to 1e-5 relative, at 20 random cells and in omega."""
    import paper_2105_11993_gb300 as thm
    P, region = _cube12()
    S = fem.assemble(P)
    MR = torch.tensor(adj.region_mass(P, S, region).toarray(), dtype=torch.complex128, device="cuda")
    mesh = thm.Mesh.from_workload(P.mesh, P.order)

    def solve(mu_c, omega):
        s = thm.System(mesh, mu_c, omega, P.kappa, P.pol, P.direction)
        u, _ = s.solve(mode="mixed", rtol=1e-13)
        return s, u

    s, u = solve(P.mu_inv, P.omega)
    a = MR @ torch.conj(u)
    g_mu, g_w, _ = s.adjoint(u, a, mode="mixed", rtol=1e-13)
    g_mu = g_mu.cpu().numpy()
    L = lambda uu: float(torch.real(torch.vdot(uu, MR @ uu)))
    h = 1e-4
    scale = np.abs(g_mu).max()
    for c in np.random.default_rng(7).choice(P.mesh.n_cell, 20, replace=False):
        mp = P.mu_inv.copy(); mp[c] += h
        mm = P.mu_inv.copy(); mm[c] -= h
        fd = (L(solve(mp, P.omega)[1]) - L(solve(mm, P.omega)[1])) / (2 * h)
        assert abs(g_mu[c] - fd) <= 1e-5 * max(abs(fd), 1e-3 * scale), (c, g_mu[c], fd)
    fdw = (L(solve(P.mu_inv, P.omega + h)[1]) - L(solve(P.mu_inv, P.omega - h)[1])) / (2 * h)
    assert abs(g_w - fdw) <= 1e-5 * abs(fdw), (g_w, fdw)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_given_dirichlet_data_solve_adjoint_and_scaling_invariant(mode):
    """thm_assemble_dirichlet: arbitrary Dirichlet values (not a plane wave)
    against the oracle's monolithic solve with the same values; the adjoint of
    that system (data independent of omega and kappa) against the oracle
    adjoint, dL/dkappa included; and the scaling invariant
    sum_c mu_c dL/dmu_c + (omega/2) dL/domega + (kappa/2) dL/dkappa = 0
    on the GPU gradients."""
    import paper_2105_11993_gb300 as thm
    P = W.square_problem(12, 2, 2, 9.0, mu_inv=W.mu_inv_lognormal(144, 0.3, "given-gpu"), relabel=True,
                         rotate_cells=True)
    S = fem.assemble(P)
    mesh = thm.Mesh.from_workload(P.mesh, P.order)
    ids = mesh.dirichlet_dofs()
    assert np.array_equal(ids, np.flatnonzero(S.is_dir))
    r = np.random.default_rng(17)
    d = r.standard_normal(len(ids)) + 1j * r.standard_normal(len(ids))
    Sg = fem.with_dirichlet(S, d)
    u0 = fem.solve_monolithic(Sg)
    tol = 1e-12 if mode == "fp64" else 1e-11
    for on_device in (False, True):
        sysg = thm.System(mesh, P.mu_inv, P.omega, P.kappa, stream=None,
                          dirichlet=torch.tensor(d, device="cuda") if on_device else d)
        u, st = sysg.solve(mode=mode, rtol=tol)
        uh = u.cpu().numpy()
        assert np.array_equal(uh[ids], d)
        assert np.linalg.norm(uh - u0) <= (1e-8 if mode == "fp64" else 1e-6) * np.linalg.norm(u0)
    X = P.mesh.coords[P.mesh.cells].mean(1)
    region = np.flatnonzero((X[:, 0] > 0.3) & (X[:, 0] < 0.7) & (X[:, 1] > 0.3) & (X[:, 1] < 0.7))
    MR = adj.region_mass(P, S, region)
    g_mu, g_w, g_k, _ = sysg.adjoint(u, torch.tensor(MR @ np.conj(uh), device="cuda"), mode=mode, rtol=tol,
                                     with_kappa=True)
    g_mu = g_mu.cpu().numpy()
    # oracle: data independent of omega (direction (1,0): zero phase on x = 0)
    assert np.allclose(adj.dirichlet_domega(P, Sg), 0)
    g_ref, gw_ref, lam = adj.adjoint_gradients(P, Sg, u0, MR @ np.conj(u0))
    gk_ref = adj.kappa_gradient(P, Sg, u0, lam)
    assert np.linalg.norm(g_mu - g_ref) <= 1e-8 * np.linalg.norm(g_ref)
    assert abs(g_w - gw_ref) <= 1e-8 * abs(gw_ref)
    assert abs(g_k - gk_ref) <= 1e-8 * abs(gk_ref)
    total = np.sum(P.mu_inv * g_mu) + 0.5 * P.omega * g_w + 0.5 * P.kappa * g_k
    assert abs(total) <= 1e-9 * (np.abs(P.mu_inv * g_mu).sum() + abs(P.omega * g_w))
