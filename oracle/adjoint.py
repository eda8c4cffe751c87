"""Oracle adjoint of the discrete THM solve (no counterpart in the paper).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  FP64, monolithic.

For a real loss L(u) of the discrete field u = [u_F; u_D] with
K_FF u_F = -K_FD u_D and parameters p (per-cell mu^{-1}, omega):

    dL/dp = -2 Re( lambda^T [ (dK/dp) u + K_{:,D} du_D/dp ] ) + 2 Re( a_D . du_D/dp )

with a = dL/du (Wirtinger, a = M_R conj(u) for L = u^H M_R u) and
K_FF lambda = a_F (K is complex symmetric, so K^T = K and the adjoint solve is
the forward solve with a different right-hand side); lambda is zero on the
Dirichlet DOFs.  dK/dmu_c = A_c (the cell's curl-curl matrix; the boundary
term does not contain mu^{-1}), dK/domega = -2 omega M + i kappa M_Gamma.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem


def region_mass(problem, sys_: fem.System, cells) -> sp.csr_matrix:
    """M_R: the mass matrix assembled over the given cells only."""
    _, M = fem.assemble_volume(problem.mesh, sys_.dofs, np.ones(problem.mesh.n_cell), problem.omega, cells)
    return M.tocsr()


def loss(u, MR) -> float:
    """L = u^H M_R u (real because M_R is real symmetric)."""
    return float(np.real(np.vdot(u, MR @ u)))


def dirichlet_domega(problem, sys_: fem.System) -> np.ndarray:
    """d u_D / d omega on all DOFs (0 on free DOFs), by differentiating the
    tangential moments under the quadrature: d/dw exp(-i w d.x) = -i d.x exp(-i w d.x)."""
    mesh = problem.mesh
    dofs = sys_.dofs
    out = np.zeros(dofs.n_dof, np.complex128)
    x, w = fem.gauss01(16)
    le = fem.LOCAL_EDGES[2]
    seen = set()
    for f, tag in zip(mesh.bfaces, mesh.btag):
        if tag != 1:
            continue
        pairs = [tuple(f)] if mesh.dim == 2 else [(f[a], f[b]) for a, b in le]
        for a, b in pairs:
            e = int(dofs.edge_id([a], [b])[0])
            if e in seen:
                continue
            seen.add(e)
            lo, hi = dofs.edges[e]
            t = mesh.coords[hi] - mesh.coords[lo]
            ell = np.sqrt(t @ t)
            pts = mesh.coords[lo][None, :] + x[:, None] * t[None, :]
            phase = pts @ problem.direction
            Et = fem.e_inc(pts, problem.omega, problem.pol, problem.direction) @ (t / ell)
            dEt = -1j * phase * Et
            gd = dofs.edge_dofs(np.array([e]))[0]
            out[gd[0]] = np.sum(w * dEt) * ell
            if dofs.order == 2:
                out[gd[1]] = 3.0 * ell * np.sum(w * dEt * (1.0 - 2.0 * x))
    return out


def adjoint_gradients(problem, sys_: fem.System, u: np.ndarray, a: np.ndarray):
    """(dL/dmu^{-1} per cell [n_cell], dL/domega) for dL/du = a."""
    mesh = problem.mesh
    free = sys_.free
    Kff = sys_.K[free][:, free].tocsc()
    lam = np.zeros_like(u)
    lam[free] = spla.spsolve(Kff.T, a[free])        # K^T = K; the transpose states the definition
    A_loc, M_loc = fem.cell_matrices(mesh, problem.order)
    cd = sys_.dofs.cell_dofs
    cs = sys_.dofs.cell_signs.astype(np.float64)
    lc = lam[cd] * cs
    uc = u[cd] * cs
    g_mu = -2.0 * np.real(np.einsum("ci,cij,cj->c", lc, A_loc, uc))
    dK_dw = (-2.0 * problem.omega * sys_.M).astype(np.complex128) + 1j * problem.kappa * sys_.Mg
    duD = dirichlet_domega(problem, sys_)
    g_w = -2.0 * np.real(lam @ (dK_dw @ u) + lam @ (sys_.K @ duD)) + 2.0 * np.real(a @ duD)
    return g_mu, float(g_w), lam


def kappa_gradient(problem, sys_: fem.System, u: np.ndarray, lam: np.ndarray) -> float:
    """dL/dkappa = -2 Re(lambda^T (dK/dkappa) u) with dK/dkappa = i omega M_Gamma
    (the impedance term of Eq. 1 is the only place kappa enters; the Dirichlet
    data do not depend on it)."""
    return float(-2.0 * np.real(lam @ (1j * problem.omega * (sys_.Mg @ u))))


def gradients_by_fd(problem, MR, cells_to_check, h=1e-6, d_omega=True):
    """Central finite differences of L through the monolithic solve."""
    import copy

    def L_of(P):
        S = fem.assemble(P)
        return loss(fem.solve_monolithic(S), MR)

    out = {}
    for c in cells_to_check:
        Pp = copy.copy(problem); Pp.mu_inv = problem.mu_inv.copy(); Pp.mu_inv[c] += h
        Pm = copy.copy(problem); Pm.mu_inv = problem.mu_inv.copy(); Pm.mu_inv[c] -= h
        out[int(c)] = (L_of(Pp) - L_of(Pm)) / (2 * h)
    if d_omega:
        Pp = copy.copy(problem); Pp.omega = problem.omega + h
        Pm = copy.copy(problem); Pm.omega = problem.omega - h
        out["omega"] = (L_of(Pp) - L_of(Pm)) / (2 * h)
    return out
