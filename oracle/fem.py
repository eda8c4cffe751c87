"""Oracle FEM: Nedelec discretisation of the THM system (Section 2, Eqs. 1-3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain, slow, FP64.

Definitions used here (stated once, pinned by tests/test_oracle_fem.py):

* Global edges are the distinct vertex pairs of the cells' local edges; edge
  ids follow the lexicographic order of (smaller vertex id, larger vertex id).
  The global direction of an edge runs from its smaller to its larger vertex
  id; a cell's local edge (a -> b) has orientation sign +1 iff id(a) < id(b).
* Cells list their corners in tensor order: 2-D (00,10,01,11), 3-D
  v = i + 2j + 4k.  Local coordinates xi (v0->v1), eta (v0->v2), zeta (v0->v4).
* Order-1 DOF e = the tangential moment of the field along global edge e.
* Order-2 (2-D) adds per edge the gradient function grad(q(s) * ramp),
  q(t) = t(1-t), which is even under edge reversal (no sign), and per cell the
  four bubbles (q(eta)(1-xi),0), (q(eta)xi,0), (0,q(xi)(1-eta)), (0,q(xi)eta).
  Numbering: Whitney of edge e -> 2e, gradient of edge e -> 2e+1,
  bubble k of cell c -> 2E + 4c + k.  (Hierarchical de-Rham-compatible bases
  as in the Zaglmayr reference cited in Section 2.)
* Reference functions map by the covariant Piola map phi = J^{-T} phi_hat,
  curl by the contravariant one (1/det J) J curl_hat (a scalar 1/det J in 2-D).
* An optional relative permittivity eps per cell weights the mass term,
  sum_c eps_c M_c (Eq. 1 is printed with eps = 1; the paper's Example 1
  describes its centre block by a refractive index n, eps = n^2).
* K = mu^{-1} A - omega^2 M + i kappa omega M_Gamma_inf, i.e. Eq. 3's
  K = A - w^2 M + iB with B = kappa*omega*M_Gamma_inf: the coefficient of the
  boundary integral is taken from the strong form's impedance condition
  (Eq. 1), not from the garbled mu^{-1} of Eq. 2.  Dirichlet DOFs (tag 1
  faces) are eliminated strongly with the tangential moments of E_inc.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

LOCAL_EDGES = {
    2: np.array([(0, 1), (2, 3), (0, 2), (1, 3)], dtype=np.int64),
    3: np.array([(0, 1), (2, 3), (4, 5), (6, 7), (0, 2), (1, 3), (4, 6), (5, 7),
                 (0, 4), (1, 5), (2, 6), (3, 7)], dtype=np.int64),
}
# hex faces, each in face-local tensor order
LOCAL_FACES_3D = np.array([(0, 2, 4, 6), (1, 3, 5, 7), (0, 1, 4, 5), (2, 3, 6, 7),
                           (0, 1, 2, 3), (4, 5, 6, 7)], dtype=np.int64)


def gauss01(n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


# ---------------------------------------------------------------------------
# Numbering
# ---------------------------------------------------------------------------
@dataclass
class Dofs:
    dim: int
    order: int
    edges: np.ndarray        # [E,2] (lo, hi) vertex ids, sorted lexicographically
    edge_of_cell: np.ndarray  # [nc, n_local_edges]
    edge_sign: np.ndarray     # [nc, n_local_edges] int8
    cell_dofs: np.ndarray     # [nc, dpc] int64
    cell_signs: np.ndarray    # [nc, dpc] int8
    n_dof: int

    @property
    def n_edge(self):
        return self.edges.shape[0]

    def edge_id(self, a, b) -> np.ndarray:
        """Global edge ids of vertex pairs (a, b) (any order); -1 if absent."""
        a = np.asarray(a, np.int64); b = np.asarray(b, np.int64)
        lo = np.minimum(a, b); hi = np.maximum(a, b)
        nv = int(self.edges.max()) + 1
        keys = self.edges[:, 0] * nv + self.edges[:, 1]
        q = lo * nv + hi
        pos = np.searchsorted(keys, q)
        pos = np.clip(pos, 0, len(keys) - 1)
        return np.where(keys[pos] == q, pos, -1)

    def edge_dofs(self, e: np.ndarray) -> np.ndarray:
        """[len(e), dofs per edge] global DOFs living on edges e."""
        e = np.asarray(e, np.int64)
        if self.order == 1:
            return e[:, None]
        return np.stack([2 * e, 2 * e + 1], 1)


def number_dofs(cells: np.ndarray, dim: int, order: int) -> Dofs:
    le = LOCAL_EDGES[dim]
    a = cells[:, le[:, 0]]
    b = cells[:, le[:, 1]]
    lo = np.minimum(a, b).ravel()
    hi = np.maximum(a, b).ravel()
    keys = np.stack([lo, hi], 1)
    edges, inv = np.unique(keys, axis=0, return_inverse=True)
    eoc = inv.reshape(a.shape).astype(np.int64)
    esign = np.where(a < b, 1, -1).astype(np.int8)
    nc = cells.shape[0]
    E = edges.shape[0]
    if order == 1:
        return Dofs(dim, order, edges, eoc, esign, eoc.copy(), esign.copy(), E)
    if order == 2 and dim == 2:
        dofs = np.empty((nc, 12), np.int64)
        signs = np.ones((nc, 12), np.int8)
        for k in range(4):
            dofs[:, 2 * k] = 2 * eoc[:, k]
            signs[:, 2 * k] = esign[:, k]
            dofs[:, 2 * k + 1] = 2 * eoc[:, k] + 1
        for k in range(4):
            dofs[:, 8 + k] = 2 * E + 4 * np.arange(nc) + k
        return Dofs(dim, order, edges, eoc, esign, dofs, signs, 2 * E + 4 * nc)
    raise NotImplementedError(f"dim={dim} order={order}")


# ---------------------------------------------------------------------------
# Reference bases: values [nq, nb, dim] and curls (2-D: [nq, nb]; 3-D: [nq, nb, 3])
# ---------------------------------------------------------------------------
def _q(t):
    return t * (1.0 - t)


def _dq(t):
    return 1.0 - 2.0 * t


def ref_basis_2d(order: int, xi: np.ndarray, eta: np.ndarray):
    z = np.zeros_like(xi)
    one = np.ones_like(xi)
    # Whitney functions of local edges 0..3 and their reference curls
    W = [((1 - eta), z), (eta, z), (z, 1 - xi), (z, xi)]
    Wc = [one, -one, -one, one]
    if order == 1:
        vals = [W[0], W[1], W[2], W[3]]
        curls = Wc
    else:
        G = [(_dq(xi) * (1 - eta), -_q(xi)),
             (_dq(xi) * eta, _q(xi)),
             (-_q(eta), _dq(eta) * (1 - xi)),
             (_q(eta), _dq(eta) * xi)]
        Bv = [(_q(eta) * (1 - xi), z), (_q(eta) * xi, z), (z, _q(xi) * (1 - eta)), (z, _q(xi) * eta)]
        Bc = [-_dq(eta) * (1 - xi), -_dq(eta) * xi, _dq(xi) * (1 - eta), _dq(xi) * eta]
        vals, curls = [], []
        for k in range(4):
            vals += [W[k], G[k]]
            curls += [Wc[k], z]
        vals += Bv
        curls += Bc
    V = np.stack([np.stack(v, -1) for v in vals], 1)      # [nq, nb, 2]
    C = np.stack(curls, 1)                                # [nq, nb]
    return V, C


def ref_basis_3d(xi, eta, zeta):
    """Order-1 hex: 12 Whitney functions, local edges in LOCAL_EDGES[3] order."""
    L = lambda t, s: (1 - t) if s == 0 else t
    dL = lambda s: -1.0 if s == 0 else 1.0
    z = np.zeros_like(xi)
    vals, curls = [], []
    for (e0, e1) in [(0, 0), (1, 0), (0, 1), (1, 1)]:            # xi-edges at (eta, zeta)
        f = L(eta, e0) * L(zeta, e1)
        vals.append(np.stack([f, z, z], -1))
        curls.append(np.stack([z, L(eta, e0) * dL(e1), -dL(e0) * L(zeta, e1)], -1))
    for (e0, e1) in [(0, 0), (1, 0), (0, 1), (1, 1)]:            # eta-edges at (xi, zeta)
        g = L(xi, e0) * L(zeta, e1)
        vals.append(np.stack([z, g, z], -1))
        curls.append(np.stack([-L(xi, e0) * dL(e1), z, dL(e0) * L(zeta, e1)], -1))
    for (e0, e1) in [(0, 0), (1, 0), (0, 1), (1, 1)]:            # zeta-edges at (xi, eta)
        k = L(xi, e0) * L(eta, e1)
        vals.append(np.stack([z, z, k], -1))
        curls.append(np.stack([L(xi, e0) * dL(e1), -dL(e0) * L(eta, e1), z], -1))
    return np.stack(vals, 1), np.stack(curls, 1)


def cell_jacobian(coords: np.ndarray, cell: np.ndarray, dim: int) -> np.ndarray:
    v0 = coords[cell[0]]
    cols = [coords[cell[1]] - v0, coords[cell[2]] - v0]
    if dim == 3:
        cols.append(coords[cell[4]] - v0)
    return np.stack(cols, 1)      # J[:, a] = d x / d xi_a


def element_matrices(dim: int, order: int, J: np.ndarray, nq: int = 5):
    """Local curl-curl A (mu^{-1}=1) and mass M by Gauss quadrature on the
    reference cell, for an affine cell with Jacobian J (Section 2, (A), (M))."""
    x, w = gauss01(nq)
    detJ = np.linalg.det(J)
    JinvT = np.linalg.inv(J).T
    if dim == 2:
        XI, ETA = np.meshgrid(x, x, indexing="ij")
        W = np.outer(w, w).ravel()
        V, C = ref_basis_2d(order, XI.ravel(), ETA.ravel())
        phys = np.einsum("ab,qnb->qna", JinvT, V)
        curl = C / detJ
        A = np.einsum("q,qn,qm->nm", W * abs(detJ), curl, curl)
    else:
        XI, ETA, ZETA = np.meshgrid(x, x, x, indexing="ij")
        W = np.einsum("i,j,k->ijk", w, w, w).ravel()
        V, C = ref_basis_3d(XI.ravel(), ETA.ravel(), ZETA.ravel())
        phys = np.einsum("ab,qnb->qna", JinvT, V)
        curl = np.einsum("ab,qnb->qna", J, C) / detJ
        A = np.einsum("q,qna,qma->nm", W * abs(detJ), curl, curl)
    M = np.einsum("q,qna,qma->nm", W * abs(detJ), phys, phys)
    return A, M


# ---------------------------------------------------------------------------
# Faces: tangential-trace mass of the lower-dimensional element on a face
# ---------------------------------------------------------------------------
def face_dofs_and_mass(dofs: Dofs, coords: np.ndarray, face: np.ndarray, nq: int = 6):
    """Global DOFs, signs and tangential mass  int_F gamma^T phi_a . gamma^T phi_b
    of one boundary/interface face.  2-D: face = (a, b) edge; 3-D: quad in
    face-local tensor order.  The traces of the volume basis on the face are
    the face's own Nedelec basis (tangential conformity)."""
    face = np.asarray(face, np.int64)
    x, w = gauss01(nq)
    if dofs.dim == 2:
        a, b = face
        t = coords[b] - coords[a]
        G = float(t @ t)                      # metric of the 1-D map
        e = int(dofs.edge_id([a], [b])[0])
        sgn = 1 if a < b else -1
        if dofs.order == 1:
            vals = np.ones((len(x), 1))
            gd = np.array([e]); sg = np.array([sgn])
        else:
            # Whitney trace (const) and gradient trace q'(s) in the face's
            # parameter s (a -> b); the gradient DOF carries no sign, and
            # q'(1-s) = -q'(s) matches the opposite direction -t exactly.
            s = x
            vals = np.stack([np.ones_like(s), _dq(s)], 1)
            gd = np.array([2 * e, 2 * e + 1]); sg = np.array([sgn, 1])
        Mloc = np.einsum("q,qa,qb->ab", w, vals, vals) / G * np.sqrt(G)
        return gd, sg, Mloc
    # 3-D quad face
    J = np.stack([coords[face[1]] - coords[face[0]], coords[face[2]] - coords[face[0]]], 1)  # 3x2
    G = J.T @ J
    Ginv = np.linalg.inv(G)
    XI, ETA = np.meshgrid(x, x, indexing="ij")
    W = np.outer(w, w).ravel()
    V, _ = ref_basis_2d(1, XI.ravel(), ETA.ravel())       # face Whitney basis
    Mloc = np.einsum("q,qna,ab,qmb->nm", W * np.sqrt(np.linalg.det(G)), V, Ginv, V)
    le = LOCAL_EDGES[2]
    va = face[le[:, 0]]; vb = face[le[:, 1]]
    gd = dofs.edge_id(va, vb)
    sg = np.where(va < vb, 1, -1)
    return gd, sg, Mloc


def cell_faces(mesh) -> tuple[np.ndarray, np.ndarray]:
    """All (cell, face-vertex-list) pairs: 2-D faces are the cells' edges,
    3-D faces the hexes' six quads.  Returns (face_vertices [nf, 2|4] in the
    face-local order of the *first* cell listing it, cells_of_face [nf, 2],
    -1 for a boundary face)."""
    if mesh.dim == 2:
        le = LOCAL_EDGES[2]
        fv = mesh.cells[:, le]                    # [nc, 4, 2]
    else:
        fv = mesh.cells[:, LOCAL_FACES_3D]        # [nc, 6, 4]
    nc, nf_loc, k = fv.shape
    flat = fv.reshape(-1, k)
    key = np.sort(flat, 1)
    uniq, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    owner = np.repeat(np.arange(nc), nf_loc)
    cells_of = -np.ones((uniq.shape[0], 2), np.int64)
    for idx in range(flat.shape[0]):
        f = inv[idx]
        if cells_of[f, 0] < 0:
            cells_of[f, 0] = owner[idx]
        else:
            cells_of[f, 1] = owner[idx]
    return flat[first], cells_of


# ---------------------------------------------------------------------------
# Incident field and Dirichlet data
# ---------------------------------------------------------------------------
def e_inc(points: np.ndarray, omega: float, pol: np.ndarray, direction: np.ndarray) -> np.ndarray:
    """E_inc(x) = pol * exp(-i omega d.x)  (time factor e^{i omega tau}, Section 2)."""
    phase = np.exp(-1j * omega * (points @ direction))
    return phase[:, None] * pol[None, :]


def edge_moments(dofs: Dofs, coords, e: int, omega, pol, direction, nq: int = 16):
    """Tangential moments of E_inc on global edge e (global direction lo->hi):
    order 1: int_e E.t ds;  order 2 adds 3 l int_0^1 (E.t)(s) q'(s) ds, the
    coefficient of the gradient function (L2 projection onto the trace space)."""
    lo, hi = dofs.edges[e]
    x, w = gauss01(nq)
    t = coords[hi] - coords[lo]
    ell = np.sqrt(t @ t)
    pts = coords[lo][None, :] + x[:, None] * t[None, :]
    Et = e_inc(pts, omega, pol, direction) @ (t / ell)
    m0 = np.sum(w * Et) * ell
    if dofs.order == 1:
        return np.array([m0])
    m1 = 3.0 * ell * np.sum(w * Et * _dq(x))
    return np.array([m0, m1])


def dirichlet_data(mesh, dofs: Dofs, omega, pol, direction):
    """(mask of Dirichlet DOFs, u_D values on all DOFs (0 elsewhere))."""
    is_d = np.zeros(dofs.n_dof, bool)
    uD = np.zeros(dofs.n_dof, np.complex128)
    le = LOCAL_EDGES[2]
    for f, tag in zip(mesh.bfaces, mesh.btag):
        if tag != 1:
            continue
        if mesh.dim == 2:
            pairs = [tuple(f)]
        else:
            pairs = [(f[a], f[b]) for a, b in le]
        for a, b in pairs:
            e = int(dofs.edge_id([a], [b])[0])
            gd = dofs.edge_dofs(np.array([e]))[0]
            is_d[gd] = True
            uD[gd] = edge_moments(dofs, mesh.coords, e, omega, pol, direction)
    return is_d, uD


# ---------------------------------------------------------------------------
# Assembly
# ---------------------------------------------------------------------------
def _unique_jacobians(mesh):
    Js = np.stack([cell_jacobian(mesh.coords, c, mesh.dim) for c in mesh.cells])
    scale = np.abs(Js).max()
    keyarr = np.round(Js / scale * 1e12).astype(np.int64).reshape(len(Js), -1)
    uniq, first, inv = np.unique(keyarr, axis=0, return_index=True, return_inverse=True)
    return Js[first], inv


def cell_matrices(mesh, order):
    """Per-cell local A (mu^{-1}=1) and M: arrays [nc, nb, nb] (local basis)."""
    Jus, inv = _unique_jacobians(mesh)
    mats = [element_matrices(mesh.dim, order, J) for J in Jus]
    A = np.stack([m[0] for m in mats])[inv]
    M = np.stack([m[1] for m in mats])[inv]
    return A, M


def assemble_volume(mesh, dofs: Dofs, mu_inv, omega, cells=None, eps=None):
    """Signed global (mu^{-1} A, M) from the given cells (default all); with
    eps (relative permittivity per cell) the mass is sum_c eps_c M_c."""
    A, M = cell_matrices(mesh, dofs.order)
    if cells is None:
        cells = np.arange(mesh.n_cell)
    cd = dofs.cell_dofs[cells]
    cs = dofs.cell_signs[cells].astype(np.float64)
    ss = cs[:, :, None] * cs[:, None, :]
    Av = (mu_inv[cells][:, None, None] * A[cells]) * ss
    Mv = M[cells] * ss
    if eps is not None:
        Mv = eps[cells][:, None, None] * Mv
    rows = np.repeat(cd, cd.shape[1], axis=1).ravel()
    cols = np.tile(cd, (1, cd.shape[1])).ravel()
    n = dofs.n_dof
    Ag = sp.csr_matrix((Av.ravel(), (rows, cols)), shape=(n, n))
    Mg = sp.csr_matrix((Mv.ravel(), (rows, cols)), shape=(n, n))
    return Ag, Mg


def assemble_faces(mesh, dofs: Dofs, faces) -> sp.csr_matrix:
    """Sum of tangential face masses over the listed faces."""
    rows, cols, vals = [], [], []
    for f in faces:
        gd, sg, Ml = face_dofs_and_mass(dofs, mesh.coords, f)
        S = np.outer(sg, sg) * Ml
        rows.append(np.repeat(gd, len(gd))); cols.append(np.tile(gd, len(gd))); vals.append(S.ravel())
    n = dofs.n_dof
    if not rows:
        return sp.csr_matrix((n, n))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


@dataclass
class System:
    dofs: Dofs
    K: sp.csr_matrix          # complex, all DOFs
    A: sp.csr_matrix          # mu^{-1}-weighted curl-curl
    M: sp.csr_matrix          # mass (eps-weighted when the problem has a permittivity field)
    Mg: sp.csr_matrix         # impedance boundary mass (Gamma^inf)
    is_dir: np.ndarray
    uD: np.ndarray
    free: np.ndarray          # indices of free DOFs
    f: np.ndarray             # free-DOF RHS  -K_FD u_D


def assemble(problem) -> System:
    mesh = problem.mesh
    dofs = number_dofs(mesh.cells, mesh.dim, problem.order)
    A, M = assemble_volume(mesh, dofs, problem.mu_inv, problem.omega, eps=problem.eps)
    imp = [f for f, t in zip(mesh.bfaces, mesh.btag) if t == 0]
    Mg = assemble_faces(mesh, dofs, imp)
    K = (A - problem.omega ** 2 * M).astype(np.complex128) + 1j * problem.kappa * problem.omega * Mg
    is_d, uD = dirichlet_data(mesh, dofs, problem.omega, problem.pol, problem.direction)
    free = np.flatnonzero(~is_d)
    dd = np.flatnonzero(is_d)
    K = K.tocsr()
    f = -(K[free][:, dd] @ uD[dd])
    return System(dofs, K, A.tocsr(), M.tocsr(), Mg.tocsr(), is_d, uD, free, f)


def with_dirichlet(sys_: System, values: np.ndarray) -> System:
    """The same discrete problem with the Dirichlet trace of Eq. 1 given
    directly as the values of the Dirichlet DOFs (`values`, complex, in
    increasing global-DOF order) instead of the moments of a plane wave:
    u_D replaced and f = -K_FD u_D formed again."""
    dd = np.flatnonzero(sys_.is_dir)
    uD = np.zeros(sys_.dofs.n_dof, np.complex128)
    uD[dd] = values
    f = -(sys_.K[sys_.free][:, dd] @ uD[dd])
    return System(sys_.dofs, sys_.K, sys_.A, sys_.M, sys_.Mg, sys_.is_dir, uD, sys_.free, f)


def solve_monolithic(sys_: System) -> np.ndarray:
    """The plain definition of the discrete solution: u_F = K_FF^{-1}(-K_FD u_D)."""
    Kff = sys_.K[sys_.free][:, sys_.free].tocsc()
    uF = spla.spsolve(Kff, sys_.f)
    u = sys_.uD.copy()
    u[sys_.free] = uF
    return u


def residual(sys_: System, u: np.ndarray) -> float:
    """Relative true residual ||f - K_FF u_F - K_FD u_D|| / ||f|| on free rows."""
    r = -(sys_.K @ u)[sys_.free]
    return float(np.linalg.norm(r) / np.linalg.norm(sys_.f))


# ---------------------------------------------------------------------------
# Field evaluation (for pins against continuous / 1-D solutions)
# ---------------------------------------------------------------------------
def evaluate_field(mesh, dofs: Dofs, u: np.ndarray, cell: int, xi: np.ndarray):
    """E_h at reference points xi [np, dim] of `cell` -> complex [np, dim]."""
    J = cell_jacobian(mesh.coords, mesh.cells[cell], mesh.dim)
    JinvT = np.linalg.inv(J).T
    if mesh.dim == 2:
        V, _ = ref_basis_2d(dofs.order, xi[:, 0], xi[:, 1])
    else:
        V, _ = ref_basis_3d(xi[:, 0], xi[:, 1], xi[:, 2])
    coef = u[dofs.cell_dofs[cell]] * dofs.cell_signs[cell]
    phys = np.einsum("ab,qnb->qna", JinvT, V)
    return np.einsum("n,qna->qa", coef, phys)


def physical_point(mesh, cell, xi):
    J = cell_jacobian(mesh.coords, mesh.cells[cell], mesh.dim)
    return mesh.coords[mesh.cells[cell][0]][None, :] + xi @ J.T
