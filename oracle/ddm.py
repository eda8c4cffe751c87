"""Oracle DDM: non-overlapping optimized Schwarz with impedance transmission.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Sequential, FP64.

Follows Section 3.1 of the paper:
* the domain is split into cell-aligned subdomains Omega_i with interfaces
  Sigma_ij (shared faces);
* each subdomain solves the THM problem with the impedance transmission
  condition of Eq. 5 on Sigma_ij (S = identity, Section 3.1 end), k = kappa*omega;
* the interface data are updated by Eq. 6; one sweep is the map A of Eq. 8, and
  (I - A) g = b is solved by GMRES (or by the Jacobi fixed point, Eq. 8).

Discrete reading (the paper gives only the continuous equations).  With
M_ij the tangential face mass on Sigma_ij and the receiver-indexed dual vector
G_{i<-j} standing for -int g_{i<-j} . phi on Sigma_ij:

  subdomain i:  (K_i + i k sum_j M_ij) u_i = s_i + sum_j G_{i<-j}
  update:       G_{i<-j}  <-  -G_{j<-i} + 2 i k M_ij u_j

(i k is the impedance coefficient; `setup(..., transmission=c)` puts c k in
its place to study other interface conditions.)

where K_i is the part of the global matrix assembled from the cells of
Omega_i (volume terms and the Gamma^inf impedance terms of its boundary).  At a
fixed point, adding and subtracting the two updates of a pair gives
M_ij (u_i - u_j) = 0 and G_{i<-j} + G_{j<-i} = i k M_ij (u_i + u_j); the
transmission terms then cancel when the subdomain rows are summed, so the
fixed point is the monolithic discrete solution (pinned by a test).

Subdomain solves are either direct (sparse LU) or, as in Section 3.2, GMRES
right-preconditioned with the block-diagonal operator of Eq. 7, i.e. the real
matrix P_i = A_i - omega^2 M_i applied to real and imaginary parts alike, or
with the full 2x2 block operator that Section 3.2 describes as the
alternative (its exact inverse; with the sign of Eq. 3 it is T_ff^{-1}).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem
from .krylov import gmres


@dataclass
class Sub:
    idx: int
    cells: np.ndarray
    dofs: np.ndarray          # global DOFs touched by the subdomain's cells (sorted)
    free: np.ndarray          # positions (into dofs) of free DOFs
    dirl: np.ndarray          # positions of Dirichlet DOFs
    T: sp.csr_matrix          # K_i + i k sum_j M_ij over `dofs`
    K_loc: sp.csr_matrix      # K_i over `dofs` (no transmission terms)
    Tff: sp.csc_matrix = None
    P: sp.csc_matrix = None   # Re(T_ff) = A_i - omega^2 M_i on free DOFs
    lu_T: object = None
    lu_P: object = None


@dataclass
class Pair:
    i: int                    # receiver
    j: int                    # sender
    dofs: np.ndarray          # all global DOFs on Sigma_ij (sorted)
    free: np.ndarray          # global free DOFs on Sigma_ij (sorted)
    M: sp.csr_matrix          # tangential mass over `dofs`


@dataclass
class DDM:
    sys: fem.System
    subs: list
    pairs: list               # directed (i <- j), sorted by (i, j)
    kw: complex               # i * kappa * omega (the Gamma^inf impedance coefficient)
    offsets: np.ndarray       # start of each pair's block in the interface vector
    kt: complex = None        # transmission coefficient on Sigma_ij (default kw)
    stats: dict = field(default_factory=dict)

    @property
    def n_iface(self):
        return int(self.offsets[-1])


def setup(problem, sys_: fem.System | None = None, transmission: complex = 1j) -> DDM:
    """transmission: the interface coefficient in units of kappa*omega.  1j is
    the impedance condition of Eq. 5 (S = 1); a real value replaces it by a
    Robin condition with a real coefficient, and a large real value is the
    penalty form of the Dirichlet-like classical interface condition of
    Section 3.1.  The fixed point is the monolithic solution for any nonzero
    coefficient (the argument above does not use its value)."""
    mesh = problem.mesh
    if sys_ is None:
        sys_ = fem.assemble(problem)
    dofs = sys_.dofs
    kw = 1j * problem.kappa * problem.omega
    kt = complex(transmission) * problem.kappa * problem.omega
    fverts, fcells = fem.cell_faces(mesh)
    sub_of = mesh.cell_sub
    # interface faces: two cells in different subdomains
    both = fcells[:, 1] >= 0
    iface = np.flatnonzero(both & (sub_of[fcells[:, 0]] != sub_of[np.maximum(fcells[:, 1], 0)]))
    pair_faces: dict = {}
    for f in iface:
        a, b = int(sub_of[fcells[f, 0]]), int(sub_of[fcells[f, 1]])
        pair_faces.setdefault((min(a, b), max(a, b)), []).append(fverts[f])
    imp = [(f, t) for f, t in zip(mesh.bfaces, mesh.btag) if t == 0]
    # owner cell of each impedance face: map its sorted key to a cell
    fkey = {tuple(sorted(fv)): fc[0] for fv, fc in zip(fverts, fcells) if fc[1] < 0}
    nsub = int(sub_of.max()) + 1
    imp_by_sub = [[] for _ in range(nsub)]
    for f, _ in imp:
        imp_by_sub[int(sub_of[fkey[tuple(sorted(f))]])].append(f)

    A_all, M_all = fem.cell_matrices(mesh, dofs.order)
    subs = []
    pair_M = {}
    for key, faces in pair_faces.items():
        pair_M[key] = fem.assemble_faces(mesh, dofs, faces)
    for i in range(nsub):
        cells = np.flatnonzero(sub_of == i)
        gd = np.unique(dofs.cell_dofs[cells])
        A, M = fem.assemble_volume(mesh, dofs, problem.mu_inv, problem.omega, cells, eps=problem.eps)
        Mg = fem.assemble_faces(mesh, dofs, imp_by_sub[i])
        Kg = (A - problem.omega ** 2 * M).astype(np.complex128) + kw * Mg
        Tg = Kg.copy()
        for (a, b), Mp in pair_M.items():
            if i in (a, b):
                Tg = Tg + kt * Mp
        T = Tg.tocsr()[gd][:, gd].tocsr()
        Kl = Kg.tocsr()[gd][:, gd].tocsr()
        isd = sys_.is_dir[gd]
        s = Sub(i, cells, gd, np.flatnonzero(~isd), np.flatnonzero(isd), T, Kl)
        s.Tff = T[s.free][:, s.free].tocsc()
        # P = Re(T_ff): A_i - omega^2 M_i (plus the real part of the transmission term, if any)
        Pm = s.Tff.copy()
        s.P = sp.csc_matrix((np.ascontiguousarray(Pm.data.real), Pm.indices.copy(), Pm.indptr.copy()), shape=Pm.shape)
        subs.append(s)
    pairs = []
    for (a, b), Mp in sorted(pair_M.items()):
        Mp = Mp.tocsr()
        d_all = np.unique(Mp.nonzero()[0])
        d_free = d_all[~sys_.is_dir[d_all]]
        Ml = Mp[d_all][:, d_all].tocsr()
        pairs.append(Pair(a, b, d_all, d_free, Ml))
        pairs.append(Pair(b, a, d_all, d_free, Ml))
    pairs.sort(key=lambda p: (p.i, p.j))
    offsets = np.concatenate([[0], np.cumsum([len(p.free) for p in pairs])])
    return DDM(sys_, subs, pairs, kw, offsets, kt=kt)


def local_sources(ddm: DDM) -> list:
    """Per-subdomain RHS from the Dirichlet lifting: -(T_i)_{F,D} u_D."""
    out = []
    for s in ddm.subs:
        uD = ddm.sys.uD[s.dofs[s.dirl]]
        out.append(-(s.T[s.free][:, s.dirl] @ uD) if len(s.dirl) else np.zeros(len(s.free), np.complex128))
    return out


def subdomain_solver(ddm: DDM, kind: str = "direct", inner_tol: float = 1e-12,
                     restart: int = 60, maxiter: int = 2000):
    """Return solve(i, rhs) -> u_free for the subdomain problems of Eq. 5."""
    ddm.stats.setdefault("inner_iters", [])
    if kind == "direct":
        for s in ddm.subs:
            if s.lu_T is None:
                s.lu_T = spla.splu(s.Tff)
        return lambda i, rhs: ddm.subs[i].lu_T.solve(rhs)
    if kind == "full_block":
        # the full 2x2 block operator of Section 3.2 with the sign of Eq. 3,
        # [[P, -B], [B, P]], is the real form of T_ff itself: its exact inverse
        # is T_ff^{-1}, so right-preconditioned GMRES stops after one step
        for s in ddm.subs:
            if s.lu_T is None:
                s.lu_T = spla.splu(s.Tff)

        def solve_full(i, rhs):
            s = ddm.subs[i]
            x, it, _ = gmres(lambda v: s.Tff @ v, rhs, precond=s.lu_T.solve, tol=inner_tol, restart=restart,
                             maxiter=maxiter)
            ddm.stats["inner_iters"].append((i, it))
            return x
        return solve_full
    if kind == "full_block_printed":
        # the same block operator with the off-diagonal signs as printed in
        # Section 3.2, [[P, -B], [-B, P]] (a real symmetric matrix), applied
        # to the real/imaginary splitting of the residual
        lus = {}

        def solve_printed(i, rhs):
            s = ddm.subs[i]
            if i not in lus:
                Bm = sp.csc_matrix((np.ascontiguousarray(s.Tff.data.imag), s.Tff.indices.copy(),
                                    s.Tff.indptr.copy()), shape=s.Tff.shape)
                lus[i] = spla.splu(sp.bmat([[s.P, -Bm], [-Bm, s.P]], format="csc"))
            nf = s.Tff.shape[0]

            def prec(v):
                y = lus[i].solve(np.concatenate([v.real, v.imag]))
                return y[:nf] + 1j * y[nf:]
            x, it, _ = gmres(lambda v: s.Tff @ v, rhs, precond=prec, tol=inner_tol, restart=restart,
                             maxiter=maxiter)
            ddm.stats["inner_iters"].append((i, it))
            return x
        return solve_printed
    if kind == "block_gmres":
        for s in ddm.subs:
            if s.lu_P is None:
                s.lu_P = spla.splu(s.P)

        def solve(i, rhs):
            s = ddm.subs[i]
            # Eq. 7: blockdiag(P, P)^{-1} on (Re, Im) == real P^{-1} on a complex vector
            prec = lambda v: s.lu_P.solve(v.real) + 1j * s.lu_P.solve(v.imag)
            x, it, _ = gmres(lambda v: s.Tff @ v, rhs, precond=prec, tol=inner_tol,
                             restart=restart, maxiter=maxiter)
            ddm.stats["inner_iters"].append((i, it))
            return x
        return solve
    raise ValueError(kind)


def sweep(ddm: DDM, g: np.ndarray, sources, with_dirichlet: bool, solve):
    """One application of Eqs. 5-6: returns (g_new, [u_i over s.dofs])."""
    sysd = ddm.sys
    us = []
    for s in ddm.subs:
        rhs = np.zeros(len(s.free), np.complex128)
        if sources is not None:
            rhs += sources[s.idx]
        pos_of = {int(d): k for k, d in enumerate(s.dofs[s.free])}
        for p, (lo, hi) in zip(ddm.pairs, zip(ddm.offsets[:-1], ddm.offsets[1:])):
            if p.i != s.idx:
                continue
            for d, val in zip(p.free, g[lo:hi]):
                rhs[pos_of[int(d)]] += val
        u = np.zeros(len(s.dofs), np.complex128)
        if np.any(rhs != 0):
            u[s.free] = solve(s.idx, rhs)
        if with_dirichlet:
            u[s.dirl] = sysd.uD[s.dofs[s.dirl]]
        us.append(u)
    g_new = np.zeros_like(g)
    # partner block of (i <- j) is (j <- i); same DOF order in both
    index = {(p.i, p.j): k for k, p in enumerate(ddm.pairs)}
    for k, p in enumerate(ddm.pairs):
        lo, hi = ddm.offsets[k], ddm.offsets[k + 1]
        q = index[(p.j, p.i)]
        plo, phi = ddm.offsets[q], ddm.offsets[q + 1]
        sj = ddm.subs[p.j]
        uj = us[p.j][np.searchsorted(sj.dofs, p.dofs)]
        Mu = p.M @ uj
        sel = np.searchsorted(p.dofs, p.free)
        g_new[lo:hi] = -g[plo:phi] + 2.0 * ddm.kt * Mu[sel]
    return g_new, us


def glue(ddm: DDM, us) -> np.ndarray:
    """Global u: each DOF from the lowest-numbered subdomain holding it."""
    u = ddm.sys.uD.copy()
    done = ddm.sys.is_dir.copy()
    for s in ddm.subs:                       # ascending subdomain id
        gd = s.dofs[s.free]
        new = ~done[gd]
        u[gd[new]] = us[s.idx][s.free][new]
        done[gd] = True
    return u


def solve(problem_or_ddm, *, outer: str = "gmres", inner: str = "direct", outer_tol=1e-10,
          inner_tol=1e-12, outer_restart=200, outer_maxiter=500, inner_restart=60,
          sources=None):
    """DDM solve of Eq. 8 followed by the final subdomain solves and gluing.

    Returns (u_global, info) with info = dict(outer_iters, inner_iters, hist).
    """
    ddm = problem_or_ddm if isinstance(problem_or_ddm, DDM) else setup(problem_or_ddm)
    ddm.stats["inner_iters"] = []
    sv = subdomain_solver(ddm, inner, inner_tol=inner_tol, restart=inner_restart)
    src = local_sources(ddm) if sources is None else sources
    zero = np.zeros(ddm.n_iface, np.complex128)
    b, _ = sweep(ddm, zero, src, True, sv)
    if outer == "gmres":
        op = lambda v: v - sweep(ddm, v, None, False, sv)[0]
        g, it, hist = gmres(op, b, tol=outer_tol, restart=outer_restart, maxiter=outer_maxiter)
    elif outer == "jacobi":
        g = zero.copy()
        hist = []
        bn = np.linalg.norm(b)
        it = 0
        while it < outer_maxiter:
            gn, _ = sweep(ddm, g, None, False, sv)
            res = np.linalg.norm(g - gn - b) / bn
            hist.append(res)
            if res < outer_tol:
                break
            g = gn + b
            it += 1
    else:
        raise ValueError(outer)
    _, us = sweep(ddm, g, src, True, sv)
    u = glue(ddm, us)
    return u, dict(outer_iters=it, inner_iters=list(ddm.stats["inner_iters"]), hist=hist,
                   g=g, us=us, ddm=ddm)
