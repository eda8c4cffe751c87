"""Parity at the size the bench runs.

* square64_p2: 64x64 order-2 quads in 2x2 subdomains of 32x32 cells, so each
  subdomain is exactly the bench's (8,320 free DOFs away from the Dirichlet
  side, about 66 BFS levels, the autotuned tile ring), omega*h as in the bench.
  P_i^{-1} (Eq. 7) and T_i (Eq. 5) per subdomain against the oracle's sparse
  LU and matrices, and the full DDM solve against the oracle's monolithic
  solve, element by element, in FP64 and mixed precision.
* square256_p2 itself (525,312 DOFs, 8x8 subdomains), in the launch
  configuration bench.py times: P_i^{-1} and T_i on sampled subdomains against
  the oracle, and the mixed-precision solve against stored samples of the
  oracle's monolithic solution (tests/golden, written by a script that calls
  only the oracle) plus the oracle's FP64 residual of the whole answer.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import ddm as odd
from oracle import fem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2105_11993_gb300 import build
    build.build()


def _system(P):
    import paper_2105_11993_gb300 as thm
    mesh = thm.Mesh.from_workload(P.mesh, P.order)
    return mesh, thm.System(mesh, torch.tensor(P.mu_inv, device="cuda"), P.omega, P.kappa, P.pol, P.direction)


def _local_perm(sysg, D):
    gd, sub = sysg.local_dofs()
    pos = np.empty(len(gd), np.int64)
    for s in D.subs:
        idx = np.flatnonzero(sub == s.idx)
        pos[idx] = np.searchsorted(s.dofs[s.free], gd[idx])
        assert np.array_equal(s.dofs[s.free][pos[idx]], gd[idx])
    return sub, pos


def _rand_local(n, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(n) + 1j * r.standard_normal(n)


@pytest.fixture(scope="module")
def sub_size():
    P = W.config("square64_p2")
    mesh, sysg = _system(P)
    D = odd.setup(P)
    return P, mesh, sysg, D


@pytest.fixture(scope="module")
def full_size():
    P = W.config("square256_p2")
    mesh, sysg = _system(P)
    D = odd.setup(P)
    return P, mesh, sysg, D


def _check_ops(sysg, D, subs, mode, seed):
    import paper_2105_11993_gb300 as thm
    sub, pos = _local_perm(sysg, D)
    x = _rand_local(sysg.n_local, seed)
    xt = torch.tensor(x, device="cuda")
    y_t = sysg.apply_local(thm.OP_T, xt, mode=mode).cpu().numpy()
    y_p = sysg.apply_local(thm.OP_PINV, xt, mode=mode).cpu().numpy()
    tol_t = 1e-14 if mode == "fp64" else 1e-6
    tol_p = 1e-10 if mode == "fp64" else 2e-3
    for i in subs:
        s = D.subs[i]
        idx = np.flatnonzero(sub == i)
        xs = np.zeros(len(s.free), np.complex128)
        xs[pos[idx]] = x[idx]
        ys = s.Tff @ xs
        assert np.linalg.norm(y_t[idx] - ys[pos[idx]]) <= tol_t * np.linalg.norm(ys), (i, "T")
        lu = spla.splu(s.P)
        ys = lu.solve(xs.real) + 1j * lu.solve(xs.imag)
        err = np.linalg.norm(y_p[idx] - ys[pos[idx]]) / np.linalg.norm(ys)
        assert err <= tol_p, (i, "PINV", err)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_bench_subdomain_operators(sub_size, mode):
    """T_i and P_i^{-1} on subdomains of the bench's size and shape."""
    P, mesh, sysg, D = sub_size
    assert max(len(s.free) for s in D.subs) == 8320
    _check_ops(sysg, D, range(len(D.subs)), mode, 21)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_bench_subdomain_full_solve(sub_size, mode):
    """The whole DDM-GMRES solve on bench-sized subdomains against the
    monolithic oracle (33,024 DOFs), element by element."""
    P, mesh, sysg, D = sub_size
    S = D.sys
    u0 = fem.solve_monolithic(S)
    u, st = sysg.solve(mode=mode, rtol=1e-11 if mode == "fp64" else 1e-9, relax=1)
    u = u.cpu().numpy()
    err = np.linalg.norm(u - u0) / np.linalg.norm(u0)
    assert err <= (1e-8 if mode == "fp64" else 1e-6), err
    r_or = fem.residual(S, u)
    assert abs(r_or - st["rel_residual"]) <= 1e-2 * st["rel_residual"] + 1e-13


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_full_size_sampled_operators(full_size, mode):
    """T_i and P_i^{-1} of the 256x256 workload itself on sampled subdomains
    (a corner on the Dirichlet side, an interior and an opposite corner),
    applied to all 64 subdomains in one launch as in the bench."""
    P, mesh, sysg, D = full_size
    _check_ops(sysg, D, [0, 27, 63], mode, 22)


def test_full_size_mixed_solve_against_stored_oracle_samples(full_size):
    """The bench's mixed-precision solve at full size: sampled DOFs against the
    oracle's monolithic solution, and the oracle's FP64 residual of the whole
    answer."""
    P, mesh, sysg, D = full_size
    g = json.load(open(os.path.join(HERE, "golden", "square256_p2_monolithic_samples.json")))
    assert g["n_dof"] == sysg.n_dof
    u, st = sysg.solve(mode="mixed", rtol=1e-9, relax=1)
    u = u.cpu().numpy()
    dof = np.array(g["dof"])
    ref = np.array(g["re"]) + 1j * np.array(g["im"])
    err = np.linalg.norm(u[dof] - ref) / np.linalg.norm(ref)
    assert err <= 1e-6, err
    assert abs(np.linalg.norm(u) - g["norm_u"]) <= 1e-6 * g["norm_u"]
    r_or = fem.residual(D.sys, u)
    assert r_or <= 1e-9 and abs(r_or - st["rel_residual"]) <= 1e-2 * st["rel_residual"] + 1e-13
