"""Error returns of the C ABI on the GPU, produced without faulting the GPU:

* THM_ETIMEOUT: the block-preconditioner apply's bounded waits (tile stream
  held back by a test switch, 50 ms limit) give up, the kernel finishes and
  the host reads the flag; the system stays usable afterwards;
* THM_ESINGULAR: a non-finite mu^{-1} given on the device (not checked on the
  host) makes a pivot of the factorisation fail;
* THM_EBREAKDOWN: non-finite Dirichlet values given on the device give a
  non-finite residual, reported instead of a result.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2105_11993_gb300 import build
    build.build()


def _problem():
    return W.square_problem(12, 2, 2, 9.0, mu_inv=W.mu_inv_lognormal(144, 0.3, "err"))


def test_bounded_wait_expires_and_the_context_survives(monkeypatch):
    import scipy.sparse.linalg as spla
    import paper_2105_11993_gb300 as thm
    from oracle import ddm as odd
    P = _problem()
    monkeypatch.setenv("THM_BT_TILE_BYTES", "16384")      # no autotuning launches
    mesh = thm.Mesh.from_workload(P.mesh, P.order)
    sysg = thm.System(mesh, P.mu_inv, P.omega, P.kappa, P.pol, P.direction)
    x = torch.randn(sysg.n_local, dtype=torch.complex128, device="cuda")
    monkeypatch.setenv("THM_BT_WAIT_LIMIT_MS", "50")
    monkeypatch.setenv("THM_TEST_STALL_TMA", "1")
    with pytest.raises(thm.ThmError) as ei:
        sysg.apply_local(thm.OP_PINV, x, mode="mixed")
    assert ei.value.code == -5
    monkeypatch.delenv("THM_TEST_STALL_TMA")
    # the same system, the same launch, without the switch: the oracle's P^{-1}
    y = sysg.apply_local(thm.OP_PINV, x, mode="fp64").cpu().numpy()
    D = odd.setup(P)
    gd, sub = sysg.local_dofs()
    xh = x.cpu().numpy()
    for s in D.subs:
        idx = np.flatnonzero(sub == s.idx)
        pos = np.searchsorted(s.dofs[s.free], gd[idx])
        xs = np.zeros(len(s.free), np.complex128)
        xs[pos] = xh[idx]
        lu = spla.splu(s.P)
        ref = lu.solve(xs.real) + 1j * lu.solve(xs.imag)
        assert np.linalg.norm(y[idx] - ref[pos]) <= 1e-10 * np.linalg.norm(ref)


def test_non_finite_mu_inv_on_device_is_singular():
    import paper_2105_11993_gb300 as thm
    P = _problem()
    mu = torch.tensor(P.mu_inv, device="cuda")
    mu[7] = float("nan")
    mesh = thm.Mesh.from_workload(P.mesh, P.order)
    with pytest.raises(thm.ThmError) as ei:          # at assembly (the cell-bubble blocks) or at the factorisation
        sysg = thm.System(mesh, mu, P.omega, P.kappa, P.pol, P.direction)
        sysg.solve(mode="fp64", rtol=1e-8)
    assert ei.value.code == -4


def test_non_finite_dirichlet_values_on_device_are_a_breakdown():
    import paper_2105_11993_gb300 as thm
    P = _problem()
    mesh = thm.Mesh.from_workload(P.mesh, P.order)
    d = torch.ones(len(mesh.dirichlet_dofs()), dtype=torch.complex128, device="cuda")
    d[3] = complex(float("nan"), 0.0)
    sysg = thm.System(mesh, P.mu_inv, P.omega, P.kappa, dirichlet=d)
    with pytest.raises(thm.ThmError) as ei:
        sysg.solve(mode="fp64", rtol=1e-8)
    assert ei.value.code == -3
