"""The device work counters behind thm_work_bytes (the byte counts of the
bench line's roofline entries), checked against values fixed by the byte
model: one operator or preconditioner apply with every subdomain active moves
exactly thm_alg_bytes; a Gram-Schmidt pass moves whole subdomain vectors, so
its byte count is a sum of multiples of the subdomain sizes; and a solve whose
subdomains converge at different steps counts less SpMV work than a full
launch per step."""
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


def _system():
    import paper_2105_11993_gb300 as thm
    P = W.square_problem(16, 2, 2, 13.0, mu_inv=W.mu_inv_lognormal(256, 0.3, "work"))
    mesh = thm.Mesh.from_workload(P.mesh, P.order)
    return thm, thm.System(mesh, P.mu_inv, P.omega, P.kappa, P.pol, P.direction)


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_single_applies_count_the_full_model(mode):
    thm, s = _system()
    dt = torch.complex128
    x = torch.randn(s.n_local, dtype=dt, device="cuda")
    b0 = thm.work_bytes(s, mode, thm.K_SPMV)
    s.apply_local(thm.OP_T, x, mode=mode)
    assert thm.work_bytes(s, mode, thm.K_SPMV) - b0 == pytest.approx(thm.algorithmic_bytes(s, mode, thm.K_SPMV),
                                                                      rel=1e-12)
    before = thm.work_bytes(s, mode, thm.K_PINV)
    s.apply_local(thm.OP_PINV, x, mode=mode)          # the first apply also runs the tile autotuner
    after = thm.work_bytes(s, mode, thm.K_PINV)
    full = thm.algorithmic_bytes(s, mode, thm.K_PINV)
    ratio = (after - before) / full
    assert ratio == pytest.approx(round(ratio), rel=1e-12) and round(ratio) >= 1
    s.apply_local(thm.OP_PINV, x, mode=mode)
    assert thm.work_bytes(s, mode, thm.K_PINV) - after == pytest.approx(full, rel=1e-12)


def test_solve_counts_whole_vector_passes_and_skips_converged_subdomains():
    thm, s = _system()
    _, st = s.solve(mode="mixed", rtol=1e-8)
    vec = 8.0                                           # complex FP32 entry
    dots = thm.work_bytes(s, "mixed", thm.K_DOTS)
    upd = thm.work_bytes(s, "mixed", thm.K_UPDATE)
    assert dots > 0 and upd > 0
    # every chunk of a subdomain is counted together, so a pass adds whole
    # multiples of the subdomain's entries; the counts are sums of (k x n_s)
    # vector entries over the passes
    sizes = np.bincount(s.local_dofs()[1])
    g = np.gcd.reduce(sizes.astype(np.int64))
    assert (dots / vec) % g == 0 and (upd / vec) % g == 0
    # the SpMV work of the solve is below (launches x full launch) once
    # subdomains converge at different steps, and at least one full launch
    full = thm.algorithmic_bytes(s, "mixed", thm.K_SPMV)
    spmv = thm.work_bytes(s, "mixed", thm.K_SPMV)
    assert spmv >= full
    assert spmv / full < st["inner_iters"]
