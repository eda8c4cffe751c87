"""Batches of independent problems in one system (thm_mesh_set_problems,
thm_assemble_batch): every problem's slice of the batched solution against
the FP64 monolithic oracle of that problem alone."""
import numpy as np
import pytest

import workloads as W
from oracle import fem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2105_11993_gb300 import build
    build.build()


def _problems():
    """Uneven sizes, subdomain counts (1, 4, 9, 4, 1) and omegas."""
    spec = [(8, 2, 6.0), (12, 3, 9.0), (6, 1, 5.0), (10, 2, 7.5), (4, 1, 4.0)]
    probs = []
    for p, (n, s, om) in enumerate(spec):
        mesh = W.structured_mesh_2d(n, n, s, s, relabel=(p % 2 == 1), rotate_cells=(p % 2 == 1))
        mu = W.mu_inv_lognormal(mesh.n_cell, 0.3, f"batch-test/{p}")
        pol, d = W.plane_wave_y(2)
        probs.append(W.Problem(f"b{p}", mesh, 1, mu, om, 1.0, pol, d))
    return probs


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_batch_matches_each_problem_alone(mode):
    import paper_2105_11993_gb300 as thm
    probs = _problems()
    mesh, offs = thm.Mesh.batch([P.mesh for P in probs], 1)
    mu = np.concatenate([P.mu_inv for P in probs])
    om = np.array([P.omega for P in probs])
    sysg = thm.System(mesh, mu, om, 1.0, probs[0].pol, probs[0].direction)
    rtol = 1e-11 if mode == "fp64" else 1e-9
    u, st = sysg.solve(mode=mode, rtol=rtol)
    u = u.cpu().numpy()
    assert st["rel_residual"] <= rtol
    d0 = 0
    for P in probs:
        S = fem.assemble(P)
        u0 = fem.solve_monolithic(S)
        up = u[d0:d0 + len(u0)]
        d0 += len(u0)
        assert np.linalg.norm(up - u0) <= (1e-8 if mode == "fp64" else 1e-6) * np.linalg.norm(u0), P.name
        # each problem's own FP64 residual meets the target
        assert fem.residual(S, up) <= rtol * (1 + 1e-6), P.name
    assert d0 == len(u)


def test_batch_declaration_errors():
    import paper_2105_11993_gb300 as thm
    probs = _problems()[:2]
    mesh, _ = thm.Mesh.batch([P.mesh for P in probs], 1)
    # a batch mesh takes one omega per problem
    with pytest.raises(thm.ThmError):
        thm.System(mesh, np.concatenate([P.mu_inv for P in probs]), 6.0, 1.0, probs[0].pol, probs[0].direction)
    # problems must own increasing subdomain ranges
    m2 = thm.Mesh(2, 1, *_union_arrays(probs))
    ns = int(m2._keep[2].max()) + 1
    with pytest.raises(thm.ThmError):
        m2.set_problems(np.arange(ns, dtype=np.int32)[::-1] % 2)


def _union_arrays(probs):
    coords, cells, subs, bf, bt = [], [], [], [], []
    v0 = s0 = 0
    for P in probs:
        mh = P.mesh
        coords.append(mh.coords); cells.append(mh.cells + v0); subs.append(mh.cell_sub + s0)
        bf.append(mh.bfaces + v0); bt.append(mh.btag)
        v0 += mh.coords.shape[0]; s0 += int(mh.cell_sub.max()) + 1
    return (np.concatenate(coords), np.concatenate(cells), np.concatenate(subs), np.concatenate(bf),
            np.concatenate(bt))


def test_batch_3d_matches_each_problem_alone():
    """Order-1 hexes: a batch of three cubes (1, 8 and 8 subdomains, different
    omega) against the monolithic oracle of each cube."""
    import paper_2105_11993_gb300 as thm
    probs = []
    for p, (n, s, om) in enumerate([(3, 1, 4.0), (4, 2, 6.0), (6, 2, 5.5)]):
        mesh = W.structured_mesh_3d(n, s, relabel=(p == 1), rotate_cells=(p == 1))
        mu = W.mu_inv_lognormal(mesh.n_cell, 0.3, f"batch3/{p}")
        pol, d = W.plane_wave_y(3)
        probs.append(W.Problem(f"c{p}", mesh, 1, mu, om, 1.0, pol, d))
    mesh, _ = thm.Mesh.batch([P.mesh for P in probs], 1)
    sysg = thm.System(mesh, np.concatenate([P.mu_inv for P in probs]), np.array([P.omega for P in probs]), 1.0,
                      probs[0].pol, probs[0].direction)
    u, st = sysg.solve(mode="mixed", rtol=1e-9)
    u = u.cpu().numpy()
    d0 = 0
    for P in probs:
        u0 = fem.solve_monolithic(fem.assemble(P))
        assert np.linalg.norm(u[d0:d0 + len(u0)] - u0) <= 1e-6 * np.linalg.norm(u0), P.name
        d0 += len(u0)
    assert d0 == len(u)
