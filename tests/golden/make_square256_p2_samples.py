"""Write sampled values of the FP64 oracle's monolithic solution of the
256x256 order-2 workload (525,312 complex DOFs) to
square256_p2_monolithic_samples.json, for the full-size GPU parity test.

The monolithic solve of the plain definition u_F = K_FF^{-1}(-K_FD u_D)
(Section 2, Eqs. 1-3) takes about two minutes of one CPU core at this size,
so the test reads these stored samples instead of re-solving.  Only the
oracle (and the seeded input generators) is called here.

    python tests/golden/make_square256_p2_samples.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import fem  # noqa: E402

N_SAMPLES = 256


def main():
    P = W.config("square256_p2")
    S = fem.assemble(P)
    u0 = fem.solve_monolithic(S)
    # free DOFs only (the Dirichlet entries are inputs), seeded choice
    pick = np.sort(S.free[W.Rng("golden/square256_p2").permutation(len(S.free))[:N_SAMPLES]])
    out = {
        "workload": "square256_p2",
        "what": "oracle.fem.solve_monolithic: u = K_FF^{-1}(-K_FD u_D), sampled free DOFs",
        "n_dof": int(S.dofs.n_dof),
        "norm_u": float(np.linalg.norm(u0)),
        "oracle_rel_residual": fem.residual(S, u0),
        "dof": [int(d) for d in pick],
        "re": [float(v) for v in u0[pick].real],
        "im": [float(v) for v in u0[pick].imag],
    }
    with open(os.path.join(HERE, "square256_p2_monolithic_samples.json"), "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")


if __name__ == "__main__":
    main()
