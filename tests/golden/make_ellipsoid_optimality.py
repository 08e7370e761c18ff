"""Writes ellipsoid_optimality_h8.txt: the oracle's PCG-BDDC iteration counts and
condition-number estimates on the truncated ellipsoid with 4x4x4 subdomains and
H/h = 8 (the first row of the ellipsoid optimality test, Section 6, Table 8),
for the V, V+E and V+E+F primal spaces with deluxe and rho scaling.

The system is the first Newton step of the first time step from the seeded
resting state (synth.initial_state, seed 0) with the endocardial stimulus on.
Calls only oracle/ and synth/; takes about eight minutes on one core.

    python tests/golden/make_ellipsoid_optimality.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import ionic  # noqa: E402
from oracle.bidomain import Problem  # noqa: E402
from oracle.dd import DDSolver  # noqa: E402


def main():
    lines = ["# Oracle PCG-BDDC on the truncated ellipsoid, 4x4x4 subdomains, H/h = 8 (32^3 elements),",
             "# first Newton step of the first time step from the seeded resting state, stimulus on.",
             "# Written by tests/golden/make_ellipsoid_optimality.py (oracle only).",
             "# columns: primal scaling its cond"]
    for prim in ("V", "VE", "VEF"):
        w = dict(n=(32, 32, 32), ellipsoid=synth.ELLIPSOID, s=(8, 8, 8), primal=prim, name="ellopt8")
        prob = Problem(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, synth.stimulus(w))
        ui, ue, wg = synth.initial_state(prob.N, 0)
        wn = ionic.gating_step(ui - ue, wg, prob.tau, prob.p)
        r_i, r_e = prob.residual(ui, ue, wn, ui, ue, prob.tau)
        kc = prob.kc(ui, ue, wn)
        for scaling in ("deluxe", "rho"):
            dd = DDSolver(prob, scaling=scaling)
            _, _, info = dd.solve(kc / prob.fem.M, -r_i, -r_e)
            lines.append(f"{prim} {scaling} {info['its']} {info['cond']:.4f}")
            print(lines[-1], flush=True)
    with open(os.path.join(HERE, "ellipsoid_optimality_h8.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
