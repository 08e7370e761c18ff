"""Writes ellipsoid_optimality_h<H/h>.txt: the oracle's PCG-BDDC iteration counts and
condition-number estimates on the truncated ellipsoid with 4x4x4 subdomains
(the ellipsoid optimality test, Section 6, Table 8): at H/h = 8 for the V, V+E
and V+E+F primal spaces with deluxe and rho scaling, at H/h = 12 for V+E with
deluxe scaling.

The system is the first Newton step of the first time step from the seeded
resting state (synth.initial_state, seed 0) with the endocardial stimulus on.
Calls only oracle/ and synth/; takes about eight minutes on one core for H/h = 8.

    python tests/golden/make_ellipsoid_optimality.py        # H/h = 8
    python tests/golden/make_ellipsoid_optimality.py 12     # H/h = 12, V+E deluxe
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import ionic  # noqa: E402
from oracle.bidomain import Problem  # noqa: E402
from oracle.dd import DDSolver  # noqa: E402


def main(hh=8):
    n = 4 * hh
    lines = [f"# Oracle PCG-BDDC on the truncated ellipsoid, 4x4x4 subdomains, H/h = {hh} ({n}^3 elements),",
             "# first Newton step of the first time step from the seeded resting state, stimulus on.",
             "# Written by tests/golden/make_ellipsoid_optimality.py (oracle only).",
             "# columns: primal scaling its cond"]
    cases = (("V", "VE", "VEF"), ("deluxe", "rho")) if hh == 8 else (("VE",), ("deluxe",))
    for prim in cases[0]:
        w = dict(n=(n, n, n), ellipsoid=synth.ELLIPSOID, s=(hh, hh, hh), primal=prim, name=f"ellopt{hh}")
        prob = Problem(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, synth.stimulus(w))
        ui, ue, wg = synth.initial_state(prob.N, 0)
        wn = ionic.gating_step(ui - ue, wg, prob.tau, prob.p)
        r_i, r_e = prob.residual(ui, ue, wn, ui, ue, prob.tau)
        kc = prob.kc(ui, ue, wn)
        for scaling in cases[1]:
            dd = DDSolver(prob, scaling=scaling)
            _, _, info = dd.solve(kc / prob.fem.M, -r_i, -r_e)
            lines.append(f"{prim} {scaling} {info['its']} {info['cond']:.4f}")
            print(lines[-1], flush=True)
    with open(os.path.join(HERE, f"ellipsoid_optimality_h{hh}.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main(*(int(a) for a in sys.argv[1:2]))
