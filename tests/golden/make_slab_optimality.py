"""Writes slab_optimality.txt: the oracle's PCG-BDDC iteration counts and Lanczos
condition-number estimates on the 0.8 cm cube with 4x4x4 subdomains at H/h = 4, 8
and 12 (the optimality test of Section 6, Test 3 / Table 7), for the V+E and the
vertex-only (V) primal spaces with deluxe scaling.

The system is the first Newton step of the first time step from the seeded resting
state (synth.initial_state, seed 0) with the corner stimulus on, at the paper's
Krylov tolerance (rtol 1e-8).  Calls only oracle/ and synth/.  H/h = 12 takes
several minutes per primal space on a few cores.

    python tests/golden/make_slab_optimality.py          # H/h = 4, 8, 12
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import ionic  # noqa: E402
from oracle.bidomain import Problem  # noqa: E402
from oracle.dd import DDSolver  # noqa: E402


def first_newton_solve(hh, primal):
    """(its, cond) of the oracle's PCG-BDDC deluxe solve of the first Newton system."""
    w = synth.workload(f"opt{hh}")
    w["primal"] = primal
    prob = Problem(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, synth.stimulus(w))
    ui, ue, wg = synth.initial_state(prob.N, 0)
    wn = ionic.gating_step(ui - ue, wg, prob.tau, prob.p)
    r_i, r_e = prob.residual(ui, ue, wn, ui, ue, prob.tau)
    kc = prob.kc(ui, ue, wn)
    _, _, info = DDSolver(prob, keep_fetidp=False).solve(kc / prob.fem.M, -r_i, -r_e)
    return info["its"], info["cond"]


def main(hhs=(4, 8, 12)):
    lines = ["# Oracle PCG-BDDC deluxe on the 0.8 cm cube, 4x4x4 subdomains (opt<H/h> workloads),",
             "# first Newton step of the first time step from the seeded resting state, stimulus on.",
             "# Written by tests/golden/make_slab_optimality.py (oracle only).",
             "# columns: H/h primal its cond"]
    for hh in hhs:
        for primal in ("VE", "V"):
            its, cond = first_newton_solve(hh, primal)
            lines.append(f"{hh} {primal} {its} {cond:.6f}")
            print(lines[-1], flush=True)
    with open(os.path.join(HERE, "slab_optimality.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main(tuple(int(a) for a in sys.argv[1:]) or (4, 8, 12))
