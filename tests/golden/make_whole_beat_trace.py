"""Writes whole_beat_<workload>.txt: a whole activation-recovery beat (Section 6,
Test 4) computed by the oracle, sampled every 40 steps (2 ms).

Time stepping follows Sections 3b-3c with Newton tightened to rtol 1e-10 and
the linear systems solved directly (the plain definition of each Newton step),
from the seeded resting state with the workload's stimulus.  Each row holds
t, the Newton iterations of that step, min / max / mass-weighted mean of v
over the nodes, and v and u_e at five fixed nodes.  Calls only oracle/ and synth/.

    python tests/golden/make_whole_beat_trace.py [workload] [steps]
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle.bidomain import Problem, direct_solve, time_step  # noqa: E402

EVERY = 40


def sample_nodes(n_node):
    """Five fixed nodes spread over the node numbering (corners and centre)."""
    return [0, n_node // 4, n_node // 2, (3 * n_node) // 4, n_node - 1]


def main(name="beat_mini", steps=2400):
    w = synth.workload(name)
    prob = Problem(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, synth.stimulus(w))
    ui, ue, wg = synth.initial_state(prob.N, 0)
    nodes = sample_nodes(prob.N)
    M = prob.fem.M
    ls = lambda kc, a, b: direct_solve(prob, kc, a, b)  # noqa: E731
    rows = []
    for n in range(steps):
        ui, ue, wg, st = time_step(prob, ui, ue, wg, n, ls, rtol=1e-10, atol=1e-16)
        if (n + 1) % EVERY == 0:
            v = ui - ue
            rows.append([(n + 1) * prob.tau, st["newton_its"], v.min(), v.max(), float(M @ v) / M.sum()]
                        + list(v[nodes]) + list(ue[nodes]))
    hdr = ["# Oracle whole beat on %s: %d steps of %g ms from the seeded resting state," % (name, steps, prob.tau),
           "# workload stimulus, Newton rtol 1e-10 with direct linear solves; every %d steps." % EVERY,
           "# Written by tests/golden/make_whole_beat_trace.py (oracle only).",
           "# nodes: " + " ".join(str(x) for x in nodes),
           "# columns: t newton_its v_min v_max v_mean v(nodes) ue(nodes)"]
    with open(os.path.join(HERE, f"whole_beat_{name}.txt"), "w") as f:
        f.write("\n".join(hdr) + "\n")
        for r in rows:
            f.write(" ".join(f"{x:.17g}" for x in r) + "\n")


if __name__ == "__main__":
    main(*(sys.argv[1:2] or ["beat_mini"]), *(int(a) for a in sys.argv[2:3]))
