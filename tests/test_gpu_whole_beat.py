"""Whole-beat runner on the GPU (Section 6, Test 4): many consecutive steps through the
stimulus and the upstroke, against the oracle's own run of the same steps."""
import numpy as np
import pytest

import synth
from conftest import oracle_problem
from oracle.bidomain import time_step
from oracle.dd import DDSolver

pytestmark = pytest.mark.gpu


def test_runner_follows_the_oracle_through_the_upstroke():
    from paper_2101_02959_gb300 import beat, binding, build
    build.build()
    name, steps = "cube8ve", 24  # 1.2 ms: the 1 ms stimulus and the start of propagation
    prob = oracle_problem(name)
    dd = DDSolver(prob, rtol=1e-12, atol=0.0)
    ui, ue, w = synth.initial_state(prob.N, 0)
    newton = []
    for n in range(steps):
        ui, ue, w, st = time_step(prob, ui, ue, w, n, dd.linsolve(), rtol=1e-10, atol=1e-16)
        newton.append(st["newton_its"])
    opt = dict(precision="fp64", ksp_rtol=1e-12, ksp_atol=0.0, snes_rtol=1e-10, snes_atol=1e-16)
    recs = list(beat.run(synth.workload(name), steps, **opt))
    assert len(recs) == steps and all(r["reason"] == 0 for r in recs)
    summ = beat.summarize(recs)
    assert abs(summ["nlit"] - np.mean(newton)) <= 0.5
    # the same steps through the public handle give the oracle's state at the end
    s = binding.Solver(synth.workload(name), synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, **opt)
    u0 = synth.initial_state(prob.N, 0)
    s.set_state(*u0, 0.0)
    for n in range(steps):
        assert s.step(synth.stimulus(prob.workload))["reason"] == 0
    gui, gue, _, _ = s.get_state()
    s.close()
    v, gv = ui - ue, gui - gue
    for a, b in ((gv, v), (gue, ue)):  # 2-norm and entry-wise
        assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b)
        assert np.max(np.abs(a - b)) <= 1e-8 * np.max(np.abs(b))


def _trace(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", f"whole_beat_{name}.txt")
    nodes, rows = None, []
    for line in open(path):
        if line.startswith("# nodes:"):
            nodes = [int(x) for x in line.split(":")[1].split()]
        elif line.strip() and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return nodes, np.array(rows)


def test_whole_beat_against_the_oracle_trace():
    """A whole activation-recovery beat (2,400 steps, 120 ms) on the GPU against the
    oracle's stored run (direct solves, tight Newton): v and u_e at five nodes and the
    extremes and mean of v every 2 ms, and the Newton iteration counts."""
    from paper_2101_02959_gb300 import binding, build
    build.build()
    name = "beat_mini"
    nodes, ref = _trace(name)
    prob = oracle_problem(name)
    s = binding.Solver(synth.workload(name), synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU,
                       precision="fp64", ksp_rtol=1e-12, ksp_atol=0.0, snes_rtol=1e-10, snes_atol=1e-16)
    s.set_state(*synth.initial_state(prob.N, 0), 0.0)
    stim = synth.stimulus(prob.workload)
    M = prob.fem.M
    every = int(round(ref[0, 0] / synth.TAU))
    k = 0
    for n in range(int(round(ref[-1, 0] / synth.TAU))):
        st = s.step(stim)
        assert st["reason"] == 0
        if (n + 1) % every:
            continue
        ui, ue, _, t = s.get_state()
        row = ref[k]
        k += 1
        assert abs(t - row[0]) < 1e-9
        assert abs(st["newton_its"] - row[1]) <= 1
        v = ui - ue
        got = np.r_[v.min(), v.max(), float(M @ v) / M.sum(), v[nodes], ue[nodes]]
        assert np.abs(got - row[2:]).max() < 1e-3, (t, np.abs(got - row[2:]).max())
    s.close()
    assert k == len(ref)


def test_runner_activation_time_matches_the_oracle_beat():
    """The runner's activation map (sampled every 2 ms) on beat_mini: the time by which the
    whole slab is active is the first sample of the oracle's stored beat with v_min >= 50 mV."""
    from paper_2101_02959_gb300 import beat, build
    build.build()
    _, ref = _trace("beat_mini")
    t_all = ref[np.nonzero(ref[:, 2] >= 50.0)[0][0], 0]
    maps = {}
    steps = int(round((t_all + 4.0) / synth.TAU))
    recs = list(beat.run(synth.workload("beat_mini"), steps, maps=maps, record_every=40, precision="fp64",
                         ksp_rtol=1e-12, ksp_atol=0.0, snes_rtol=1e-10, snes_atol=1e-16))
    assert all(r["reason"] == 0 for r in recs)
    summ = beat.activation_summary(maps)
    assert summ["active_fraction"] == 1.0
    assert abs(summ["all_active_ms"] - t_all) < 1e-9


def test_checkpoint_resume_is_bit_exact(tmp_path):
    """A run checkpointed at step 5 and resumed in a new handle ends, after step 10, in
    exactly the state of the uninterrupted run (the solver keeps no hidden state across
    steps without the learned guess or a lagged preconditioner)."""
    from paper_2101_02959_gb300 import beat, binding, build
    build.build()
    w = synth.workload("cube8ve")
    opt = dict(precision="mixed", use_graphs=1)
    list(beat.run(w, 10, checkpoint=str(tmp_path / "full.npz"), checkpoint_every=10, **opt))
    list(beat.run(w, 10, checkpoint=str(tmp_path / "half.npz"), checkpoint_every=5, **opt))
    half = np.load(tmp_path / "half.npz")
    assert int(half["step"]) == 10
    import shutil
    list(beat.run(w, 5, checkpoint=str(tmp_path / "five.npz"), checkpoint_every=5, **opt))
    shutil.copy(tmp_path / "five.npz", tmp_path / "resume.npz")
    list(beat.run(w, 10, resume=str(tmp_path / "resume.npz"), checkpoint=str(tmp_path / "resumed.npz"),
                  checkpoint_every=5, **opt))
    full, resumed = np.load(tmp_path / "full.npz"), np.load(tmp_path / "resumed.npz")
    for k in ("ui", "ue", "w"):
        np.testing.assert_array_equal(resumed[k], full[k])
    assert float(resumed["t"]) == float(full["t"]) and int(resumed["step"]) == 10
