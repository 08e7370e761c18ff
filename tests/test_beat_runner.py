"""Host logic of the whole-beat runner (Section 6, Test 4): the loop, the records and
Table 11's summary columns, with a stand-in solver handle (no GPU)."""
import numpy as np

import synth
from paper_2101_02959_gb300 import beat


class _FakeSolver:
    instances = []

    def __init__(self, w, sigma_i, sigma_e, ionic, tau, **opt):
        self.N = synth.n_nodes(w)
        self.opt = opt
        self.steps = 0
        self.closed = False
        self.stims = []
        _FakeSolver.instances.append(self)

    def set_state(self, ui, ue, w, t):
        assert len(ui) == self.N and t == 0.0

    def step(self, stim):
        self.steps += 1
        self.stims.append(stim)
        out = dict(newton_its=1 + self.steps % 2, krylov_its=10 * (1 + self.steps % 2), reason=0)
        if self.opt.get("fail_at") == self.steps:  # as the binding does: raise, with the step's stats
            raise beat.binding.BidomainError(-3, "bidomain_step", stats=dict(out, reason=-3))
        return out

    def get_state(self):
        # node x activates at step 3 + x and recovers at step 20 + 2 x (v in mV)
        k = self.steps
        x = np.arange(self.N)
        v = np.where((k >= 3 + x) & (k < 20 + 2 * x), 90.0, 0.0)
        return v + 1.0, np.ones(self.N), np.zeros(self.N), k * synth.TAU

    def close(self):
        self.closed = True


def test_run_records_and_summary(monkeypatch):
    monkeypatch.setattr(beat.binding, "Solver", _FakeSolver)
    w = synth.workload("ell8")
    recs = list(beat.run(w, 6, method="bddc"))
    fake = _FakeSolver.instances[-1]
    assert fake.closed and fake.steps == 6
    assert fake.stims[0] == synth.stimulus(w)  # the endocardium on the ellipsoid
    assert [r["step"] for r in recs] == [1, 2, 3, 4, 5, 6]
    assert abs(recs[-1]["t"] - 6 * synth.TAU) < 1e-15
    s = beat.summarize(recs)
    # newton its alternate 2, 1, ...: 9 in 6 steps; krylov 10 per Newton iteration
    assert s["steps"] == 6 and s["nlit"] == 1.5 and s["lit"] == 10.0 and s["failed"] == 0
    assert s["time_s"] >= 0.0


def test_run_stops_at_a_failed_step(monkeypatch):
    monkeypatch.setattr(beat.binding, "Solver", _FakeSolver)
    recs = list(beat.run(synth.workload("cube8ve"), 10, fail_at=3))
    assert len(recs) == 3 and recs[-1]["reason"] == -3
    assert recs[-1]["newton_its"] == 2 and recs[-1]["krylov_its"] == 20  # the failed step's own counts
    assert _FakeSolver.instances[-1].closed
    assert beat.summarize(recs)["failed"] == 1
    assert beat.summarize([])["steps"] == 0


def test_whole_beat_workloads_match_test4():
    """192x96x24 elements on 8x8x2 subdomains: 8,450 dofs per local problem (Section 6)."""
    for name, steps in (("beat_slab", 2400), ("beat_ell", 3400)):
        w = synth.workload(name)
        assert w["n"] == (192, 96, 24) and w["steps"] == steps
        nb = [w["n"][d] // w["s"][d] for d in range(3)]
        assert nb == [8, 8, 2]
        assert 2 * (w["s"][0] + 1) * (w["s"][1] + 1) * (w["s"][2] + 1) == 8450


def test_activation_and_recovery_maps(monkeypatch):
    """Sampled every 2 steps, node x (activating at step 3 + x, recovering at 20 + 2x)
    gets the first sample at or after each event; nodes still active keep NaN recovery."""
    monkeypatch.setattr(beat.binding, "Solver", _FakeSolver)
    w = dict(synth.workload("tiny"))
    maps = {}
    recs = list(beat.run(w, 40, maps=maps, record_every=2))
    assert len(recs) == 40
    act, rec = maps["activation"], maps["recovery"]
    N = len(act)
    x = np.arange(N)
    first = lambda k: 2 * np.ceil(k / 2.0)  # noqa: E731  first even step >= k
    seen = first(3 + x) <= 40
    np.testing.assert_allclose(act[seen], first(3 + x)[seen] * synth.TAU)
    assert np.all(np.isnan(act[~seen]))
    back = seen & (first(20 + 2 * x) <= 40)
    np.testing.assert_allclose(rec[back], first(20 + 2 * x)[back] * synth.TAU)
    assert np.all(np.isnan(rec[~back]))
    summ = beat.activation_summary(maps)
    assert np.isnan(summ["all_active_ms"]) == (not seen.all())
    assert abs(summ["active_fraction"] - seen.mean()) < 1e-15
    np.testing.assert_allclose(summ["mean_ari_ms"], np.mean((rec - act)[back]))


class _StateSolver(_FakeSolver):
    """Stand-in whose step is a deterministic function of the state alone."""

    def set_state(self, ui, ue, w, t):
        self.u = [np.array(ui, float), np.array(ue, float), np.array(w, float), float(t)]

    def step(self, stim):
        ui, ue, w, t = self.u
        self.u = [np.sin(ui) + 0.5 * ue, np.cos(ue) * 0.9, w * 0.99 + 0.01 * ui, t + synth.TAU]
        self.steps += 1
        return dict(newton_its=2, krylov_its=20, reason=0)

    def get_state(self):
        ui, ue, w, t = self.u
        return ui.copy(), ue.copy(), w.copy(), t


def test_checkpoint_and_resume_repeat_the_run(monkeypatch, tmp_path):
    monkeypatch.setattr(beat.binding, "Solver", _StateSolver)
    w = synth.workload("tiny")
    full_maps, part_maps = {}, {}
    full = list(beat.run(w, 12, maps=full_maps, record_every=2))
    ref = _StateSolver.instances[-1].get_state()
    ck = str(tmp_path / "beat.npz")
    first = list(beat.run(w, 12, maps=part_maps, record_every=2, checkpoint=ck, checkpoint_every=5))
    z = np.load(ck)
    assert int(z["step"]) == 10 and abs(float(z["t"]) - 10 * synth.TAU) < 1e-15
    resumed_maps = {}
    rest = list(beat.run(w, 12, maps=resumed_maps, record_every=2, resume=ck))
    assert [r["step"] for r in rest] == [11, 12]
    got = _StateSolver.instances[-1].get_state()
    for a, b in zip(got[:3], ref[:3]):
        np.testing.assert_array_equal(a, b)
    assert got[3] == ref[3]
    for k in ("activation", "recovery"):
        np.testing.assert_array_equal(resumed_maps[k], full_maps[k])
    assert len(full) == len(first) == 12


def test_checkpoint_refuses_hidden_state():
    import pytest
    w = synth.workload("tiny")
    with pytest.raises(ValueError):
        list(beat.run(w, 2, checkpoint="x.npz", checkpoint_every=1, learned_guess=1))
    with pytest.raises(ValueError):
        list(beat.run(w, 2, resume="x.npz", precond_every=2))


def test_resume_refuses_another_run(monkeypatch, tmp_path):
    """A checkpoint carries its workload, node count and options; resuming it with other
    ones, or recording maps it does not hold, is refused."""
    import pytest
    monkeypatch.setattr(beat.binding, "Solver", _StateSolver)
    w = synth.workload("tiny")
    ck = str(tmp_path / "beat.npz")
    list(beat.run(w, 4, checkpoint=ck, checkpoint_every=2, method="bddc"))
    rest = list(beat.run(w, 6, resume=ck, method="bddc"))
    assert [r["step"] for r in rest] == [5, 6]
    with pytest.raises(ValueError, match="method"):
        list(beat.run(w, 6, resume=ck, method="fetidp"))
    with pytest.raises(ValueError, match="workload"):
        list(beat.run(synth.workload("cube8"), 6, resume=ck, method="bddc"))
    with pytest.raises(ValueError, match="maps"):
        list(beat.run(w, 6, resume=ck, method="bddc", maps={}, record_every=2))
