"""Host logic of the whole-beat runner (Section 6, Test 4): the loop, the records and
Table 11's summary columns, with a stand-in solver handle (no GPU)."""
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
        fail = self.opt.get("fail_at") == self.steps
        return dict(newton_its=1 + self.steps % 2, krylov_its=10 * (1 + self.steps % 2), reason=-3 if fail else 0)

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
