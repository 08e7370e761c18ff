"""schur_apply_noalloc: the S_hat x product without any device allocation.

Callers that must not allocate device memory while they apply the operator
(code under a fixed device-memory budget, or inside a host framework that owns
every allocation) use this entry point; its scratch is a fixed array compiled
into the library.  It must give the same result as schur_apply, call after call
(the shared scratch keeps the previous call's contents).
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,precision", [("cube8ve", "fp64"), ("ragged", "mixed")])
def test_noalloc_matches_schur_apply(name, precision):
    torch = pytest.importorskip("torch")
    from paper_2101_02959_gb300 import binding, build
    build.build()
    lib = binding.load()
    w = synth.workload(name)
    s = binding.Solver(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, precision=precision)
    n = s.sizes["n_iface"]
    x0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    y0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    # before the Jacobian exists the call is refused
    assert lib.schur_apply_noalloc(s._h, x0.data_ptr(), y0.data_ptr()) == -10
    N = s.N
    ui, ue, wv = synth.initial_state(N, 0)
    ui = ui + 20.0
    s.linearize(ui, ue, wv)
    for seed in (1, 2):  # two calls in a row with different inputs
        x = torch.from_numpy(synth.random_vector(n, seed)).cuda()
        ref = s.schur_apply(x)
        y = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        code = lib.schur_apply_noalloc(s._h, x.data_ptr(), y.data_ptr())
        assert code == 0, binding.ERRORS.get(code, code)
        rel = float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref))
        assert rel < 1e-9
        assert float((y - ref).abs().max() / ref.abs().max()) < 1e-9  # entry-wise too
    s.close()
