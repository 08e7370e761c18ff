"""The synthetic workloads use the values the paper prints (Table 1, Section 6)."""
import os

import numpy as np

import synth
from oracle import ionic

HERE = os.path.dirname(__file__)


def _golden(name):
    out = {}
    for line in open(os.path.join(HERE, "golden", name)):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_table1_parameters():
    g = _golden("table1_parameters.txt")
    assert synth.SIGMA_I == (g["sigma_l_i"], g["sigma_t_i"], g["sigma_n_i"])
    assert synth.SIGMA_E == (g["sigma_l_e"], g["sigma_t_e"], g["sigma_n_e"])
    for k in ("G", "eta1", "eta2", "vth", "vp", "chi_cm"):
        assert synth.IONIC[k] == g[k]
    assert synth.TAU == g["tau"]
    assert synth.STIMULUS["amp"] == g["stimulus_amp"]
    assert synth.STIMULUS["t_off"] - synth.STIMULUS["t_on"] == g["stimulus_duration"]
    # the printed bound rounds 1 / max(-dI/dv) = 0.366 up to 0.37
    v = np.linspace(0, 100, 100001)
    tmax = 1.0 / -ionic.di_ion_dv(v, 0.0, synth.IONIC).min()
    assert abs(tmax - g["tau_max_remark"]) < 0.005
