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


def _rows(name):
    out = {}
    for line in open(os.path.join(HERE, "golden", name)):
        if line.strip() and not line.startswith("#"):
            prim, scaling, its, cond = line.split()
            out[prim, scaling] = (float(its), float(cond))
    return out


def test_ellipsoid_optimality_against_table8():
    """The oracle on the truncated ellipsoid (4^3 subdomains, H/h = 8; stored by
    tests/golden/make_ellipsoid_optimality.py) against Table 8's first row.  The paper
    averages 40 steps of activation on its own axes; the stored run is one Newton step
    from rest on the axes read here, so only the shape is compared: a richer primal
    space lowers cond (V >> V+E >= V+E+F), rho and deluxe agree closely on this
    homogeneous medium as in the table, and V+E, V+E+F land within 30 % (cond) and
    3 iterations of the printed values."""
    paper = _rows("table8_ellipsoid_h8.txt")
    ours = _rows("ellipsoid_optimality_h8.txt")
    assert set(paper) == set(ours)
    for sc in ("deluxe", "rho"):
        assert ours["V", sc][1] > 5 * ours["VE", sc][1]
        assert ours["VE", sc][1] >= ours["VEF", sc][1] * (1 - 1e-6)
        for prim in ("VE", "VEF"):
            its, cond = ours[prim, sc]
            pits, pcond = paper[prim, sc]
            assert abs(cond - pcond) <= 0.3 * pcond
            assert abs(its - pits) <= 3
    for prim in ("V", "VE", "VEF"):
        a, b = ours[prim, "deluxe"][1], ours[prim, "rho"][1]
        assert abs(a - b) <= 0.05 * a


def test_whole_beat_trace_activates_and_recovers():
    """The oracle's stored whole beat (tests/golden/make_whole_beat_trace.py) on a
    0.2 x 0.2 x 0.05 cm slab: the corner stimulus activates the whole domain within a few
    ms, the plateau stays below v_p = 100 mV (the excited rest point of Rogers-McCulloch),
    and by 120 ms the tissue is back at rest, the activation-recovery interval Section 6
    gives for the slab's whole beat with this model."""
    rows = []
    for line in open(os.path.join(HERE, "golden", "whole_beat_beat_mini.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    rows = np.array(rows)
    t, nit, vmin, vmax = rows[:, 0], rows[:, 1], rows[:, 2], rows[:, 3]
    assert abs(t[-1] - 120.0) < 1e-9 and len(rows) == 60
    active = np.nonzero(vmin > 50.0)[0]
    assert len(active) > 0 and t[active[0]] <= 10.0
    assert vmax.max() < 100.0 and vmax.max() > 90.0
    assert vmax[-1] < 1.0 and abs(vmin[-1]) < 1.0
    assert nit.max() <= 3


def test_ellipsoid_optimality_growth_to_h12():
    """From H/h = 8 to 12 (Table 8, V+E deluxe) the condition number grows like the
    (1 + log(H/h))^2 bound: the oracle's growth ratio is within 10 % of the table's, and
    its H/h = 12 values within 30 % (cond) and 3 iterations of the printed ones."""
    p8, p12 = _rows("table8_ellipsoid_h8.txt"), _rows("table8_ellipsoid_h12.txt")
    o8, o12 = _rows("ellipsoid_optimality_h8.txt"), _rows("ellipsoid_optimality_h12.txt")
    k = ("VE", "deluxe")
    paper_growth = p12[k][1] / p8[k][1]
    ours_growth = o12[k][1] / o8[k][1]
    assert ours_growth > 1.0 and abs(ours_growth - paper_growth) <= 0.1 * paper_growth
    assert abs(o12[k][1] - p12[k][1]) <= 0.3 * p12[k][1]
    assert abs(o12[k][0] - p12[k][0]) <= 3
