"""Oracle: Rogers-McCulloch ionic model and the Step-1 gating update.

Section 2: I_ion(v, w) = G v (1 - v/v_th)(1 - v/v_p) + eta1 v w and
R(v, w) = eta2 (v/v_p - w), with v the potential measured from rest.
Section 3b, Step 1: w^{n+1} - tau R(v^n, w^{n+1}) = w^n; R is linear in w, so
w^{n+1} = (w^n + tau eta2 v^n / v_p) / (1 + tau eta2).

Pinned by: the closed form above, a finite-difference check of dI_ion/dv, and
the remark after the coercivity lemma (chi Cm + tau dI/dv > 0 for every v iff
tau < 0.37 ms with chi Cm = 1, w = 0).
"""
from __future__ import annotations


def i_ion(v, w, p):
    return p["G"] * v * (1.0 - v / p["vth"]) * (1.0 - v / p["vp"]) + p["eta1"] * v * w


def di_ion_dv(v, w, p):
    """d I_ion / d v, differentiated by hand from the product form."""
    a, b = 1.0 / p["vth"], 1.0 / p["vp"]
    return p["G"] * (1.0 - 2.0 * v * (a + b) + 3.0 * v * v * a * b) + p["eta1"] * w


def gating_step(v_n, w_n, tau, p):
    """Backward-Euler gating update of Step 1 (closed form, R linear in w)."""
    return (w_n + tau * p["eta2"] * v_n / p["vp"]) / (1.0 + tau * p["eta2"])
