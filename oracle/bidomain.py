"""Oracle: the segregated implicit Bidomain time step (Sections 3b and 3c).

Unknowns u = [u_i; u_e] (SoA blocks), v = u_i - u_e measured from rest.

Step 2 residual (Section 3b):
  F(u) = (chi Cm Mcal + tau Acal) u + tau [M I_ion(v, w^{n+1}); -M I_ion(v, w^{n+1})]
  G    = chi Cm Mcal u^n + tau [M I_app; -M I_app]
with Acal = diag(A_i, A_e), Mcal = [[M, -M], [-M, M]] and lumped M.

Stimulus reading: the paper puts I_app only in the u_e equation yet asks its
integral to vanish and applies 100 mA/cm^3 locally.  It is read here as a
transmembrane current entering both equations with opposite signs, which keeps
(1,1)^T G = 0, active while t_on <= t_{n+1} < t_off on the nodes inside the
stimulus box.  The box is in the grid's parametric coordinates: cm for a box
geometry, (phi, theta, r) for the ellipsoid, where r = 0 selects the
endocardial surface that Section 6 stimulates.

Jacobian (Section 3c, exact Newton at the current iterate):
  J = [[Kc + tau A_i, -Kc], [-Kc, Kc + tau A_e]],  Kc = diag(M_l (chi Cm + tau dI_ion/dv)).
J (1,1) = 0.  Gauge: the u_e correction at the partition's gauge vertex is
held at zero (row and column removed), and after every step both potentials
are shifted so that u_e has zero lumped-mass mean (v is unchanged).

Newton (Section 6: PETSc SNES defaults): stop when ||F - G|| <= max(atol,
rtol ||F(u^0) - G||) or when ||lambda s|| <= stol ||u||; cubic backtracking
line search of Dennis and Schnabel (Algorithm A6.3.1) on f = ||F - G||^2 / 2
with slope -||F - G||^2 and alpha = 1e-4.

Pinned by: the direct sparse solve (a library primitive) against which the
DD solvers are checked; (1,1)^T (F - G) = 0; u^{n+1} = u^n at rest with no
stimulus; the Jacobian against central finite differences of F.
"""
from __future__ import annotations

import numpy as np

from . import ionic
from .fem import FEM
from .mesh import DofMaps, Mesh, Partition


class Problem:
    def __init__(self, w, sigma_i, sigma_e, ionic_p, tau, stimulus):
        self.workload = w
        self.mesh = Mesh(w["n"], w.get("l"), elem_mask=w.get("mask"), ellipsoid=w.get("ellipsoid"))
        self.part = Partition(self.mesh, w["s"], w.get("primal", "V"))
        self.dofs = DofMaps(self.part)
        self.fem = FEM(self.mesh, sigma_i, sigma_e)
        self.p = dict(ionic_p)
        self.tau = float(tau)
        self.stim = dict(stimulus)
        b = self.stim["box"]
        c = self.mesh.pcoords  # the box is in parametric coordinates (the grid's own for a box)
        eps = 1e-12
        self.stim_mask = ((c[:, 0] >= b[0] - eps) & (c[:, 0] <= b[1] + eps)
                          & (c[:, 1] >= b[2] - eps) & (c[:, 1] <= b[3] + eps)
                          & (c[:, 2] >= b[4] - eps) & (c[:, 2] <= b[5] + eps))
        self.N = self.mesh.n_node

    # -- Step 2 pieces -------------------------------------------------------
    def i_app(self, t_next):
        on = self.stim["t_on"] <= t_next < self.stim["t_off"]
        return np.where(self.stim_mask, self.stim["amp"] if on else 0.0, 0.0)

    def residual(self, ui, ue, w_next, ui_n, ue_n, t_next):
        """F(u) - G as (r_i, r_e)."""
        p, tau, M = self.p, self.tau, self.fem.M
        v, v_n = ui - ue, ui_n - ue_n
        cap = p["chi_cm"] * M * (v - v_n)
        ion = tau * M * ionic.i_ion(v, w_next, p)
        app = tau * M * self.i_app(t_next)
        r_i = cap + tau * (self.fem.A_i @ ui) + ion - app
        r_e = -cap + tau * (self.fem.A_e @ ue) - ion + app
        return r_i, r_e

    def kc(self, ui, ue, w_next):
        """Diagonal coupling Kc = M (chi Cm + tau dI_ion/dv) of the Jacobian."""
        p = self.p
        return self.fem.M * (p["chi_cm"] + self.tau * ionic.di_ion_dv(ui - ue, w_next, p))

    def jacobian(self, kc):
        import scipy.sparse as sp
        K = sp.diags(kc)
        return sp.bmat([[K + self.tau * self.fem.A_i, -K], [-K, K + self.tau * self.fem.A_e]]).tocsr()


def direct_solve(prob: Problem, kc, f_i, f_e):
    """Solve J s = f with the gauge dof removed (sparse LU, a library primitive)."""
    import scipy.sparse.linalg as spla
    N = prob.N
    J = prob.jacobian(kc)
    g = N + prob.part.gauge_node
    keep = np.ones(2 * N, bool)
    keep[g] = False
    f = np.concatenate([f_i, f_e])
    s = np.zeros(2 * N)
    s[keep] = spla.spsolve(J[keep][:, keep].tocsc(), f[keep])
    return s[:N], s[N:], dict(its=0)


def line_search_bt(fnorm2, trial, alpha=1e-4, minlambda=1e-12, maxsteps=40):
    """Cubic backtracking (Dennis & Schnabel A6.3.1) on f = ||R||^2/2.

    ``trial(lam)`` returns ||R(u + lam s)||^2.  Returns (lam, new_norm2, ok).
    """
    f0 = 0.5 * fnorm2
    slope = -fnorm2
    lam = 1.0
    g = trial(lam)
    if 0.5 * g <= f0 + alpha * lam * slope:
        return lam, g, True
    lam_prev, f_prev = lam, 0.5 * g
    lam_t = -slope / (2.0 * (0.5 * g - f0 - slope))
    lam = max(min(lam_t, 0.5 * lam), 0.1 * lam)
    for _ in range(maxsteps):
        if lam < minlambda:
            return lam, g, False
        g = trial(lam)
        fl = 0.5 * g
        if fl <= f0 + alpha * lam * slope:
            return lam, g, True
        t1 = fl - f0 - lam * slope
        t2 = f_prev - f0 - lam_prev * slope
        d = lam - lam_prev
        a = (t1 / lam ** 2 - t2 / lam_prev ** 2) / d
        b = (-lam_prev * t1 / lam ** 2 + lam * t2 / lam_prev ** 2) / d
        if a == 0.0:
            lam_t = -slope / (2.0 * b)
        else:
            disc = b * b - 3.0 * a * slope
            lam_t = (-b + np.sqrt(max(disc, 0.0))) / (3.0 * a)
        lam_prev, f_prev = lam, fl
        lam = max(min(lam_t, 0.5 * lam), 0.1 * lam)
    return lam, g, False


def newton(prob: Problem, ui_n, ue_n, w_next, t_next, linsolve, rtol=1e-4, atol=1e-8,
           stol=1e-8, maxit=50, u0=None):
    """Newton iteration for F(u) = G (Section 3c)."""
    ui, ue = (ui_n.copy(), ue_n.copy()) if u0 is None else (u0[0].copy(), u0[1].copy())
    r_i, r_e = prob.residual(ui, ue, w_next, ui_n, ue_n, t_next)
    fn2 = float(r_i @ r_i + r_e @ r_e)
    fn0 = np.sqrt(fn2)
    stats = dict(newton_its=0, krylov_its=[], res0=fn0, reason="")
    for k in range(maxit):
        if np.sqrt(fn2) <= max(atol, rtol * fn0):
            stats["reason"] = "fnorm"
            break
        kc = prob.kc(ui, ue, w_next)
        s_i, s_e, ls = linsolve(kc, -r_i, -r_e)
        stats["krylov_its"].append(ls.get("its", 0))

        def trial(lam):
            a, b = prob.residual(ui + lam * s_i, ue + lam * s_e, w_next, ui_n, ue_n, t_next)
            return float(a @ a + b @ b)

        lam, fn2_new, ok = line_search_bt(fn2, trial)
        ui = ui + lam * s_i
        ue = ue + lam * s_e
        stats["newton_its"] = k + 1
        r_i, r_e = prob.residual(ui, ue, w_next, ui_n, ue_n, t_next)
        fn2 = float(r_i @ r_i + r_e @ r_e)
        if not ok:
            stats["reason"] = "linesearch"
            break
        snorm = lam * np.sqrt(float(s_i @ s_i + s_e @ s_e))
        unorm = np.sqrt(float(ui @ ui + ue @ ue))
        if snorm <= stol * unorm:
            stats["reason"] = "snorm"
            break
    else:
        stats["reason"] = "maxit"
    stats["res_final"] = np.sqrt(fn2)
    return ui, ue, stats


def gauge_shift(prob: Problem, ui, ue):
    """Shift both potentials so that u_e has zero lumped-mass mean."""
    M = prob.fem.M
    c = float(M @ ue) / float(M.sum())
    return ui - c, ue - c


def time_step(prob: Problem, ui, ue, w, n, linsolve, **newton_kw):
    """One decoupled backward-Euler step from t_n = n tau (Steps 1 and 2)."""
    t_next = (n + 1) * prob.tau
    w_next = ionic.gating_step(ui - ue, w, prob.tau, prob.p)
    ui1, ue1, st = newton(prob, ui, ue, w_next, t_next, linsolve, **newton_kw)
    ui1, ue1 = gauge_shift(prob, ui1, ue1)
    return ui1, ue1, w_next, st
