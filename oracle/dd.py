"""Oracle: BDDC and FETI-DP with deluxe scaling for the Jacobian system.

Follows Sections 4.1-4.4 of the paper, written with dense numpy/scipy blocks:

* local matrices K^(j) are subassembled from the elements of Omega_j only
  (local bilinear form a^(j), Section 4.1), ordered [interior; interface];
* static condensation: S_Gamma^(j) = K_GG - K_GI K_II^-1 K_IG; the interface
  system is S_hat u_G = f_hat with S_hat = sum_j R_j^T S^(j) R_j (the printed
  formula has a stray transpose);
* primal constraints through a change of basis (edge averages, see
  ``mesh.DofMaps``): Kbar^(j) = B^T K^(j) B, B = diag(I, T^(j)), ordered
  [I; Delta; Pi];
* deluxe scaling (Section 4.2): for a dual class C shared by the subdomains
  in N_C, S_C^(j) is the principal minor of the transformed S_Gamma^(j) on
  the dual dofs of C and D_C^(j) = (sum_{m in N_C} S_C^(m))^-1 S_C^(j);
  with scaling="rho" D_C^(j) is the diagonal rho-scaling of Section 4.2 instead;
* BDDC (Section 4.4): M^-1 = Rt_D^T St^-1 Rt_D with St^-1 from the paper's
  block-Cholesky formula: local solves with [[K_II, K_ID], [K_DI, K_DD]]
  plus the coarse term Phi S_PP^-1 Phi^T;
* FETI-DP (Section 4.3): F = B St^-1 B^T, d = B St^-1 f~,
  M^-1 = B_D St B_D^T, with fully redundant multipliers
  lambda_{jm} = u_j - u_m (j < m) on every dual dof, and B_D^T mapping
  lambda_{jm} to +D^(m) lambda_{jm} on Omega_j and -D^(j) lambda_{jm} on
  Omega_m, so that B_D^T B = P_D (eq. PdDeluxe).  f~ splits the global
  interface right-hand side equally among the subdomains sharing each node.

Lagged preconditioner (option, BDDC only; the paper rebuilds it at every
Newton step): with precond_every = k the local Schur operator is rebuilt at
every setup but the preconditioner (transformed local matrices, deluxe
blocks, coarse problem) only at every k-th, so PCG runs with the current
S_hat and an older BDDC preconditioner.  Two Jacobians differ only in the
lumped reaction term Kc = M (chi Cm + tau dI_ion/dv): with rho = Kc_new /
Kc_old nodewise (Kc > 0), alpha J_old <= J_new <= beta J_old for alpha =
min(1, min rho) and beta = max(1, max rho); the interface Schur complements
inherit the bounds (each is a minimum of the energy over interior
extensions), so cond(M_old^-1 S_new) <= (beta / alpha) cond(M_old^-1 S_old).
FETI-DP's operator contains St^-1 itself, so it cannot lag.

Gauge: the u_e dof of the gauge vertex is removed from the coarse problem
(fixed at zero), which makes S_hat and the coarse matrix nonsingular.

Pinned by: agreement with the direct sparse solve of the Jacobian; E_D^2 =
E_D; B_D^T B = P_D; eigenvalues of the BDDC-preconditioned operator >= 1 and
equal to the nonzero, non-unit eigenvalues of the FETI-DP operator (tests).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import ionic
from .krylov import gmres, lanczos_cond, pcg


class DDSolver:
    """Per-Newton-step BDDC / FETI-DP solver of J s = f (SoA vectors)."""

    def __init__(self, prob, method="bddc", krylov="pcg", rtol=1e-8, atol=1e-10,
                 dtol=1e4, maxit=1000, restart=30, scaling="deluxe", precond_every=1, keep_fetidp=True):
        """keep_fetidp=False drops the two local blocks that only FETI-DP's preconditioner
        reads (the transformed matrix and its interior factor): storage only, for large
        BDDC runs; the arithmetic is unchanged."""
        self.prob = prob
        self.keep_fetidp = keep_fetidp or method == "fetidp"
        self.method, self.krylov = method, krylov
        if scaling not in ("deluxe", "rho"):
            raise ValueError(scaling)
        if precond_every < 1 or (precond_every > 1 and method != "bddc"):
            raise ValueError("a lagged preconditioner needs BDDC and precond_every >= 1")
        self.precond_every = int(precond_every)
        self.n_setup = 0          # setups so far
        self.precond_fresh = False  # whether the last setup rebuilt the preconditioner
        self.scaling = scaling
        self.kw = dict(rtol=rtol, atol=atol, dtol=dtol, maxit=maxit)
        self.restart = restart
        p, d = prob.part, prob.dofs
        self.loc = []
        for j in range(p.n_sub):
            L = d.local(j)
            nodes = np.concatenate([L["interior_nodes"], L["iface_nodes"]])
            Ai, Ae, Ml = prob.fem.local(p.sub_elems[j], nodes)
            L.update(nodes=nodes, Ai=Ai, Ae=Ae, Ml=Ml, nI=2 * len(L["interior_nodes"]))
            self.loc.append(L)
        self.g_iface = 2 * d.gnode_to_iface[p.gauge_node] + 1
        self.dual_classes = [c for c in range(p.n_cls) if len(d.cls_dual_nodes[c]) > 0]
        self.last = {}

    # -- per Newton step: local matrices, Schur blocks, deluxe, coarse -------
    def setup(self, factor):
        """``factor`` = chi Cm + tau dI_ion/dv at every node."""
        prob, p, d = self.prob, self.prob.part, self.prob.dofs
        tau = prob.tau
        fresh = self.n_setup % self.precond_every == 0
        self.n_setup += 1
        self.precond_fresh = fresh
        for L in self.loc:
            n = len(L["nodes"])
            kc = L["Ml"] * factor[L["nodes"]]
            K = np.zeros((2 * n, 2 * n))
            K[0::2, 0::2] = tau * L["Ai"]
            K[1::2, 1::2] = tau * L["Ae"]
            idx = np.arange(n)
            K[2 * idx, 2 * idx] += kc
            K[2 * idx + 1, 2 * idx + 1] += kc
            K[2 * idx, 2 * idx + 1] -= kc
            K[2 * idx + 1, 2 * idx] -= kc
            nI = L["nI"]
            L["K"] = K
            L["KII"] = sla.cho_factor(K[:nI, :nI])
            if not fresh:
                continue  # operator only: the preconditioner below stays from an older setup
            KIG, KGG = K[:nI, nI:], K[nI:, nI:]
            S = KGG - KIG.T @ sla.cho_solve(L["KII"], KIG)
            L["S"] = S
            T = L["Tloc"]
            B = sla.block_diag(np.eye(nI), T)
            Kb = B.T @ K @ B
            nD = len(L["dual"])
            nID = nI + nD
            L["KbIDID"] = sla.cho_factor(Kb[:nID, :nID])
            if self.keep_fetidp:
                L["Kb"] = Kb
                L["KbII"] = sla.cho_factor(Kb[:nI, :nI])
            L["Sbar"] = T.T @ S @ T
            # coarse pieces (Section 4.4): solves with the I+Delta block
            KX = Kb[:nID, nID:]
            Y = sla.cho_solve(L["KbIDID"], KX)
            L["PhiD"] = -Y[nI:, :]
            L["SPPj"] = Kb[nID:, nID:] - KX.T @ Y
        if not fresh:
            return
        # coarse matrix, gauge dof removed
        nP = p.n_primal
        SPP = np.zeros((nP, nP))
        for L in self.loc:
            SPP[np.ix_(L["primal"], L["primal"])] += L["SPPj"]
        keep = np.ones(nP, bool)
        keep[p.gauge_primal] = False
        self.coarse_keep = keep
        self.SPP = SPP
        self.SPP_f = sla.cho_factor(SPP[np.ix_(keep, keep)])
        # deluxe blocks per dual class
        self.Dc = {}
        for c in self.dual_classes:
            subs = p.cls_subs[c]
            blocks = {}
            for j in subs:
                L = self.loc[j]
                r = self._class_range(j, c)
                blocks[j] = L["Sbar"][r, r]
            if self.scaling == "rho":
                self.Dc[c] = self._rho_blocks(c, subs, blocks)
                continue
            Ssum = sum(blocks.values())
            self.Dc[c] = {j: np.linalg.solve(Ssum, blocks[j]) for j in subs}

    def _rho_blocks(self, c, subs, blocks):
        """rho-scaling (Section 4.2): at a node of class c, field f in {i, e},
        delta_j = sigma_M^(j) / sum_{k in N_x} sigma_M^(k) with sigma_M the largest
        principal conductivity of that medium in subdomain k.  The conductivities are
        the same in every subdomain here, so delta_j = 1 / |N_x| for both fields."""
        fem = self.prob.fem
        sig = {0: max(fem.sigma_i), 1: max(fem.sigma_e)}  # per field, identical in every subdomain
        out = {}
        for j in subs:
            n = blocks[j].shape[0]
            w = np.array([sig[k % 2] / sum(sig[k % 2] for _ in subs) for k in range(n)])
            out[j] = np.diag(w)
        return out

    def _class_range(self, j, c):
        d = self.prob.dofs
        L = self.loc[j]
        start = d.cls_dual_start[c]
        n = 2 * len(d.cls_dual_nodes[c])
        pos = int(np.searchsorted(L["dual"], start))
        return slice(pos, pos + n)

    # -- St^-1 (block-Cholesky formula of Section 4.4) -----------------------
    def st_inv(self, rP, rD):
        """Apply St^-1 to (global primal rP, per-subdomain dual rD[j])."""
        p = self.prob.part
        coarse = rP.copy()
        for j, L in enumerate(self.loc):
            coarse[L["primal"]] += L["PhiD"].T @ rD[j]
        zP = np.zeros_like(rP)
        zP[self.coarse_keep] = sla.cho_solve(self.SPP_f, coarse[self.coarse_keep])
        zD = []
        for j, L in enumerate(self.loc):
            nI = L["nI"]
            rhs = np.concatenate([np.zeros(nI), rD[j]])
            zD.append(sla.cho_solve(L["KbIDID"], rhs)[nI:] + L["PhiD"] @ zP[L["primal"]])
        return zP, zD

    # -- BDDC ----------------------------------------------------------------
    def schur_apply(self, x):
        out = np.zeros_like(x)
        for L in self.loc:
            nI = L["nI"]
            K = L["K"]
            xj = x[L["R"]]
            y = K[nI:, nI:] @ xj - K[nI:, :nI] @ sla.cho_solve(L["KII"], K[:nI, nI:] @ xj)
            np.add.at(out, L["R"], y)
        out[self.g_iface] = 0.0
        return out

    def bddc_apply(self, r):
        d, p = self.prob.dofs, self.prob.part
        rb = d.T.T @ r
        rP = rb[d.n_dual:].copy()
        rP[p.gauge_primal] = 0.0
        rD = []
        for j, L in enumerate(self.loc):
            v = np.zeros(len(L["dual"]))
            for c in L["classes"]:
                if c in self.Dc:
                    rg = self._class_range(j, c)
                    s0 = d.cls_dual_start[c]
                    v[rg] = self.Dc[c][j].T @ rb[s0:s0 + (rg.stop - rg.start)]
            rD.append(v)
        zP, zD = self.st_inv(rP, rD)
        zb = np.zeros(d.n_dual + p.n_primal)
        zb[d.n_dual:] = zP
        for j, L in enumerate(self.loc):
            for c in L["classes"]:
                if c in self.Dc:
                    rg = self._class_range(j, c)
                    s0 = d.cls_dual_start[c]
                    zb[s0:s0 + (rg.stop - rg.start)] += self.Dc[c][j] @ zD[j][rg]
        z = d.T @ zb
        z[self.g_iface] = 0.0
        return z

    def e_d(self, w_loc):
        """Deluxe average E_D of per-subdomain transformed dual vectors."""
        d = self.prob.dofs
        out = [np.zeros_like(w) for w in w_loc]
        for c, D in self.Dc.items():
            n = 2 * len(d.cls_dual_nodes[c])
            avg = np.zeros(n)
            for j, Dj in D.items():
                avg += Dj @ w_loc[j][self._class_range(j, c)]
            for j in D:
                out[j][self._class_range(j, c)] = avg
        return out

    # -- condensation and interior recovery -----------------------------------
    def condense(self, f):
        """f_hat = f_G - sum_j R_j^T K_GI K_II^-1 f_I^(j) (global interface vector)."""
        d, p = self.prob.dofs, self.prob.part
        fG = np.zeros(d.n_iface)
        fG[0::2] = f[0][p.iface_nodes]
        fG[1::2] = f[1][p.iface_nodes]
        fI = []
        for L in self.loc:
            inodes = L["interior_nodes"]
            v = np.empty(2 * len(inodes))
            v[0::2], v[1::2] = f[0][inodes], f[1][inodes]
            fI.append(v)
            nI = L["nI"]
            y = L["K"][nI:, :nI] @ sla.cho_solve(L["KII"], v)
            np.add.at(fG, L["R"], -y)
        fG[self.g_iface] = 0.0
        return fG, fI

    def recover(self, uG, fI):
        N = self.prob.N
        s_i, s_e = np.zeros(N), np.zeros(N)
        p = self.prob.part
        s_i[p.iface_nodes] = uG[0::2]
        s_e[p.iface_nodes] = uG[1::2]
        for L, v in zip(self.loc, fI):
            nI = L["nI"]
            uI = sla.cho_solve(L["KII"], v - L["K"][:nI, nI:] @ uG[L["R"]])
            s_i[L["interior_nodes"]] = uI[0::2]
            s_e[L["interior_nodes"]] = uI[1::2]
        return s_i, s_e

    # -- FETI-DP -------------------------------------------------------------
    def _lambda_layout(self):
        p, d = self.prob.part, self.prob.dofs
        lay, start = [], 0
        for c in self.dual_classes:
            subs = p.cls_subs[c]
            n = 2 * len(d.cls_dual_nodes[c])
            for a in range(len(subs)):
                for b in range(a + 1, len(subs)):
                    lay.append((c, subs[a], subs[b], start, n))
                    start += n
        return lay, start

    def bt(self, lam, lay):
        w = [np.zeros(len(L["dual"])) for L in self.loc]
        for c, ja, jb, s0, n in lay:
            w[ja][self._class_range(ja, c)] += lam[s0:s0 + n]
            w[jb][self._class_range(jb, c)] -= lam[s0:s0 + n]
        return w

    def b(self, w, lay, nlam):
        lam = np.zeros(nlam)
        for c, ja, jb, s0, n in lay:
            lam[s0:s0 + n] = w[ja][self._class_range(ja, c)] - w[jb][self._class_range(jb, c)]
        return lam

    def bd_t(self, mu, lay):
        w = [np.zeros(len(L["dual"])) for L in self.loc]
        for c, ja, jb, s0, n in lay:
            w[ja][self._class_range(ja, c)] += self.Dc[c][jb] @ mu[s0:s0 + n]
            w[jb][self._class_range(jb, c)] -= self.Dc[c][ja] @ mu[s0:s0 + n]
        return w

    def bd(self, y, lay, nlam):
        mu = np.zeros(nlam)
        for c, ja, jb, s0, n in lay:
            mu[s0:s0 + n] = (self.Dc[c][jb].T @ y[ja][self._class_range(ja, c)]
                             - self.Dc[c][ja].T @ y[jb][self._class_range(jb, c)])
        return mu

    def sdd_apply(self, j, w):
        """Sbar_DD^(j) w as a Dirichlet solve on the transformed local matrix."""
        L = self.loc[j]
        nI = L["nI"]
        nD = len(L["dual"])
        Kb = L["Kb"]
        KDD = Kb[nI:nI + nD, nI:nI + nD]
        KDI = Kb[nI:nI + nD, :nI]
        return KDD @ w - KDI @ sla.cho_solve(L["KbII"], KDI.T @ w)

    def fetidp_operators(self):
        lay, nlam = self._lambda_layout()
        nP = self.prob.part.n_primal

        def F(lam):
            zP, zD = self.st_inv(np.zeros(nP), self.bt(lam, lay))
            return self.b(zD, lay, nlam)

        def Minv(mu):
            w = self.bd_t(mu, lay)
            y = [self.sdd_apply(j, w[j]) for j in range(len(self.loc))]
            return self.bd(y, lay, nlam)

        return F, Minv, lay, nlam

    def fetidp_rhs(self, f):
        """f~ (primal assembled, dual per subdomain) from the equal split of f."""
        d, p = self.prob.dofs, self.prob.part
        fG = np.zeros(d.n_iface)
        fG[0::2] = f[0][p.iface_nodes]
        fG[1::2] = f[1][p.iface_nodes]
        mult = np.repeat(p.mult[p.iface_nodes], 2).astype(float)
        fI = []
        rP = np.zeros(p.n_primal)
        rD = []
        for L in self.loc:
            inodes = L["interior_nodes"]
            v = np.empty(2 * len(inodes))
            v[0::2], v[1::2] = f[0][inodes], f[1][inodes]
            fI.append(v)
            nI = L["nI"]
            g = fG[L["R"]] / mult[L["R"]] - L["K"][nI:, :nI] @ sla.cho_solve(L["KII"], v)
            gb = L["Tloc"].T @ g
            nD = len(L["dual"])
            rD.append(gb[:nD])
            rP[L["primal"]] += gb[nD:]
        rP[p.gauge_primal] = 0.0
        return rP, rD, fI

    # -- the linear solve --------------------------------------------------------
    def solve(self, factor, f_i, f_e):
        self.setup(factor)
        f = (f_i, f_e)
        solver = pcg if self.krylov == "pcg" else gmres
        kw = dict(self.kw)
        if self.krylov == "gmres":
            kw["restart"] = self.restart
        if self.method == "bddc":
            fhat, fI = self.condense(f)
            uG, info = solver(self.schur_apply, self.bddc_apply, fhat, **kw)
        else:
            d, p = self.prob.dofs, self.prob.part
            F, Minv, lay, nlam = self.fetidp_operators()
            rP, rD, fI = self.fetidp_rhs(f)
            zP, zD = self.st_inv(rP, rD)
            dvec = self.b(zD, lay, nlam)
            lam, info = solver(F, Minv, dvec, **kw)
            btl = self.bt(lam, lay)
            wP, wD = self.st_inv(rP, [rD[j] - btl[j] for j in range(len(rD))])
            ub = np.zeros(d.n_dual + p.n_primal)
            cnt = np.zeros(d.n_dual)
            ub[d.n_dual:] = wP
            for j, L in enumerate(self.loc):
                ub[L["dual"]] += wD[j]
                cnt[L["dual"]] += 1.0
            ub[:d.n_dual] /= cnt
            uG = d.T @ ub
            uG[self.g_iface] = 0.0
        if self.krylov == "pcg" and info["its"] > 0:
            info["cond"] = lanczos_cond(info["alphas"], info["betas"])
        info["precond_fresh"] = self.precond_fresh
        s_i, s_e = self.recover(uG, fI)
        self.last = info
        return s_i, s_e, info

    def linsolve(self):
        """Callback for ``bidomain.newton``: (kc, f_i, f_e) -> (s_i, s_e, info)."""
        M = self.prob.fem.M

        def ls(kc, f_i, f_e):
            return self.solve(kc / M, f_i, f_e)
        return ls


def newton_factor(prob, ui, ue, w_next):
    """chi Cm + tau dI_ion/dv at every node (the Jacobian's pointwise factor)."""
    return prob.p["chi_cm"] + prob.tau * ionic.di_ion_dv(ui - ue, w_next, prob.p)
