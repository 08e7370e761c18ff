"""Pins for the oracle's BDDC / FETI-DP deluxe solvers and Krylov methods (Sections 4-5)."""
import numpy as np
import pytest

import synth
from conftest import oracle_problem
from oracle import ionic
from oracle.bidomain import direct_solve, time_step
from oracle.dd import DDSolver
from oracle.krylov import gmres, lanczos_cond, pcg


def _jacobian_system(prob, seed=0):
    ui, ue, w = synth.initial_state(prob.N, seed)
    ui = ui + 30.0 * np.exp(-np.sum(prob.mesh.coords ** 2, axis=1) / 0.01)
    w1 = ionic.gating_step(ui - ue, w, prob.tau, prob.p)
    r_i, r_e = prob.residual(ui, ue, w1, ui - 1.0, ue, prob.tau)
    kc = prob.kc(ui, ue, w1)
    return kc, -r_i, -r_e


@pytest.mark.parametrize("name,scaling", [("tiny", "deluxe"), ("cube8", "deluxe"), ("cube8ve", "deluxe"),
                                          ("ragged", "deluxe"), ("cube8ve", "rho"), ("shell_small", "deluxe")])
@pytest.mark.parametrize("method", ["bddc", "fetidp"])
@pytest.mark.parametrize("krylov", ["pcg", "gmres"])
def test_dd_matches_direct(name, scaling, method, krylov):
    prob = oracle_problem(name)
    kc, f_i, f_e = _jacobian_system(prob)
    si, se, _ = direct_solve(prob, kc, f_i, f_e)
    dd = DDSolver(prob, method=method, krylov=krylov, rtol=1e-13, atol=0.0, scaling=scaling)
    ai, ae, info = dd.solve(kc / prob.fem.M, f_i, f_e)
    assert info["reason"] == "converged"
    err = np.linalg.norm(np.r_[ai - si, ae - se]) / np.linalg.norm(np.r_[si, se])
    assert err < 1e-10


def _local_dual_vectors(dd, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(len(L["dual"])) for L in dd.loc]


@pytest.mark.parametrize("name,scaling", [("cube8", "deluxe"), ("cube8ve", "deluxe"), ("ragged", "deluxe"),
                                          ("cube8ve", "rho"), ("ragged", "rho"), ("shell_small", "deluxe")])
def test_deluxe_projection_and_pd(name, scaling):
    prob = oracle_problem(name)
    kc, _, _ = _jacobian_system(prob)
    dd = DDSolver(prob, scaling=scaling)
    dd.setup(kc / prob.fem.M)
    w = _local_dual_vectors(dd, 5)
    e1 = dd.e_d(w)
    e2 = dd.e_d(e1)
    for a, b in zip(e1, e2):
        np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-12)
    # B_D^T B = P_D = I - E_D (eq. PdDeluxe) for fully redundant multipliers
    lay, nlam = dd._lambda_layout()
    pd = dd.bd_t(dd.b(w, lay, nlam), lay)
    for a, x, e in zip(pd, w, e1):
        np.testing.assert_allclose(a, x - e, rtol=1e-9, atol=1e-12)


def _dense(apply, n, keep):
    A = np.zeros((n, n))
    for k in np.nonzero(keep)[0]:
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = apply(e)
    return A[np.ix_(keep, keep)]


@pytest.mark.parametrize("name,scaling", [("cube8", "deluxe"), ("cube8ve", "deluxe"), ("cube8ve", "rho")])
def test_bddc_fetidp_spectra(name, scaling):
    """BDDC eigenvalues are >= 1; FETI-DP has the same ones apart from 0 and 1."""
    prob = oracle_problem(name)
    kc, _, _ = _jacobian_system(prob)
    dd = DDSolver(prob, scaling=scaling)
    dd.setup(kc / prob.fem.M)
    n = prob.dofs.n_iface
    keep = np.ones(n, bool)
    keep[dd.g_iface] = False
    S = _dense(dd.schur_apply, n, keep)
    Minv = _dense(dd.bddc_apply, n, keep)
    ev_b = np.sort(np.linalg.eigvals(Minv @ S).real)
    assert ev_b[0] > 1.0 - 1e-8
    F, Mf, lay, nlam = dd.fetidp_operators()
    allk = np.ones(nlam, bool)
    Fm = _dense(F, nlam, allk)
    Mm = _dense(Mf, nlam, allk)
    ev_f = np.sort(np.linalg.eigvals(Mm @ Fm).real)
    big_b = ev_b[ev_b > 1.0 + 1e-6]
    big_f = ev_f[ev_f > 1.0 + 1e-6]
    assert len(big_b) == len(big_f)
    np.testing.assert_allclose(big_b, big_f, rtol=1e-7)


def test_primal_space_ordering_of_cond():
    """A richer primal space gives a smaller condition number (Table 7: V > V+E >= V+E+F)."""
    conds, sols = {}, {}
    for prim in ("V", "VE", "VEF"):
        prob = oracle_problem("cube8", prim)
        kc, f_i, f_e = _jacobian_system(prob)
        dd = DDSolver(prob, rtol=1e-10, atol=0.0)
        si, se, info = dd.solve(kc / prob.fem.M, f_i, f_e)
        conds[prim] = info["cond"]
        sols[prim] = np.concatenate([si, se])
    assert 1.0 <= conds["VEF"] <= conds["VE"] * (1 + 1e-6) and conds["VE"] < conds["V"]
    # every primal space solves the same Jacobian system
    for prim in ("V", "VEF"):
        assert np.linalg.norm(sols[prim] - sols["VE"]) <= 1e-8 * np.linalg.norm(sols["VE"])


def test_vef_primal_counts_and_change_of_basis():
    """V+E+F on the 8^3 grid with 2x2x2 subdomains: 1 vertex, 6 edges (4 nodes), 12 faces
    (16 nodes) -> 19 primal classes (38 primal dofs) and 12*15 + 6*3 = 198 dual nodes; the
    change of basis reproduces nodal values: T [d; a] has class mean a and deviations d."""
    prob = oracle_problem("cube8", "VEF")
    part, dofs = prob.part, prob.dofs
    assert part.n_primal == 38
    assert dofs.n_dual == 2 * 198
    T = dofs.T
    # a constant field on every class maps to its own average with zero deviations
    rng = np.random.default_rng(3)
    z = rng.standard_normal(T.shape[1])
    u = T @ z
    for c in part.primal_cls:
        nodes = part.cls_nodes[c]
        for f in range(2):
            vals = u[2 * dofs.gnode_to_iface[nodes] + f]
            a = z[dofs.n_dual + 2 * part.primal_index[c] + f]
            assert abs(vals.mean() - a) < 1e-12


def test_pcg_gmres_lanczos_small_spd():
    rng = np.random.default_rng(2)
    n = 12
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.linspace(1.0, 40.0, n)
    A = Q @ np.diag(ev) @ Q.T
    b = rng.standard_normal(n)
    x, info = pcg(lambda v: A @ v, lambda v: v, b, rtol=1e-14, atol=0.0, maxit=50)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9)
    assert info["its"] <= n + 2
    # after n steps the Lanczos matrix holds the whole spectrum
    _, info_n = pcg(lambda v: A @ v, lambda v: v, b, rtol=0.0, atol=0.0, maxit=n)
    assert abs(lanczos_cond(info_n["alphas"][:n], info_n["betas"][:n - 1]) - 40.0) < 1e-6
    N = rng.standard_normal((n, n)) + 5 * np.eye(n)
    x, info = gmres(lambda v: N @ v, lambda v: v, b, rtol=1e-13, atol=0.0, restart=5, maxit=200)
    np.testing.assert_allclose(x, np.linalg.solve(N, b), rtol=1e-8)


def test_rho_scaling_is_multiplicity_here():
    """With equal conductivities in every subdomain the rho weights are 1 / |N_x|
    (Section 4.2): on the 8^3 cube a face is shared by 2, an edge by 4 subdomains."""
    prob = oracle_problem("cube8ve")
    kc, _, _ = _jacobian_system(prob)
    dd = DDSolver(prob, scaling="rho")
    dd.setup(kc / prob.fem.M)
    for c, D in dd.Dc.items():
        k = len(prob.part.cls_subs[c])
        for Dj in D.values():
            np.testing.assert_allclose(Dj, np.eye(Dj.shape[0]) / k, rtol=0, atol=1e-15)


def _factor(prob, seed, bump):
    ui, ue, w = synth.initial_state(prob.N, seed)
    ui = ui + bump * np.exp(-np.sum(prob.mesh.coords ** 2, axis=1) / 0.01)
    w1 = ionic.gating_step(ui - ue, w, prob.tau, prob.p)
    r_i, r_e = prob.residual(ui, ue, w1, ui - 1.0, ue, prob.tau)
    return prob.kc(ui, ue, w1), -r_i, -r_e


def test_lagged_preconditioner_solution_and_spectral_bound():
    """precond_every = 2: the second solve runs the current Schur operator with the first
    setup's preconditioner.  It still reaches the direct solution, and its eigenvalues lie
    in [alpha lmin, beta lmax] of the fresh pair, alpha, beta from the ratio of the
    lumped reaction terms (Loewner bounds inherited by the Schur complements)."""
    prob = oracle_problem("cube8ve")
    kc_old, _, _ = _factor(prob, 0, 0.0)
    kc_new, f_i, f_e = _factor(prob, 1, 60.0)
    rho = kc_new / kc_old
    assert rho.min() > 0
    alpha, beta = min(1.0, rho.min()), max(1.0, rho.max())
    # chi Cm + tau dI_ion/dv stays within about 0.8 .. 1.07 for tau = 0.05 ms, which is why
    # an older preconditioner stays close; the upstroke bump uses most of that range
    assert beta / alpha > 1.2
    lag = DDSolver(prob, rtol=1e-13, atol=0.0, precond_every=2)
    lag.solve(kc_old / prob.fem.M, f_i, f_e)
    assert lag.last["precond_fresh"]
    ai, ae, info = lag.solve(kc_new / prob.fem.M, f_i, f_e)
    assert not info["precond_fresh"] and info["reason"] == "converged"
    si, se, _ = direct_solve(prob, kc_new, f_i, f_e)
    assert np.linalg.norm(np.r_[ai - si, ae - se]) < 1e-10 * np.linalg.norm(np.r_[si, se])
    # dense spectra: M_old^-1 S_new against M_old^-1 S_old
    old = DDSolver(prob)
    old.setup(kc_old / prob.fem.M)
    n = prob.dofs.n_iface
    keep = np.ones(n, bool)
    keep[old.g_iface] = False
    Minv = _dense(old.bddc_apply, n, keep)
    ev_old = np.sort(np.linalg.eigvals(Minv @ _dense(old.schur_apply, n, keep)).real)
    ev_new = np.sort(np.linalg.eigvals(Minv @ _dense(lag.schur_apply, n, keep)).real)
    assert ev_new[0] >= alpha * ev_old[0] * (1 - 1e-8)
    assert ev_new[-1] <= beta * ev_old[-1] * (1 + 1e-8)
    assert info["cond"] <= (ev_new[-1] / ev_new[0]) * (1 + 1e-6)
    # the third setup rebuilds it again
    lag.solve(kc_new / prob.fem.M, f_i, f_e)
    assert lag.last["precond_fresh"]


def test_lagged_preconditioner_only_for_bddc():
    prob = oracle_problem("cube8ve")
    with pytest.raises(ValueError):
        DDSolver(prob, method="fetidp", precond_every=2)
    with pytest.raises(ValueError):
        DDSolver(prob, precond_every=0)


def test_lagged_preconditioner_time_steps():
    """Through the stimulus-driven upstroke, rebuilding the preconditioner only every
    4th Jacobian gives the same states (Krylov and Newton tightened) and, at the paper's
    tolerances, at most a few more Krylov iterations per solve."""
    prob = oracle_problem("cube8ve")
    states, its = {}, {}
    for k in (1, 4):
        for tight in (True, False):
            kw = dict(rtol=1e-12, atol=0.0) if tight else {}
            nkw = dict(rtol=1e-10, atol=1e-16) if tight else {}
            dd = DDSolver(prob, precond_every=k, **kw)
            ui, ue, w = synth.initial_state(prob.N, 0)
            lits = []
            for n in range(4):
                ui, ue, w, st = time_step(prob, ui, ue, w, n, dd.linsolve(), **nkw)
                lits += st["krylov_its"]
            states[k, tight] = (ui, ue)
            its[k, tight] = np.array(lits)
            assert dd.n_setup == len(lits)
    a, b = states[1, True], states[4, True]
    assert np.linalg.norm(a[0] - b[0]) < 1e-9 * np.linalg.norm(a[0])
    assert np.linalg.norm(a[1] - b[1]) < 1e-9 * np.linalg.norm(a[1])
    fresh, lag = its[1, False], its[4, False]
    assert len(fresh) == len(lag)
    assert lag.max() <= fresh.max() + 3


def test_masked_shell_has_uneven_subdomains_and_promoted_vertices():
    """The masked shell (the uneven batch): subdomains are the connected pieces of the
    blocks inside the wall, of very different sizes; every one has a vertex on its
    interface after the promotion rule, and the promoted vertices are exactly the lowest
    nodes of the edge classes of the fragments that had none."""
    from oracle.mesh import VERTEX, Mesh, Partition
    prob = oracle_problem("shell_small")
    p = prob.part
    sizes = np.array([len(x) for x in p.sub_nodes])
    assert sizes.min() * 5 < sizes.max()
    assert all(any(p.cls_type[c] == VERTEX for c in p.sub_classes(j)) for j in range(p.n_sub))
    w = prob.workload
    orig = Partition._promote_vertices  # the classes without the promotion rule, for comparison
    try:
        Partition._promote_vertices = lambda self, classes, adj: classes
        raw = Partition(Mesh(w["n"], w["l"], elem_mask=w["mask"]), w["s"], "VE")
    finally:
        Partition._promote_vertices = orig
    lacking = [j for j in range(raw.n_sub) if not any(raw.cls_type[c] == VERTEX for c in raw.sub_classes(j))]
    assert lacking
    new_vertices = {int(p.cls_nodes[c][0]) for c in range(p.n_cls) if p.cls_type[c] == VERTEX} - \
        {int(raw.cls_nodes[c][0]) for c in range(raw.n_cls) if raw.cls_type[c] == VERTEX}
    expect = set()
    for j in lacking:  # in subdomain order, as the rule applies
        mine = [c for c in range(raw.n_cls) if j in raw.cls_subs[c] and raw.cls_type[c] == 1]
        expect |= {int(raw.cls_nodes[c][0]) for c in mine}
    assert new_vertices <= expect and new_vertices
