"""GPU parity: every step of the path through the C-ABI against the CPU oracle.

Tolerances (relative): every comparison below checks both the 2-norm of the
difference against the 2-norm of the oracle's vector and the largest entry of the
difference against the oracle's largest entry, so an error confined to a few entries
(a handful of interface dofs under a large bump) cannot hide in the norm:
  pointwise kernels (gating, residual)            1e-12
  operator applications (S_hat, BDDC, FETI-DP)    1e-9   (FP64; K_II^-1 and the coarse solve
                                                          amplify rounding by their condition numbers)
  Jacobian solve, FP64                            1e-10  with Krylov iterations within +-1
  time step, FP64 / mixed                         1e-9 / 1e-8 in v and u_e
"""
import numpy as np
import pytest

import synth
from conftest import oracle_problem
from oracle import ionic
from oracle.bidomain import direct_solve, time_step
from oracle.dd import DDSolver

pytestmark = pytest.mark.gpu


def _solver(name, **opt):
    from paper_2101_02959_gb300 import binding, build
    build.build()
    w = synth.workload(name)
    return binding.Solver(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, **opt)


def _state(prob, seed=0):
    ui, ue, w = synth.initial_state(prob.N, seed)
    # a bump at the grid's origin corner (parametric coordinates on the ellipsoid)
    ui = ui + 30.0 * np.exp(-np.sum((prob.mesh.pcoords - np.array(prob.mesh.origin)) ** 2, axis=1) / 0.01)
    ue = ue + 0.5 * synth.random_vector(prob.N, seed + 11)
    w = 0.01 * np.abs(synth.random_vector(prob.N, seed + 12))
    return ui + ue, ue, w


def _rel(a, b):
    """max(||a - b||_2 / ||b||_2, max|a - b| / max|b|): the 2-norm and the entry-wise error."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    d = a - b
    two = np.linalg.norm(d) / max(np.linalg.norm(b), 1e-300)
    inf = np.max(np.abs(d)) / max(np.max(np.abs(b)), 1e-300) if d.size else 0.0
    return max(two, inf)


@pytest.mark.parametrize("name", ["tiny", "ragged", "ell10"])
def test_gating_and_residual(name):
    prob = oracle_problem(name)
    s = _solver(name)
    ui, ue, w = _state(prob)
    wn = s.gating(ui, ue, w)
    assert _rel(wn, ionic.gating_step(ui - ue, w, prob.tau, prob.p)) < 1e-14
    for t_next in (0.5, 2.0):  # stimulus on / off
        r = s.residual(synth.stimulus(prob.workload), t_next, ui, ue, wn, ui * 0.99, ue + 0.1)
        ri, re = prob.residual(ui, ue, wn, ui * 0.99, ue + 0.1, t_next)
        assert _rel(r, np.concatenate([ri, re])) < 1e-12


def _linearized(name, **opt):
    prob = oracle_problem(name)
    s = _solver(name, **opt)
    ui, ue, w = _state(prob)
    wn = ionic.gating_step(ui - ue, w, prob.tau, prob.p)
    s.linearize(ui, ue, wn)
    dd = DDSolver(prob, scaling=opt.get("scaling", "deluxe"))
    dd.setup(prob.p["chi_cm"] + prob.tau * ionic.di_ion_dv(ui - ue, wn, prob.p))
    return prob, s, dd, (ui, ue, wn)


@pytest.mark.parametrize("name,scaling", [("tiny", "deluxe"), ("cube8", "deluxe"), ("cube8ve", "deluxe"),
                                          ("cube8vef", "deluxe"), ("ragged", "deluxe"), ("cube8ve", "rho"),
                                          ("ragged", "rho"), ("ell8", "deluxe"), ("ell10", "deluxe"),
                                          ("shell_small", "deluxe")])
def test_operators_match_oracle(name, scaling):
    prob, s, dd, _ = _linearized(name, precision="fp64", scaling=scaling)
    n = prob.dofs.n_iface
    x = synth.random_vector(n, 3)
    x[dd.g_iface] = 0.0
    assert _rel(s.schur_apply(x), dd.schur_apply(x)) < 1e-9
    assert _rel(s.bddc_apply(x), dd.bddc_apply(x)) < 1e-9
    F, Minv, lay, nlam = dd.fetidp_operators()
    assert s.sizes["n_lambda"] == nlam
    lam = synth.random_vector(nlam, 4)
    assert _rel(s.fetidp_operator(lam), F(lam)) < 1e-9
    assert _rel(s.fetidp_apply(lam), Minv(lam)) < 1e-9


@pytest.mark.parametrize("name,krylov", [("tiny", "pcg"), ("cube8", "pcg"), ("cube8ve", "pcg"), ("ragged", "pcg"),
                                         ("cube8ve", "gmres"), ("ragged", "gmres"), ("cube8vef", "pcg"),
                                         ("cube8vef", "gmres"), ("ell8", "pcg"), ("shell_small", "pcg")])
@pytest.mark.parametrize("method", ["bddc", "fetidp"])
def test_jacobian_solve_fp64(name, method, krylov):
    prob = oracle_problem(name)
    ui, ue, w = _state(prob)
    wn = ionic.gating_step(ui - ue, w, prob.tau, prob.p)
    r_i, r_e = prob.residual(ui, ue, wn, ui - 1.0, ue, prob.tau)
    kc = prob.kc(ui, ue, wn)
    si, se, _ = direct_solve(prob, kc, -r_i, -r_e)
    f = -np.concatenate([r_i, r_e])
    # paper tolerance: same iteration count as the oracle within +-1 (V+E, V+E+F).  With the
    # vertex-only primal space the preconditioned residual norm oscillates by up to 10x
    # near the threshold, and the oracle alone gives 18 (x86) or 19 (Arm) iterations on
    # this system, so there the bar is +-2.
    s2 = _solver(name, method=method, krylov=krylov, precision="fp64")
    s2.linearize(ui, ue, wn)
    _, st2 = s2.krylov_solve(f)
    dd = DDSolver(prob, method=method, krylov=krylov)
    _, _, info = dd.solve(kc / prob.fem.M, -r_i, -r_e)
    ve = prob.part.primal_kind != "V"  # V+E or V+E+F
    assert abs(st2["its"] - info["its"]) <= (1 if ve else 2)
    if krylov == "pcg":
        # the Lanczos estimate follows the iteration count: 1e-3 (V+E), 1e-2 when it differs (V)
        assert abs(st2["cond"] - info["cond"]) < (1e-3 if ve else 1e-2) * info["cond"]
    # tight tolerance: the exact solution to 1e-10
    s = _solver(name, method=method, krylov=krylov, precision="fp64", ksp_rtol=1e-13, ksp_atol=0.0)
    s.linearize(ui, ue, wn)
    x, st = s.krylov_solve(f)
    assert st["reason"] == 0
    # the accuracy bar for the FP64 Jacobian solve, on every workload (the ellipsoid's
    # Jacobian has kappa 2.4e6: the coarse solve must be backward stable there, Section 4.4)
    assert _rel(x, np.concatenate([si, se])) < 1e-10


def _oracle_steps(prob, nsteps, method="bddc", krylov="pcg"):
    ui, ue, w = synth.initial_state(prob.N, 0)
    dd = DDSolver(prob, method=method, krylov=krylov, rtol=1e-12, atol=0.0)
    out = []
    for n in range(nsteps):
        ui, ue, w, st = time_step(prob, ui, ue, w, n, dd.linsolve(), rtol=1e-10, atol=1e-16)
        out.append((ui.copy(), ue.copy(), st))
    return out


@pytest.mark.parametrize("name,method,precision,tol,graphs,krylov", [
    ("cube8", "bddc", "fp64", 1e-9, 0, "pcg"),
    ("cube8ve", "fetidp", "fp64", 1e-9, 1, "pcg"),
    ("cube8ve", "bddc", "mixed", 1e-8, 1, "pcg"),
    ("ragged", "bddc", "mixed", 1e-8, 0, "pcg"),
    ("cube8ve", "bddc", "fp64", 1e-9, 0, "gmres"),
    ("ragged", "bddc", "mixed+tc", 1e-8, 1, "pcg"),
    ("cube8ve", "bddc", "mixed+tc+lag", 1e-8, 1, "pcg"),
    ("cube8vef", "bddc", "mixed", 1e-8, 1, "pcg"),
    ("ell8", "bddc", "fp64", 1e-9, 0, "pcg"),
    ("ell10", "fetidp", "mixed", 1e-8, 1, "pcg"),
    ("shell_small", "fetidp", "fp64", 1e-9, 0, "pcg"),
    ("shell_small", "bddc", "mixed+tc", 1e-8, 1, "pcg"),
])
def test_time_steps_match_oracle(name, method, precision, tol, graphs, krylov):
    prob = oracle_problem(name)
    ref = _oracle_steps(prob, 3, method, krylov)
    tc, lag = "+tc" in precision, "+lag" in precision
    # the mixed-precision Newton steps are inexact (FP32 operator): at rtol 1e-10 they stop with a
    # residual left in the smooth near-null modes of J, which the ellipsoid's Jacobian amplifies
    # to about 2e-8 in u_e; converged to 1e-12 the comparison measures the solution itself (the
    # oracle's exact Newton steps move its state by 1e-12 between rtol 1e-10 and 1e-13)
    mixed = precision.startswith("mixed")
    s = _solver(name, method=method, krylov=krylov, precision=precision.split("+")[0], ksp_rtol=1e-12,
                ksp_atol=0.0, snes_rtol=1e-12 if mixed else 1e-10, snes_atol=1e-16, use_graphs=graphs,
                use_tensor_cores=int(tc), lag_jacobian=int(lag))
    ui, ue, w = synth.initial_state(prob.N, 0)
    s.set_state(ui, ue, w, 0.0)
    for n in range(3):
        st = s.step(synth.stimulus(prob.workload))
        assert st["reason"] == 0
        gui, gue, gw, t = s.get_state()
        rui, rue, rst = ref[n]
        assert abs(t - (n + 1) * prob.tau) < 1e-12
        assert _rel(gui - gue, rui - rue) < tol
        assert _rel(gue, rue) < tol


def test_device_pointers_and_paper_tolerances():
    torch = pytest.importorskip("torch")
    prob = oracle_problem("cube8ve")
    s = _solver("cube8ve", precision="fp64")
    ui, ue, w = synth.initial_state(prob.N, 0)
    dev = [torch.from_numpy(a).cuda() for a in (ui, ue, w)]
    s.set_state(*dev, 0.0)
    st = s.step(synth.STIMULUS)
    assert st["reason"] == 0 and 1 <= st["newton_its"] <= 3
    gui, gue, gw, _ = s.get_state(like=dev[0])
    assert gui.is_cuda
    rui, rue, rw, _ = time_step(prob, ui, ue, w, 0, lambda kc, a, b: direct_solve(prob, kc, a, b))
    # default tolerances (Section 6 table): agreement limited by SNES rtol 1e-4
    assert _rel(gue.cpu().numpy(), rue) < 1e-4


def test_slab32_first_step_vs_direct_solve():
    """Full-size bench workload: one GPU step against the oracle with the direct solve."""
    prob = oracle_problem("slab32")
    ui, ue, w = synth.initial_state(prob.N, 0)
    rui, rue, _, _ = time_step(prob, ui, ue, w, 0, lambda kc, a, b: direct_solve(prob, kc, a, b),
                               rtol=1e-10, atol=1e-16)
    for precision in ("fp64", "mixed"):
        s = _solver("slab32", precision=precision, ksp_rtol=1e-12, ksp_atol=0.0,
                    snes_rtol=1e-12 if precision == "mixed" else 1e-10, snes_atol=1e-16)
        s.set_state(ui, ue, w, 0.0)
        st = s.step(synth.STIMULUS)
        assert st["reason"] == 0
        gui, gue, _, _ = s.get_state()
        assert _rel(gui - gue, rui - rue) < 1e-8
        assert _rel(gue, rue) < 1e-8


def test_tensor_core_schur_matches_fp64():
    """Full-size local matrices: the tcgen05 (3xTF32) Schur updates keep FP32 accuracy.

    The operator S_hat is checked entry-wise; the preconditioner (which only needs
    spectral equivalence, and whose FP32 rounding S_DD^-1 amplifies) by the PCG
    iteration count and the accuracy of the Jacobian solve it drives.
    """
    prob = oracle_problem("slab32")
    ui, ue, w = _state(prob)
    wn = ionic.gating_step(ui - ue, w, prob.tau, prob.p)
    r_i, r_e = prob.residual(ui, ue, wn, ui - 1.0, ue, prob.tau)
    f = -np.concatenate([r_i, r_e])
    x = synth.random_vector(prob.dofs.n_iface, 5)
    out = {}
    for key, opt in (("fp64", dict(precision="fp64")), ("simt", dict(precision="mixed", use_tensor_cores=0)),
                     ("tc", dict(precision="mixed", use_tensor_cores=1)),
                     ("tcpanel", dict(precision="mixed", use_tensor_cores=2))):
        s = _solver("slab32", **opt)
        s.linearize(ui, ue, wn)
        sol, st = s.krylov_solve(f)
        out[key] = (s.schur_apply(x), sol, st)
        s.close()
    for k in ("simt", "tc", "tcpanel"):
        assert _rel(out[k][0], out["fp64"][0]) < 2e-5
        assert abs(out[k][2]["its"] - out["fp64"][2]["its"]) <= 2
        # an FP32 operator: FP32 rounding is amplified in the near-null modes of J (u_i ~ u_e, smooth,
        # held only by tau A), which leave v = s_i - s_e almost untouched; Newton's FP64 residual
        # removes the rest (the mixed time steps match the oracle to 1e-8)
        N = prob.N
        v_k = out[k][1][:N] - out[k][1][N:]
        v_r = out["fp64"][1][:N] - out["fp64"][1][N:]
        # 2-norm 1e-4; entry-wise the largest error sits where v is small next to large
        # neighbours (the FP32 operator's error is smooth, v is not): 3e-4 of the largest entry
        assert np.linalg.norm(v_k - v_r) < 1e-4 * np.linalg.norm(v_r)
        assert np.max(np.abs(v_k - v_r)) < 3e-4 * np.max(np.abs(v_r))
        d = out[k][1] - out["fp64"][1]
        d = d - d.mean()
        assert np.linalg.norm(d) < 5e-3 * np.linalg.norm(out["fp64"][1])
    assert _rel(out["tc"][0], out["simt"][0]) < 2e-5
    assert _rel(out["tcpanel"][0], out["simt"][0]) < 2e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotune_keeps_results(precision):
    """The autotuner only changes blocking, grouping and the engine's GEMM path."""
    prob = oracle_problem("ragged")
    ui, ue, w = _state(prob)
    wn = ionic.gating_step(ui - ue, w, prob.tau, prob.p)
    s = _solver("ragged", precision=precision, use_tensor_cores=int(precision == "mixed"))
    s.linearize(ui, ue, wn)
    x = synth.random_vector(prob.dofs.n_iface, 9)
    y0 = s.schur_apply(x)
    r = s.autotune()
    assert r["candidates"] >= 9 and r["best_ms"] <= r["default_ms"]
    assert r["outer_panel"] in (128, 256, 512) and r["groups"] in (1, 2, 4)
    y1 = s.schur_apply(x)
    assert _rel(y1, y0) < (1e-12 if precision == "fp64" else 2e-5)


def test_not_spd_is_reported():
    """tau far above 0.37 ms with a depolarised state: Kc < 0, a pivot fails, status says so."""
    from paper_2101_02959_gb300 import binding
    prob = oracle_problem("cube8")
    w = synth.workload("cube8")
    s = binding.Solver(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, 5.0, precision="fp64")
    ui = np.full(prob.N, 37.67)
    z = np.zeros(prob.N)
    with pytest.raises(binding.BidomainError) as e:
        s.linearize(ui, z, z)
    assert e.value.code == -2


def test_profile_regions_nest_and_add_up():
    """Region timers (also with graph replay) nest inside the step and account for it."""
    prob = oracle_problem("cube8ve")
    ui, ue, w = synth.initial_state(prob.N, 0)
    s = _solver("cube8ve", precision="mixed", use_graphs=1)
    s.set_state(ui, ue, w, 0.0)
    s.step(synth.STIMULUS)
    s.profile(2)
    for _ in range(2):
        assert s.step(synth.STIMULUS)["reason"] == 0
    r = {k: s.profile_read(k) for k in ("step", "linearize", "krylov", "trsv", "mlp")}
    assert r["step"]["launches"] == 2
    assert r["linearize"]["launches"] >= 2 and r["krylov"]["launches"] >= 2
    assert r["trsv"]["launches"] == 2 * r["krylov"]["launches"]
    inner = r["linearize"]["ms"] + r["krylov"]["ms"] + r["trsv"]["ms"]
    assert 0.0 < inner <= r["step"]["ms"] * 1.001
    assert s.profile_read("rankk")["launches"] == 0  # kernel classes stay off in region mode
    s.close()


@pytest.mark.parametrize("method", ["bddc", "fetidp"])
def test_rho_scaling_jacobian_solve(method):
    """rho-scaling (Section 4.2): the solve reaches the direct solution and the oracle's
    iteration count within 1, for BDDC and FETI-DP."""
    name = "cube8ve"
    prob = oracle_problem(name)
    ui, ue, w = _state(prob)
    wn = ionic.gating_step(ui - ue, w, prob.tau, prob.p)
    r_i, r_e = prob.residual(ui, ue, wn, ui - 1.0, ue, prob.tau)
    kc = prob.kc(ui, ue, wn)
    si, se, _ = direct_solve(prob, kc, -r_i, -r_e)
    f = -np.concatenate([r_i, r_e])
    s = _solver(name, method=method, precision="fp64", scaling="rho", ksp_rtol=1e-13, ksp_atol=0.0)
    s.linearize(ui, ue, wn)
    x, st = s.krylov_solve(f)
    assert st["reason"] == 0
    assert _rel(x, np.concatenate([si, se])) < 1e-10
    s2 = _solver(name, method=method, precision="fp64", scaling="rho")
    s2.linearize(ui, ue, wn)
    _, st2 = s2.krylov_solve(f)
    dd = DDSolver(prob, method=method, scaling="rho")
    _, _, info = dd.solve(kc / prob.fem.M, -r_i, -r_e)
    assert abs(st2["its"] - info["its"]) <= 1


def _lag_state(prob, seed, bump):
    ui, ue, w = synth.initial_state(prob.N, seed)
    ui = ui + bump * np.exp(-np.sum(prob.mesh.coords ** 2, axis=1) / 0.01)
    wn = ionic.gating_step(ui - ue, w, prob.tau, prob.p)
    r_i, r_e = prob.residual(ui, ue, wn, ui - 1.0, ue, prob.tau)
    return (ui, ue, wn), prob.kc(ui, ue, wn), -r_i, -r_e


@pytest.mark.parametrize("name", ["cube8ve", "ragged"])
def test_lagged_preconditioner_solve(name):
    """precond_every = 2: the second Jacobian is solved with the first one's
    preconditioner.  The solution is the new system's, and the Lanczos estimate is the
    oracle's lagged one (which differs from the fresh estimate by a few per cent)."""
    prob = oracle_problem(name)
    a, kc_a, _, _ = _lag_state(prob, 0, 0.0)
    b, kc_b, f_i, f_e = _lag_state(prob, 1, 60.0)
    f = np.concatenate([f_i, f_e])
    si, se, _ = direct_solve(prob, kc_b, f_i, f_e)
    ref = {}
    for k in (1, 2):
        dd = DDSolver(prob, precond_every=k)
        dd.solve(kc_a / prob.fem.M, f_i, f_e)
        _, _, info = dd.solve(kc_b / prob.fem.M, f_i, f_e)
        ref[k] = info
    assert abs(ref[2]["cond"] - ref[1]["cond"]) > 5e-3 * ref[1]["cond"]
    for k in (1, 2):
        s = _solver(name, precision="fp64", precond_every=k)
        s.linearize(*a)
        s.linearize(*b)
        _, st = s.krylov_solve(f)
        assert st["reason"] == 0
        assert abs(st["its"] - ref[k]["its"]) <= 1
        assert abs(st["cond"] - ref[k]["cond"]) < 1e-3 * ref[k]["cond"]
        s3 = _solver(name, precision="fp64", precond_every=k, ksp_rtol=1e-13, ksp_atol=0.0)
        s3.linearize(*a)
        s3.linearize(*b)
        x, st3 = s3.krylov_solve(f)
        assert st3["reason"] == 0
        assert _rel(x, np.concatenate([si, se])) < 1e-10


def test_lagged_preconditioner_time_steps():
    """precond_every = 3 (BDDC) through three time steps: the GPU's states equal the
    oracle's at tight tolerances (the preconditioner does not change the solution)."""
    name = "cube8ve"
    prob = oracle_problem(name)
    ref = _oracle_steps(prob, 3)
    s = _solver(name, precision="mixed", ksp_rtol=1e-12, ksp_atol=0.0, snes_rtol=1e-12, snes_atol=1e-16,
                precond_every=3, use_graphs=1)
    ui, ue, w = synth.initial_state(prob.N, 0)
    s.set_state(ui, ue, w, 0.0)
    for n in range(3):
        st = s.step(synth.STIMULUS)
        assert st["reason"] == 0
        gui, gue, _, _ = s.get_state()
        assert _rel(gui - gue, ref[n][0] - ref[n][1]) < 1e-8
        assert _rel(gue, ref[n][1]) < 1e-8


def _oracle_steps_direct(prob, nsteps):
    ui, ue, w = synth.initial_state(prob.N, 0)
    out = []
    for n in range(nsteps):
        ui, ue, w, st = time_step(prob, ui, ue, w, n, lambda kc, a, b: direct_solve(prob, kc, a, b),
                                  rtol=1e-10, atol=1e-16)
        out.append((ui.copy(), ue.copy(), st))
    return out


@pytest.mark.parametrize("name", ["cube8ve", "ragged"])
def test_bench_configuration_matches_oracle(name):
    """The solver configuration bench.py times -- mixed precision, tcgen05 Schur updates,
    chord Newton, the learned initial guess trained online from scratch, the autotuned
    engine -- against the FP64 oracle at every one of 20 time steps (v and u_e to 1e-8),
    with the guess in use on several of them."""
    prob = oracle_problem(name)
    nsteps = 20
    ref = _oracle_steps_direct(prob, nsteps)
    stim = synth.stimulus(prob.workload)
    s = _solver(name, precision="mixed", use_tensor_cores=1, lag_jacobian=1, learned_guess=1,
                mlp_train_steps=nsteps, mlp_warmup=3, use_graphs=1, ksp_rtol=1e-12, ksp_atol=0.0,
                snes_rtol=1e-12, snes_atol=1e-16)
    ui, ue, w = synth.initial_state(prob.N, 0)
    s.set_state(ui, ue, w, 0.0)
    s.step(stim)
    s.autotune()
    s.set_state(ui, ue, w, 0.0)
    s.mlp_reset()
    used = 0
    for n in range(nsteps):
        st = s.step(stim)
        assert st["reason"] == 0
        used += st["guess_used"]
        gui, gue, _, _ = s.get_state()
        rui, rue, _ = ref[n]
        assert _rel(gui - gue, rui - rue) < 1e-8, n
        assert _rel(gue, rue) < 1e-8, n
    assert used >= 5
    s.close()


def test_line_search_step_matches_oracle():
    """A step whose Newton iteration backtracks (tau = 0.3 ms, V near the threshold: the
    oracle's line search cuts the step): the GPU's line search takes the same path, so the
    Newton count and the state agree with the oracle's."""
    from oracle import bidomain
    from oracle.bidomain import Problem
    w = synth.workload("cube8")
    prob = Problem(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, 0.3, synth.stimulus(w))
    ui, ue, wv = synth.initial_state(prob.N, 0, sigma_mv=5.0)
    ui = ui + 13.0
    lams = []
    orig = bidomain.line_search_bt

    def spy(fn2, trial, **kw):
        out = orig(fn2, trial, **kw)
        lams.append(out[0])
        return out

    bidomain.line_search_bt = spy
    try:
        rui, rue, _, rst = time_step(prob, ui, ue, wv, 0, lambda kc, a, b: direct_solve(prob, kc, a, b),
                                     rtol=1e-10, atol=1e-16)
    finally:
        bidomain.line_search_bt = orig
    assert min(lams) < 1.0
    from paper_2101_02959_gb300 import binding, build
    build.build()
    s = binding.Solver(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, 0.3, precision="fp64", ksp_rtol=1e-12,
                       ksp_atol=0.0, snes_rtol=1e-10, snes_atol=1e-16)
    s.set_state(ui, ue, wv, 0.0)
    st = s.step(synth.stimulus(w))
    assert st["reason"] == 0
    assert abs(st["newton_its"] - rst["newton_its"]) <= 1
    gui, gue, _, _ = s.get_state()
    assert _rel(gui - gue, rui - rue) < 1e-9
    assert _rel(gue, rue) < 1e-9
    s.close()


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-8), ("fp64", 1e-9)])
def test_coarse_problem_above_1024_unknowns(precision, tol):
    """2,310 coarse unknowns (coarse2k: 512 subdomains of 2^3 elements, V+E): the coarse
    solve stays FP64 at this size (explicit inverse in the local precision plus FP64
    refinement against the assembled S_PiPi, Section 4.4), so the time steps match the
    oracle's at the tight tolerances, and the FP64 BDDC and FETI-DP Jacobian solves
    reach the direct solution to 1e-10."""
    name = "coarse2k"
    prob = oracle_problem(name)
    assert prob.part.n_primal > 1024
    ref = _oracle_steps_direct(prob, 2)
    s = _solver(name, precision=precision, ksp_rtol=1e-12, ksp_atol=0.0,
                snes_rtol=1e-12 if precision == "mixed" else 1e-10, snes_atol=1e-16,
                use_graphs=1)
    ui, ue, w = synth.initial_state(prob.N, 0)
    s.set_state(ui, ue, w, 0.0)
    for n in range(2):
        st = s.step(synth.stimulus(prob.workload))
        assert st["reason"] == 0
        gui, gue, _, _ = s.get_state()
        assert _rel(gui - gue, ref[n][0] - ref[n][1]) < tol
        assert _rel(gue, ref[n][1]) < tol
    s.close()
    if precision != "fp64":
        return
    st_ = _state(prob)
    wn = ionic.gating_step(st_[0] - st_[1], st_[2], prob.tau, prob.p)
    r_i, r_e = prob.residual(st_[0], st_[1], wn, st_[0] - 1.0, st_[1], prob.tau)
    kc = prob.kc(st_[0], st_[1], wn)
    si, se, _ = direct_solve(prob, kc, -r_i, -r_e)
    for method in ("bddc", "fetidp"):
        s = _solver(name, method=method, precision="fp64", ksp_rtol=1e-13, ksp_atol=0.0)
        s.linearize(st_[0], st_[1], wn)
        x, sst = s.krylov_solve(-np.concatenate([r_i, r_e]))
        assert sst["reason"] == 0
        assert _rel(x, np.concatenate([si, se])) < 1e-10, method
        s.close()


@pytest.mark.parametrize("name,precision", [("cube8ve", "fp64"), ("ell8", "fp64"), ("coarse2k", "fp64"),
                                            ("coarse2k", "mixed"), ("ell8", "mixed")])
def test_coarse_matrix_and_fp64_coarse_solve(name, precision):
    """S_PiPi (Section 4.4) as the GPU assembles it equals the oracle's coarse matrix (gauge
    row and column pinned), and the coarse solve the preconditioner applies is FP64-accurate
    for it: backward error at FP64 rounding, also from the FP32 explicit inverse of BD_MIXED
    (whose error alone is orders of magnitude larger)."""
    import scipy.sparse as sp
    prob, s, dd, _ = _linearized(name, precision=precision)
    n = prob.part.n_primal
    g = prob.part.gauge_primal
    ptr, col, val = s.coarse_matrix()
    S = sp.csr_matrix((val, col, ptr), shape=(n, n)).toarray()
    ref = dd.SPP.copy()
    ref[g, :] = 0.0
    ref[:, g] = 0.0
    ref[g, g] = 1.0
    # FP64: rounding of the local Schur complements; BD_MIXED assembles FP32 local blocks
    assert _rel(S, ref) < (1e-10 if precision == "fp64" else 1e-3)
    c = synth.random_vector(n, 21)
    c[g] = 0.0
    nS = np.linalg.norm(S, 2)
    back = lambda z: np.linalg.norm(S @ z - c) / (nS * np.linalg.norm(z))  # noqa: E731
    z = s.coarse_solve(c)
    assert back(z) < 1e-15
    z0 = s.coarse_solve(c, nref=0)
    if precision == "mixed" and n > 320:  # the FP32 inverse of a large coarse problem alone
        assert back(z0) > 100 * back(z)
    np.testing.assert_allclose(z, np.linalg.solve(S, c), rtol=0, atol=1e-12 * np.abs(z).max() * np.linalg.cond(S))
    s.close()
