"""Benchmark of the Bidomain time step on one GB300 (driver contract: one JSON line).

Workload (default): 128x128x32 Q1 elements on a 3.2x3.2x0.8 cm slab, 16x16x4 =
1,024 subdomains (H/h = 8), vertex + edge-average primal space (6,030 coarse
unknowns), Table-1 physics, tau = 0.05 ms, seeded resting state with N(0, 1 mV)
noise and the corner stimulus: 1,098,306 unknowns, the paper's weak-scaling mesh
of 1.1 M dofs (Section 6, Test 1).  A "step" is one time step: gating, then
Newton with the Jacobian solved by PCG + BDDC deluxe (or FETI-DP), at the
paper's tolerances (KSP rtol 1e-8, SNES rtol 1e-4).

The chosen solver (mixed precision: float32 local factors and Schur complements
on the tensor cores, float64 Krylov / Newton / coarse solve; chord Newton; the
learned initial guess trained online from scratch over the first half of the
timed steps) is timed next to the same run without the guess and next to the
plain float64 GPU solver (a sample of the first steps).  Inputs are resident in
HBM for `value`; `e2e` repeats the chosen run through the C-ABI with pinned
host buffers (state copied in and out every step).  With --gpus N > 1 every
rank runs an independent replica (the path does not shard across GPUs); timings
are max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms/time step and Krylov solves/s at rel. res 1e-8, chosen vs plain FP64 GPU"


def describe(w, n_sub=None):
    nx, ny, nz = w["n"]
    sx, sy, sz = w["s"]
    nb = [-(-n // b) for n, b in zip(w["n"], w["s"])]
    if "shell" in w:
        (ai, bi, ci), (ao, bo, co) = w["shell"]["inner"], w["shell"]["outer"]
        h = w["l"][0] / nx
        return (f"{w['name']}: masked Q1 box grid {nx}x{ny}x{nz}, h={h:g} cm, keeping the lower half of the "
                f"ellipsoidal wall between semi-axes ({ai:g},{bi:g},{ci:g}) and ({ao:g},{bo:g},{co:g}) cm; "
                f"{sx}^3-element blocks split into {n_sub} uneven subdomains, primal {w['primal']}, tau=0.05 ms")
    if "ellipsoid" in w:
        dom = "isoparametric Q1 truncated ellipsoid (Section 6)"
    else:
        dom = f"Q1 slab {w['l'][0]}x{w['l'][1]}x{w['l'][2]} cm"
    return (f"{w['name']}: {nx}x{ny}x{nz} {dom}, "
            f"{nb[0]}x{nb[1]}x{nb[2]} subdomains H/h={sx}, primal {w['primal']}, tau=0.05 ms")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "fallback": True}


def rank_barrier(world):
    """Barrier over the replicas (no-op for one process)."""
    if world > 1:
        import torch
        torch.distributed.barrier()


def rank_max(x, world, device="cuda"):
    """Max of a scalar over the replicas: every rank gets the slowest rank's time."""
    if world == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def run_gpu(args, w, rank, world):
    import numpy as np
    import torch

    import synth
    from paper_2101_02959_gb300 import binding, build

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    build.build()
    binding.load()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    probe = binding.Plan(w)  # host-only plan: node count and subdomain sizes (masked grids too)
    N = probe.sizes()["n_node"]
    sub_nodes = np.diff(probe.index_set("SUB_NODE_PTR"))
    # packed values of the explicit symmetric operators of each subdomain (S_Gamma, X, Psi)
    sub_explicit = np.array([explicit_values_per_sub(2 * (nn - ni), nd, npr) for nn, ni, nd, npr in zip(
        sub_nodes, probe.index_set("SUB_NINT"), np.diff(probe.index_set("SUB_DUAL_PTR")),
        np.diff(probe.index_set("SUB_PRIMAL_PTR")))])
    del probe
    ui0, ue0, w0 = synth.initial_state(N, 0)
    dstate = [torch.from_numpy(a).cuda() for a in (ui0, ue0, w0)]
    K = args.steps
    # the learned guess is trained online from scratch over the first half of the timed
    # steps (the 128x128x32 slab's schedule: trained on the first 200 of 400 steps)
    train_steps = max(1, K // 2)

    def barrier():
        rank_barrier(world)

    def max_over_ranks(x):
        return rank_max(x, world, "cuda")

    def solver(precision, method, graphs=1, learned=0):
        return binding.Solver(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, stream=stream.cuda_stream,
                              precision=precision, method=method, use_graphs=graphs, learned_guess=learned,
                              mlp_train_steps=train_steps, mlp_epochs=args.mlp_epochs,
                              use_tensor_cores=int(precision == "mixed" and args.tc),
                              lag_jacobian=int(precision == "mixed" and args.lag), scaling=args.scaling,
                              precond_every=args.precond_every if method == "bddc" else 1)

    def prepare(s, learned, state):
        """Warm-up steps (graph capture, autotuning), then back to t = 0 with an untrained network."""
        s.set_state(*state, 0.0)
        for _ in range(args.warmup):
            s.step(synth.stimulus(w))
        tune = s.autotune() if args.autotune else None
        s.set_state(*state, 0.0)
        if learned:
            s.mlp_reset()
        return tune

    def timed(precision, method, profile=False, clocks=None, graphs=1, learned=0, steps=K):
        s = solver(precision, method, graphs, learned)
        tune = prepare(s, learned, dstate)
        if profile:
            s.profile(profile)
        stats = []
        barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        l0 = binding.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            stats.append(s.step(synth.stimulus(w)))
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        launches = binding.launch_count() - l0
        clk = clocks.stop() if clocks else None
        ms = max_over_ranks(e0.elapsed_time(e1))
        prof = {k: s.profile_read(k) for k in binding.PROF} if profile == 1 or profile is True else None
        regs = {k: s.profile_read(k) for k in binding.REGIONS} if profile else None
        final = s.get_state(like=dstate[0])
        s.close()
        newton = sum(st["newton_its"] for st in stats)
        kry = sum(st["krylov_its"] for st in stats)
        bad = [st["reason"] for st in stats if st["reason"] != 0]
        used = sum(st.get("guess_used", 0) for st in stats)
        return dict(ms=ms, steps=steps, newton=newton, krylov=kry, launches=launches, prof=prof, regions=regs,
                    clocks=clk, bad=bad, cond=max(st["cond_max"] for st in stats), final=final, guess_used=used,
                    tune=tune, stats=stats)

    chosen = timed(args.precision, args.method, clocks=ClockSampler(dev), learned=args.learned)
    other = timed(args.precision, args.method, learned=1 - args.learned)
    if args.step_log and rank == 0:  # per-step statistics of both variants (JSON lines)
        with open(args.step_log, "w") as fh:
            for name, run in (("chosen", chosen), ("other", other)):
                for i, st in enumerate(run["stats"]):
                    fh.write(json.dumps(dict(variant=name, step=i, **st)) + "\n")
    # per-launch CUDA events need stream launches: a second, shorter pass of the same steps
    nprof = min(K, args.profile_steps)
    profiled = timed(args.precision, args.method, profile=True, graphs=0, learned=args.learned, steps=nprof)
    chosen["prof"] = profiled["prof"]
    chosen["prof_ms"] = profiled["ms"] / nprof
    chosen["prof_newton"] = profiled["newton"] / nprof
    chosen["prof_krylov"] = profiled["krylov"] / nprof
    # where a graph-replayed step spends its time: region timers only (a third pass)
    regions = timed(args.precision, args.method, profile=2, learned=args.learned, steps=nprof)
    chosen["regions"] = {k: dict(v, ms=v["ms"] / nprof, launches=v["launches"] / nprof)
                         for k, v in regions["regions"].items()}
    chosen["regions_ms"] = regions["ms"] / nprof
    # the plain FP64 GPU solver (same algorithm, every Jacobian formed, no learned guess) on a
    # sample of the first steps
    nplain = min(K, args.plain_steps)
    plain = timed("fp64", args.method, steps=nplain) if nplain > 0 else None

    # e2e: the chosen run through the C-ABI with host buffers (pinned), the state copied in
    # and out every step; handing the state back at the handle's own time keeps the learned
    # guess's history, so this is the same solver as the timed run
    s = solver(args.precision, args.method, 1, args.learned)
    hs = [torch.from_numpy(a.copy()).pin_memory().numpy() for a in (ui0, ue0, w0)]
    prepare(s, args.learned, hs)
    outs = [torch.empty(N, dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t = 0.0
    e2e_newton = e2e_used = 0
    for _ in range(K):
        s.set_state(*hs, t)
        st = s.step(synth.stimulus(w))
        e2e_newton += st["newton_its"]
        e2e_used += st["guess_used"]
        t = s.get_state_into(*outs)
        hs, outs = outs, hs
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3)
    s.close()

    out = dict(chosen=chosen, plain=plain, other=other, e2e_ms=e2e_ms, e2e_newton=e2e_newton, e2e_used=e2e_used,
               N=N, K=K, nplain=nplain, nprof=nprof, train_steps=train_steps, sub_nodes=sub_nodes,
               sub_explicit=sub_explicit)
    if plain is not None and nplain == K:
        a, b = chosen["final"], plain["final"]
        va, vb = (a[0] - a[1]).double(), (b[0] - b[1]).double()
        out["v_rel_diff_vs_plain"] = float(torch.linalg.norm(va - vb) / torch.linalg.norm(vb))
        out["ue_rel_diff_vs_plain"] = float(torch.linalg.norm(a[1] - b[1]) / torch.linalg.norm(b[1]))
    return out


# ---- algorithmic work of the method (the per-unit figures of the scope table) ----------------
# Local problems of a box subdomain with H/h = k elements per side, dofs ordered plane by
# plane: block tridiagonal with p planes of m dofs each.  Dirichlet (interior): p = k - 1,
# m = 2 (k - 1)^2; constrained Neumann (I + Delta): p = k + 1, m = 2 (k + 1)^2.  A banded
# Cholesky costs 2.33 p m^3 flops and stores 1.5 p m^2 values.
def local_shapes(k):
    pd, md = k - 1, 2 * (k - 1) ** 2
    pn, mn = k + 1, 2 * (k + 1) ** 2
    n_gamma = 2 * ((k + 1) ** 3 - (k - 1) ** 3)
    n_int = 2 * (k - 1) ** 3
    n_face = 2 * (k - 1) ** 2
    return pd, md, pn, mn, n_gamma, n_int, n_face


def factor_flops_per_sub(k, n_primal_local=40):
    """Refactorisation flops per subdomain per Jacobian: Dirichlet and Neumann factors,
    L_II^-1 K_I,Gamma for the interface columns, the face Schur SYRKs of the deluxe blocks
    and Phi (one Neumann solve per local primal dof)."""
    pd, md, pn, mn, ng, ni, nf = local_shapes(k)
    fd, fn = 1.5 * pd * md ** 2, 1.5 * pn * mn ** 2
    return (2.33 * pd * md ** 3 + 2.33 * pn * mn ** 3 + 2.0 * fd * ng + ni * 6 * nf ** 2
            + 4.0 * fn * n_primal_local)


def solve_values_per_sub(k):
    """Factor values one Dirichlet and one Neumann solve read (forward and back)."""
    pd, md, pn, mn, *_ = local_shapes(k)
    return 2.0 * 1.5 * pd * md ** 2, 2.0 * 1.5 * pn * mn ** 2


def explicit_values_per_sub(n_gamma, n_delta, n_primal):
    """Values of the explicit symmetric operators one iteration reads, packed: the lower
    triangles of S_Gamma (n_Gamma) and of S_DeltaDelta^-1 (n_Delta), and Psi (n_Primal x n_Delta)."""
    return n_gamma * (n_gamma + 1) / 2.0 + n_delta * (n_delta + 1) / 2.0 + float(n_primal) * n_delta


# DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum of one capture), kept
# with the first 16 hex digits of the sha256 of the kernel's source text: a figure stands only
# while that text is unchanged, and is reported as null otherwise.
TRAFFIC = {
    "k_rankk_tc": {"bytes_per_launch": None, "sha": None, "file": "tc.cu",
                   "span": ("__global__ void __launch_bounds__(128, 3) k_rankk_tc(",
                            "static constexpr int kTcSmem")},
    # DRAM bytes per library byte (a capture of three launches on the 32x32x16 slab): the operator
    # and local-solve launches read their matrices once; scaled to a launch by its own bytes
    # DRAM bytes per library byte of the symmetric operator and local-solve products (a capture of
    # four launches on the 4x4x4-subdomain cube at H/h = 8, 0.5 GB of operators: larger than L2)
    "k_symv_batched": {"dram_per_library_byte": 1.069, "sha": "00ea69ed6e692111", "file": "dense.cu",
                       "span": ("__global__ void __launch_bounds__(256) k_symv_batched(",
                                "template <typename T>\nsize_t symv_smem(")},
}


def kernel_sha(name):
    import hashlib
    src = open(os.path.join(ROOT, "paper_2101_02959_gb300", "csrc", TRAFFIC[name].get("file", "dense.cu"))).read()
    a_txt, b_txt = TRAFFIC[name]["span"]
    try:
        a = src.index(a_txt)
        b = src.index(b_txt, a)
    except ValueError:
        return None
    return hashlib.sha256(src[a:b].encode()).hexdigest()[:16]


def traffic(name, library_bytes=None):
    """DRAM bytes per launch from the ncu capture, while the kernel's source is the captured one:
    an absolute figure, or a ratio to the launch's own library bytes."""
    t = TRAFFIC.get(name)
    if not t or kernel_sha(name) != t["sha"]:
        return None
    if t.get("dram_per_library_byte") is not None and library_bytes is not None:
        return t["dram_per_library_byte"] * library_bytes
    return t.get("bytes_per_launch")


def device_fp32_peak(dev=0):
    """FP32 SIMT peak derived from the device: SMs x 128 FP32 lanes x 2 flop x max SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = peaks().get("sm_max_mhz", 2070.0)
    return sms * 128 * 2 * mhz * 1e6 / 1e12, f"derived: {sms} SMs (device) x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz"


def equivalent_sides(sub_nodes):
    """H/h of a box subdomain with the same node count as each subdomain ((k + 1)^3 nodes): exact
    for box subdomains, an equivalent size for the pieces of a masked grid."""
    return np.maximum(1, np.rint(np.cbrt(np.asarray(sub_nodes, float)) - 1.0)).astype(int)


def roofline(prof, regions, w, precision, tc_used, sub_nodes, sub_explicit=None):
    """The dominant part of a step against its roofline, with the method's ALGORITHMIC work:
    the factorisation kernels (panel + rank-k classes) per Jacobian against the tensor pipe
    (3xTF32) / FP32 / FP64 peak, or the Krylov local-solve GEMVs per iteration against HBM.
    Both figures are returned; `roofline` is the one that takes more of the step."""
    pk = peaks()
    ks = equivalent_sides(sub_nodes)
    nsub = len(ks)
    k = int(np.max(ks))
    uneven = bool(np.any(ks != ks[0]))
    el = 4 if precision == "mixed" else 8
    n_jac = regions["linearize"]["launches"]
    out = {}
    # factorisation: flops the method needs per Jacobian / time of the factorisation kernels
    f_ms = prof["panel"]["ms"] + prof["rankk"]["ms"]
    f_launch = prof["panel"]["launches"] + prof["rankk"]["launches"]
    if f_ms > 0 and n_jac > 0:
        algo = sum(factor_flops_per_sub(int(kj)) for kj in ks) * n_jac
        lib = prof["panel"]["flops"] + prof["rankk"]["flops"]
        f_capped = uneven and algo > lib
        if f_capped:  # as for the Krylov bytes below: a fragment's factors cost less than the box's
            algo = lib
        if precision == "mixed" and tc_used:
            src = "bf16_tflops_sustained" if "bf16_tflops_sustained" in pk else None
            peak = (pk[src] if src else 1700.0) * 1.1 / 2.25 / 3.0
            psrc = ("of measured: bf16_tflops_sustained x 1.1/2.25 (tf32) / 3 (hi/lo split)" if src
                    else "of fallback: 1.7 PF bf16 sustained x 1.1/2.25 / 3")
            bound = "tensor"
        elif precision == "mixed":
            peak, psrc = device_fp32_peak()
            bound = "alu"
        else:
            peak, psrc = 1.25, "nominal GB300 FP64 (recipe table)"
            bound = "alu"
        ach = algo / (f_ms * 1e-3) / 1e12
        out["factorisation"] = {
            "bound": bound, "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": traffic("k_rankk_tc") if tc_used else None,
            "traffic_note": ("null: the factorisation is a class of launches of several kernels and shapes; "
                             "no per-launch DRAM count stands for it (the tensor-core kernel's own capture "
                             "is summarised in the profiles)"),
            "kernel": ("k_rankk_tc (or k_rankk128 without tensor cores) + k_bigpanel (+ k_diag_inverse with the "
                       "tensor-core panel solve): the factorisation launches of a Jacobian"),
            "peak_source": psrc, "launches": f_launch, "avg_launch_us": f_ms * 1e3 / f_launch,
            "ms_per_jacobian": f_ms / n_jac,
            "algorithmic_flops_per_jacobian": algo / n_jac, "library_flops_per_jacobian": lib / n_jac,
            "work": (f"{factor_flops_per_sub(k):.3g} flop per H/h={k} subdomain x {nsub} subdomains "
                     if not uneven else f"sum over {nsub} uneven subdomains of the flops of a box of the same node "
                     f"count (H/h {ks.min()}..{ks.max()}) ") +
                    "(banded Dirichlet + Neumann factors, L_II^-1 K_IG, face SYRKs, Phi)" +
                    ("; above the flops the launches do, so capped to them" if f_capped else "")}
    # Krylov: one Dirichlet + one Neumann local solve per subdomain and iteration
    g = prof["gemv"]
    if g["ms"] > 0 and g["launches"] > 0:
        banded = np.array([sum(solve_values_per_sub(int(kj))) for kj in ks])
        vd, vn = solve_values_per_sub(k)
        # the method's least data per iteration: the banded factors of the two local solves, or
        # the packed lower triangles of the explicit operators these kernels read, whichever is less
        explicit = np.asarray(sub_explicit, float) if sub_explicit is not None else np.full(nsub, np.inf)
        vals = float(np.sum(np.minimum(banded, explicit)))
        use_explicit = bool(np.all(explicit < banded))
        algo = (g["launches"] / 2.0) * vals * el
        # a masked fragment is flatter than the box of the same node count, so its banded factors
        # hold fewer values than the box model counts: there the bytes the launches read bound it
        capped = uneven and algo > g["bytes"]
        if capped:
            algo = g["bytes"]
        ach = algo / (g["ms"] * 1e-3) / 1e9
        peak = pk.get("hbm_gbs", 6800.0)
        out["krylov"] = {
            "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": traffic("k_symv_batched", g["bytes"] / g["launches"]),
            "kernel": "k_symv_batched (operator S_Gamma and local constrained solve [X; Psi^T], per launch)",
            "peak_source": "of measured" if "fallback" not in pk else "of fallback",
            "launches": g["launches"], "avg_launch_us": g["ms"] * 1e3 / g["launches"],
            "algorithmic_bytes_per_launch": algo / g["launches"], "library_bytes_per_launch": g["bytes"] / g["launches"],
            "work": ((f"{vals / nsub:.3g} values per subdomain and iteration: the packed lower triangles of "
                      f"S_Gamma and S_DeltaDelta^-1 plus Psi, fewer than the {vd + vn:.3g} banded factor values of a "
                      f"Dirichlet + Neumann solve (read forward and back) at H/h={k}, x {nsub} subdomains")
                     if use_explicit else
                     (f"{vd + vn:.3g} factor values per H/h={k} subdomain and iteration (Dirichlet + Neumann "
                      f"solve, read forward and back) x {nsub} subdomains" if not uneven else
                      f"per uneven subdomain the lesser of the packed explicit operators and the factor values of "
                      f"one Dirichlet + one Neumann solve of a box of the same node count, summed over {nsub}")) +
                    f" x {el} B, split over the 2 launches" +
                    ("; above the bytes the launches read, so capped to them" if capped else "")}
    if not out:
        return None, None
    dom = max(out, key=lambda c: (prof["panel"]["ms"] + prof["rankk"]["ms"]) if c == "factorisation"
              else prof["gemv"]["ms"])
    r = dict(out[dom])
    r["measured_in"] = "profiled pass: per-launch CUDA events on the library stream"
    others = {c: v for c, v in out.items() if c != dom}
    return r, others


# workloads whose oracle step is out of the CPU baseline's budget: the sample is the oracle's
# step on a workload with the same subdomains and physics, scaled by the subdomain count
CPU_SAMPLE = {"slab128": "slab32", "beat_slab": "beat_slab_half"}


def cpu_baseline(w, steps=1, method="bddc", scaling="deluxe"):
    """The oracle (numpy, FP64) on the host cores: `steps` time steps of the workload, or of its
    sample workload (same H/h, physics and primal space, fewer subdomains) scaled to it."""
    import synth
    from oracle.bidomain import Problem, time_step
    from oracle.dd import DDSolver
    ws = w
    scale = 1.0
    if w.get("name") in CPU_SAMPLE:
        ws = synth.workload(CPU_SAMPLE[w["name"]])
        ws["primal"] = w["primal"]
        nb = lambda x: np.prod([-(-x["n"][d] // x["s"][d]) for d in range(3)])  # noqa: E731
        scale = float(nb(w)) / float(nb(ws))
    prob = Problem(ws, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, synth.stimulus(ws))
    ui, ue, wv = synth.initial_state(prob.N, 0)
    dd = DDSolver(prob, method=method, scaling=scaling)
    newton = 0
    t0 = time.perf_counter()
    for n in range(steps):
        ui, ue, wv, st = time_step(prob, ui, ue, wv, n, dd.linsolve())
        newton += st["newton_its"]
    sec = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        cores = max(i.get("num_threads", 1) for i in threadpool_info()) or os.cpu_count()
    except Exception:  # threadpoolctl is not installed on every host
        cores = os.cpu_count()
    sample = f"{steps} time step(s) of {ws['name']} ({sec:.1f} s)"
    if scale != 1.0:
        sample += f", scaled x{scale:g} by subdomain count to {w['name']}"
    return dict(ms_per_step=sec * 1e3 / steps * scale, solves_per_s=newton / (sec * scale), cores=cores,
                steps=steps, seconds=sec, sample=sample)


def sweep(args):
    """Optimality sweep (Section 6, Test 3 shape): 4x4x4 subdomains, H/h = 4, 8, 12, 16, V+E primal.

    One time step of the 0.8 cm cube per H/h (after one warm-up step), mixed and FP64: Krylov
    iterations, Lanczos condition number and ms per step.
    """
    import torch

    import synth
    from paper_2101_02959_gb300 import binding, build
    build.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    rows = []
    for k in args.sweep_hh:
        w = synth.workload(f"opt{k}")
        for prec in ("mixed", "fp64"):
            if prec == "fp64" and k > 16:  # FP64 factorisations above H/h = 16 take minutes: mixed only
                continue
            s = binding.Solver(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, stream=stream.cuda_stream,
                               precision=prec, use_graphs=1, use_tensor_cores=int(prec == "mixed"))
            ui, ue, wv = synth.initial_state(s.N, 0)
            s.set_state(ui, ue, wv, 0.0)
            s.step(synth.stimulus(w))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = s.step(synth.stimulus(w))
            e1.record(stream)
            torch.cuda.synchronize()
            rows.append(dict(hh=k, precision=prec, unknowns=2 * s.N, newton=st["newton_its"],
                             krylov_per_newton=st["krylov_its"] / max(st["newton_its"], 1),
                             cond=st["cond_max"], ms=e0.elapsed_time(e1), reason=st["reason"]))
            s.close()
            del s
            torch.cuda.empty_cache()
    print(json.dumps({"sweep": "opt (4x4x4 subdomains, V+E, deluxe BDDC, PCG)", "rows": rows}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="slab128")
    ap.add_argument("--profile-steps", type=int, default=10, help="steps of the profiled passes (kernels, regions)")
    ap.add_argument("--plain-steps", type=int, default=3, help="steps of the plain FP64 sample (0: skip)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--method", default="bddc", choices=["bddc", "fetidp"])
    ap.add_argument("--scaling", default="deluxe", choices=["deluxe", "rho"])
    ap.add_argument("--primal", default=None, choices=["V", "VE", "VEF"], help="override the workload's primal space")
    ap.add_argument("--precond-every", type=int, default=1, help="BDDC: rebuild the preconditioner every k Jacobians")
    ap.add_argument("--learned", type=int, default=1, help="1: learned initial guess in the chosen solver")
    ap.add_argument("--tc", type=int, default=1, help="1: tensor-core (tcgen05) Schur updates in mixed precision")
    ap.add_argument("--lag", type=int, default=1, help="1: chord Newton (one factorisation per time step), mixed only")
    ap.add_argument("--autotune", type=int, default=1, help="1: autotune the factorisation after the warm-up")
    ap.add_argument("--mlp-epochs", type=int, default=4, help="training passes of the learned guess per step")
    ap.add_argument("--cpu-steps", type=int, default=1, help="oracle time steps in the CPU baseline (0: skip)")
    ap.add_argument("--step-log", default=None, help="write the per-step statistics of both variants here (JSONL)")
    ap.add_argument("--sweep", action="store_true", help="H/h optimality sweep instead of the benchmark")
    ap.add_argument("--sweep-hh", type=int, nargs="*", default=[4, 8, 12, 16])
    args = ap.parse_args()
    if args.sweep:
        sweep(args)
        return

    import synth
    w = synth.workload(args.workload)
    if args.primal:
        w["primal"] = args.primal
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        # the oracle is the reference arm: a bounded sample of the workload (about 3 minutes at most)
        one = cpu_baseline(w, 1, args.method, args.scaling)
        steps = max(1, min(args.steps, int(150.0 / max(one["seconds"], 1e-3))))
        res = cpu_baseline(w, steps, args.method, args.scaling) if steps > 1 else one
        line = {"impl": "reference", "metric": METRIC, "value": res["ms_per_step"], "unit": "ms/time step",
                "n_gpus": args.gpus, "steps": res["steps"], "warmup": 0, "ms_per_step": res["ms_per_step"],
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": describe(w), "method": f"{args.method}-{args.scaling}",
                                                "krylov": "pcg"},
                "krylov_solves_per_s": res["solves_per_s"],
                "cpu_baseline": {"value": res["ms_per_step"], "unit": "ms/time step", "cores": res["cores"],
                                 "kind": "oracle", "sample": res["sample"]},
                "e2e": {"value": res["ms_per_step"], "unit": "ms/time step", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    r = run_gpu(args, w, rank, world)
    if rank != 0:
        return
    K, ch, pl = r["K"], r["chosen"], r["plain"]
    ms = ch["ms"] / K
    sec = ch["ms"] * 1e-3
    tc_used = bool(args.tc and args.precision == "mixed")
    if ch["tune"] is not None:
        tc_used = bool(ch["tune"]["tensor_cores"])
    nsub = len(r["sub_nodes"])
    profiled_regions = {k: dict(v, launches=v["launches"] * r["nprof"]) for k, v in ch["regions"].items()}
    roof, roof_other = roofline(ch["prof"], profiled_regions, w, args.precision, tc_used, r["sub_nodes"],
                                r.get("sub_explicit"))
    cpu = None
    if world == 1 and args.cpu_steps > 0:
        c = cpu_baseline(w, args.cpu_steps, args.method, args.scaling)
        cpu = {"value": c["ms_per_step"], "unit": "ms/time step", "cores": c["cores"], "kind": "oracle",
               "sample": c["sample"], "krylov_solves_per_s": c["solves_per_s"]}
    nbytes = 3 * r["N"] * 8
    el = 4 if args.precision == "mixed" else 8
    line = {
        "metric": METRIC, "value": ms, "unit": "ms/time step", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 local factors (tf32 tensor cores) + f64 Krylov/Newton/coarse solve" if args.precision == "mixed"
        else "f64", "data": "synthetic",
        "config": {"workload": describe(w, nsub), "unknowns": 2 * r["N"], "subdomains": nsub,
                   "method": f"{args.method}-{args.scaling}", "krylov": "pcg", "precision": args.precision,
                   "learned_guess": bool(args.learned),
                   "learned_guess_schedule": f"untrained at step 0, trained online on the first {r['train_steps']} "
                                             f"of the {K} timed steps",
                   "tensor_cores": tc_used, "precond_every": args.precond_every,
                   "chord_newton": bool(args.lag and args.precision == "mixed"),
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": f"inputs larger than L2 (129 MB): local matrices "
                         f"{float(np.sum((2.0 * r['sub_nodes']) ** 2)) * el / 1e9:.1f} GB read every step"},
        "krylov_solves_per_s": ch["newton"] / sec,
        "dof_iterations_per_s": 2 * r["N"] * ch["krylov"] / sec,
        "newton_its": ch["newton"], "krylov_its": ch["krylov"], "cond_max": ch["cond"],
        "learned_guess": {"enabled": bool(args.learned), "steps_using_guess": ch["guess_used"],
                          "other_variant": {"learned_guess": bool(1 - args.learned),
                                            "ms_per_step": r["other"]["ms"] / K,
                                            "krylov_its": r["other"]["krylov"], "newton_its": r["other"]["newton"],
                                            "steps_using_guess": r["other"]["guess_used"]}},
        "aggregate_steps_per_s": world * K / sec,
        "e2e": {"value": r["e2e_ms"] / K, "unit": "ms/time step", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes, "host_buffers": "pinned",
                "steps_using_guess": r["e2e_used"], "newton_its": r["e2e_newton"],
                "same_solver_as_value": r["e2e_used"] == ch["guess_used"] and r["e2e_newton"] == ch["newton"]},
        "gpu_launches": ch["launches"],
        "autotune": ch["tune"],
        "roofline": roof,
        "roofline_other_parts": roof_other,
        "profiled_pass": {"steps": r["nprof"], "ms_per_step": ch["prof_ms"], "newton_per_step": ch["prof_newton"],
                          "krylov_per_step": ch["prof_krylov"]},
        "regions_ms_per_step": {"pass_ms_per_step": ch["regions_ms"],
                                **{k: v["ms"] for k, v in ch["regions"].items()}},
        "region_calls_per_step": {k: v["launches"] for k, v in ch["regions"].items()},
        "kernels": {k: dict(v, avg_us=(v["ms"] * 1e3 / v["launches"] if v["launches"] else 0.0))
                    for k, v in ch["prof"].items()},
        "clocks": ch["clocks"],
        "cpu_baseline": cpu,
        "failures": ch["bad"],
    }
    if pl is not None:
        npl = r["nplain"]
        line["plain_fp64"] = {"steps": npl, "sample": f"the first {npl} of the {K} steps",
                              "ms_per_step": pl["ms"] / npl, "krylov_solves_per_s": pl["newton"] / (pl["ms"] * 1e-3),
                              "newton_its_per_step": pl["newton"] / npl, "krylov_its_per_step": pl["krylov"] / npl,
                              "failures": pl["bad"]}
        line["speedup_vs_plain_fp64"] = (pl["ms"] / npl) / ms
        line["v_rel_diff_vs_plain"] = r.get("v_rel_diff_vs_plain")
        line["ue_rel_diff_vs_plain"] = r.get("ue_rel_diff_vs_plain")
    print(json.dumps(line))


if __name__ == "__main__":
    main()
