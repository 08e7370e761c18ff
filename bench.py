"""Benchmark of the Bidomain time step on one GB300 (driver contract: one JSON line).

Workload (default): 32x32x16 Q1 elements on a 1.6x1.6x0.8 cm slab, 4x4x2
subdomains (H/h = 8), vertex + edge-average primal space, Table-1 physics,
tau = 0.05 ms, seeded resting state with N(0, 1 mV) noise and the corner
stimulus; 20 time steps.  A "step" is one time step: gating, then Newton with
the Jacobian solved by PCG + BDDC deluxe (or FETI-DP), at the paper's
tolerances (KSP rtol 1e-8, SNES rtol 1e-4).

The chosen solver (mixed precision: float32 local factors and Schur
complements, float64 Krylov / Newton / coarse solve) is timed next to the plain
float64 GPU solver on the same mesh.  Inputs are resident in HBM for `value`;
`e2e` repeats the chosen run through the C-ABI with host buffers (state copied
in and out every step).  With --gpus N > 1 every rank runs an independent
replica (the path does not shard across GPUs); timings are max over ranks.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms/time step and Krylov solves/s at rel. res 1e-8, chosen vs plain FP64 GPU"
FP32_SIMT_PEAK = 152 * 128 * 2 * 2.07e9 / 1e12   # TFLOP/s: SMs x FP32 lanes x FMA x max SM clock
FP64_PEAK = 1.25                                  # TFLOP/s, nominal GB300 FP64


def describe(w):
    nx, ny, nz = w["n"]
    sx, sy, sz = w["s"]
    if "ellipsoid" in w:
        dom = "isoparametric Q1 truncated ellipsoid (Section 6)"
    else:
        dom = f"Q1 slab {w['l'][0]}x{w['l'][1]}x{w['l'][2]} cm"
    nb = [-(-n // b) for n, b in zip(w["n"], w["s"])]
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
    N = synth.n_nodes(w)
    ui0, ue0, w0 = synth.initial_state(N, 0)
    dstate = [torch.from_numpy(a).cuda() for a in (ui0, ue0, w0)]

    def barrier():
        rank_barrier(world)

    def max_over_ranks(x):
        return rank_max(x, world, "cuda")

    def timed(precision, method, profile=False, clocks=None, graphs=1, learned=0):
        s = binding.Solver(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, stream=stream.cuda_stream,
                           precision=precision, method=method, use_graphs=graphs, learned_guess=learned,
                           mlp_train_steps=args.steps + args.warmup + 1, mlp_epochs=args.mlp_epochs,
                           use_tensor_cores=int(precision == "mixed" and args.tc),
                           lag_jacobian=int(precision == "mixed" and args.lag), scaling=args.scaling,
                           precond_every=args.precond_every if method == "bddc" else 1)
        s.set_state(*dstate, 0.0)
        for _ in range(args.warmup):
            s.step(synth.stimulus(w))
        tune = s.autotune() if args.autotune else None
        s.set_state(*dstate, 0.0)
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
        for _ in range(args.steps):
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
        return dict(ms=ms, newton=newton, krylov=kry, launches=launches, prof=prof, regions=regs, clocks=clk, bad=bad,
                    cond=max(st["cond_max"] for st in stats), final=final, guess_used=used, tune=tune)

    chosen = timed(args.precision, args.method, clocks=ClockSampler(dev), learned=args.learned)
    other = timed(args.precision, args.method, learned=1 - args.learned)
    # per-launch CUDA events need stream launches: a second pass of the same K steps, profiled
    profiled = timed(args.precision, args.method, profile=True, graphs=0, learned=args.learned)
    chosen["prof"] = profiled["prof"]
    chosen["prof_ms"] = profiled["ms"]
    # where a graph-replayed step spends its time: region timers only (a third pass)
    regions = timed(args.precision, args.method, profile=2, learned=args.learned)
    chosen["regions"] = regions["regions"]
    chosen["regions_ms"] = regions["ms"]
    plain = timed("fp64", args.method) if not args.no_plain else None

    # e2e: the same chosen run through host buffers, state copied in and out every step
    s = binding.Solver(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, stream=stream.cuda_stream,
                       precision=args.precision, method=args.method, use_graphs=1, learned_guess=args.learned,
                       mlp_train_steps=args.steps + args.warmup + 1, mlp_epochs=args.mlp_epochs,
                       use_tensor_cores=int(args.precision == "mixed" and args.tc),
                       lag_jacobian=int(args.precision == "mixed" and args.lag), scaling=args.scaling,
                       precond_every=args.precond_every if args.method == "bddc" else 1)
    hs = (ui0.copy(), ue0.copy(), w0.copy())
    s.set_state(*hs, 0.0)
    for _ in range(args.warmup):
        s.step(synth.stimulus(w))
    if args.autotune:
        s.autotune()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    state, t = hs, 0.0
    e2e_newton = 0
    for _ in range(args.steps):
        s.set_state(*state, t)
        st = s.step(synth.stimulus(w))
        e2e_newton += st["newton_its"]
        ui, ue, wv, t = s.get_state()
        state = (ui, ue, wv)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3)
    s.close()

    K = args.steps
    out = dict(chosen=chosen, plain=plain, other=other, e2e_ms=e2e_ms, e2e_newton=e2e_newton, N=N)
    # final-state agreement of the chosen and the plain FP64 solvers after K steps
    if plain is not None:
        a, b = chosen["final"], plain["final"]
        va, vb = (a[0] - a[1]).double(), (b[0] - b[1]).double()
        out["v_rel_diff_vs_plain"] = float(torch.linalg.norm(va - vb) / torch.linalg.norm(vb))
        out["ue_rel_diff_vs_plain"] = float(torch.linalg.norm(a[1] - b[1]) / torch.linalg.norm(b[1]))
    out["K"] = K
    return out


# DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum, averaged over every
# launch of a slab32 run; profiles/*_slab32_mixed_bddc.md).  A figure stands only while its
# kernel's source text is the one it was measured on (first 16 hex digits of its sha256).
TRAFFIC = {
    # k_rankk128 is the "rankk" class only with tensor cores off; its measured launches (the
    # in-block updates, 21.1 MB each) belong to the panel class, so no figure is kept for it
    "k_rankk128": {"bytes_per_launch": None, "sha": "69ca1105c88785a7",
                   "span": ("__global__ void __launch_bounds__(256) k_rankk128(",
                            "template <typename T>\nstatic void launch_rankk(")},
    "k_bigpanel": {"bytes_per_launch": 7.78e6, "sha": "a3c19f2ca59fb23c",
                   "span": ("template <typename T, bool ROWS>\n__global__ void __launch_bounds__(256, ROWS ? 2 : 1) "
                            "k_bigpanel(", "// ---- rank-k update of lower tiles")},
    "k_rankk_tc": {"bytes_per_launch": 72.36e6, "sha": "f793e17009497dfe", "file": "tc.cu",
                   "span": ("__global__ void __launch_bounds__(128, 1) k_rankk_tc(",
                            "static constexpr int kTcSmem")},
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


def traffic(name):
    t = TRAFFIC.get(name)
    if not t or t["bytes_per_launch"] is None:
        return None
    return t["bytes_per_launch"] if kernel_sha(name) == t["sha"] else None


def roofline(prof, precision, tc_used=False):
    """Dominant profiled kernel class against its roofline."""
    pk = peaks()
    dom = max(prof, key=lambda k: prof[k]["ms"])
    p = prof[dom]
    if p["launches"] == 0 or p["ms"] <= 0:
        return None, dom
    if dom == "rankk" and precision == "mixed" and tc_used:
        # tcgen05 kind::tf32 with operands split in hi + lo TF32 parts: three MMAs per
        # FP32-accurate product, so the peak for algorithmic FP32 flops is the TF32 peak
        # (measured sustained bf16 x the nominal tf32 / bf16 ratio 1.1 / 2.25) / 3
        achieved = p["flops"] / (p["ms"] * 1e-3) / 1e12
        src = "bf16_tflops_sustained" if "bf16_tflops_sustained" in pk else None
        tf32 = (pk[src] if src else 1700.0) * 1.1 / 2.25
        peak = tf32 / 3.0
        r = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
             "traffic": traffic("k_rankk_tc"), "kernel": "k_rankk_tc",
             "peak_source": ("of measured: bf16_tflops_sustained x 1.1/2.25 (tf32) / 3 (hi/lo split)" if src
                             else "of fallback: 1.7 PF bf16 sustained x 1.1/2.25 / 3")}
    elif dom in ("rankk", "panel"):
        achieved = p["flops"] / (p["ms"] * 1e-3) / 1e12
        peak = FP32_SIMT_PEAK if precision == "mixed" else FP64_PEAK
        if dom == "rankk":
            kern = "k_rankk128" if precision == "mixed" and not tc_used else \
                "k_rankk_tc" if precision == "mixed" else "k_rankk<double>"
        else:
            kern = "k_bigpanel"  # diagonal + rows launches (the class also times the in-block updates)
        r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
             "traffic": traffic(kern) if precision == "mixed" else None,
             "kernel": kern,
             "peak_source": ("derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz" if precision == "mixed"
                             else "nominal GB300 FP64 (recipe table)")}
    else:
        achieved = p["bytes"] / (p["ms"] * 1e-3) / 1e9
        peak = pk.get("hbm_gbs", 6800.0)
        r = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
             "traffic": None, "kernel": "k_gemv" if dom == "gemv" else "k_residual",
             "peak_source": "of measured" if "fallback" not in pk else "of fallback"}
    r["launches"] = p["launches"]
    r["avg_launch_us"] = p["ms"] * 1e3 / p["launches"]
    r["measured_in"] = "profiled pass of the same K steps: per-launch CUDA events on the library stream"
    return r, dom


def cpu_baseline(w, steps=1, method="bddc", scaling="deluxe"):
    """The oracle (numpy, FP64) on the host cores: `steps` time steps of the same workload."""
    import synth
    from oracle.bidomain import Problem, time_step
    from oracle.dd import DDSolver
    prob = Problem(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, synth.stimulus(w))
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
    return dict(ms_per_step=sec * 1e3 / steps, solves_per_s=newton / sec, cores=cores, steps=steps,
                seconds=sec)


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
            if prec == "fp64" and k > 12:  # ~20 s per FP64 factorisation at this size: mixed only
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
    ap.add_argument("--workload", default="slab32")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--method", default="bddc", choices=["bddc", "fetidp"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--scaling", default="deluxe", choices=["deluxe", "rho"])
    ap.add_argument("--primal", default=None, choices=["V", "VE", "VEF"], help="override the workload's primal space")
    ap.add_argument("--precond-every", type=int, default=1, help="BDDC: rebuild the preconditioner every k Jacobians")
    ap.add_argument("--learned", type=int, default=1, help="1: learned initial guess in the chosen solver")
    ap.add_argument("--tc", type=int, default=1, help="1: tensor-core (tcgen05) Schur updates in mixed precision")
    ap.add_argument("--lag", type=int, default=1, help="1: chord Newton (one factorisation per time step), mixed only")
    ap.add_argument("--autotune", type=int, default=1, help="1: autotune the factorisation after the warm-up")
    ap.add_argument("--mlp-epochs", type=int, default=4, help="training passes of the learned guess per step")
    ap.add_argument("--cpu-steps", type=int, default=1, help="oracle time steps in the CPU baseline (0: skip)")
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
        # the oracle is the reference arm: bounded sample of the same workload (about 3 minutes at most)
        one = cpu_baseline(w, 1, args.method, args.scaling)
        steps = max(1, min(args.steps, int(150.0 / max(one["seconds"], 1e-3))))
        res = cpu_baseline(w, steps, args.method, args.scaling) if steps > 1 else one
        line = {"impl": "reference", "metric": METRIC, "value": res["ms_per_step"], "unit": "ms/time step",
                "n_gpus": args.gpus, "steps": res["steps"], "warmup": 0, "ms_per_step": res["ms_per_step"],
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": describe(w), "method": f"{args.method}-{args.scaling}", "krylov": "pcg"},
                "krylov_solves_per_s": res["solves_per_s"],
                "cpu_baseline": {"value": res["ms_per_step"], "unit": "ms/time step", "cores": res["cores"],
                                 "kind": "oracle", "sample": f"{res['steps']} time step(s) of {w['name']}"},
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
    roof, dom = roofline(ch["prof"], args.precision, tc_used)
    cpu = None
    if world == 1 and args.cpu_steps > 0:
        c = cpu_baseline(w, args.cpu_steps, args.method, args.scaling)
        cpu = {"value": c["ms_per_step"], "unit": "ms/time step", "cores": c["cores"], "kind": "oracle",
               "sample": f"{c['steps']} time step(s) of {w['name']} ({c['seconds']:.1f} s)",
               "krylov_solves_per_s": c["solves_per_s"]}
    nbytes = 3 * r["N"] * 8
    line = {
        "metric": METRIC, "value": ms, "unit": "ms/time step", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 local factors (tf32 tensor cores) + f64 Krylov/Newton/coarse solve" if args.precision == "mixed"
        else "f64", "data": "synthetic",
        "config": {"workload": describe(w), "unknowns": 2 * r["N"], "method": f"{args.method}-{args.scaling}",
                   "krylov": "pcg", "precision": args.precision, "learned_guess": bool(args.learned),
                   "tensor_cores": tc_used, "precond_every": args.precond_every,
                   "chord_newton": bool(args.lag and args.precision == "mixed"), "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "per-step working set > 129 MB L2 (local matrices 0.27 GB f32 / 0.54 GB f64)"},
        "krylov_solves_per_s": ch["newton"] / sec,
        "dof_iterations_per_s": 2 * r["N"] * ch["krylov"] / sec,
        "newton_its": ch["newton"], "krylov_its": ch["krylov"], "cond_max": ch["cond"],
        "learned_guess": {"enabled": bool(args.learned), "steps_using_guess": ch["guess_used"],
                          "other_variant": {"learned_guess": bool(1 - args.learned),
                                            "ms_per_step": r["other"]["ms"] / K,
                                            "krylov_its": r["other"]["krylov"], "newton_its": r["other"]["newton"]}},
        "aggregate_steps_per_s": world * K / sec,
        "e2e": {"value": r["e2e_ms"] / K, "unit": "ms/time step", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "gpu_launches": ch["launches"],
        "autotune": ch["tune"],
        "roofline": roof,
        "profiled_pass_ms_per_step": ch["prof_ms"] / K,
        "regions_ms_per_step": {"pass_ms_per_step": ch["regions_ms"] / K,
                                **{k: v["ms"] / K for k, v in ch["regions"].items()}},
        "region_calls_per_step": {k: v["launches"] / K for k, v in ch["regions"].items()},
        "kernels": {k: dict(v, avg_us=(v["ms"] * 1e3 / v["launches"] if v["launches"] else 0.0))
                    for k, v in ch["prof"].items()},
        "clocks": ch["clocks"],
        "cpu_baseline": cpu,
        "failures": ch["bad"],
    }
    if pl is not None:
        line["plain_fp64"] = {"ms_per_step": pl["ms"] / K, "krylov_solves_per_s": pl["newton"] / (pl["ms"] * 1e-3),
                              "newton_its": pl["newton"], "krylov_its": pl["krylov"], "failures": pl["bad"]}
        line["speedup_vs_plain_fp64"] = (pl["ms"] / K) / ms
        line["v_rel_diff_vs_plain"] = r.get("v_rel_diff_vs_plain")
        line["ue_rel_diff_vs_plain"] = r.get("ue_rel_diff_vs_plain")
    print(json.dumps(line))


if __name__ == "__main__":
    main()
