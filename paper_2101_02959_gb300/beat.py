"""Whole-beat runs (Section 6, Test 4 and Table 11): many consecutive time steps
through activation and recovery, with the per-step statistics the paper reports.

``run`` advances one solver handle for ``steps`` time steps from the seeded
resting state and yields one record per step: the Newton iterations, the Krylov
iterations summed over them, the status, the initial and final nonlinear residual
norms, the largest Lanczos condition estimate of the step and the wall time of
the step (each ``bidomain_step`` call returns after its stream has synchronised).  ``summarize``
turns the records into Table 11's columns: nlit (Newton iterations per time
step), lit (Krylov iterations per Newton iteration) and the time per step.
With ``record_every = k`` the state is read back every k steps, and each node's
activation and recovery times are kept in ``maps``: the first sampled time v
reaches ``threshold`` mV, and the first sampled time after that it is below it.
With ``checkpoint`` (a path) and ``checkpoint_every = k`` the run saves, every k
steps, the state (u_i, u_e, w, t), the step count, the maps and the run's
description (workload, node count, solver options) to that .npz file (written to
a temporary name, then renamed); ``resume`` (a path) continues from such a file
and refuses one written by a different run.  A step that fails (Krylov or Newton
limit, NaN) still yields its record, with the status, and ends the run.  The solver carries no other state from step to step with the
options the runner allows for checkpointing (no learned guess, the
preconditioner rebuilt at every Jacobian), so a resumed run repeats the
uninterrupted one bit for bit.

    python -m paper_2101_02959_gb300.beat --workload beat_slab_half --steps 2400 \\
        --method bddc --precision mixed --out beat.jsonl

Every step runs in the CUDA library; this module only loops and records.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

import synth

from . import binding, build


def summarize(records):
    """Table 11's columns from per-step records, and the mean per-step condition
    estimate (the cond column of Tables 7-8) where the solver reports one."""
    n = len(records)
    if n == 0:
        return dict(steps=0, nlit=0.0, lit=0.0, time_s=0.0, failed=0)
    newton = sum(r["newton_its"] for r in records)
    krylov = sum(r["krylov_its"] for r in records)
    conds = [r["cond_max"] for r in records if r.get("cond_max")]
    return dict(steps=n, nlit=newton / n, lit=krylov / max(newton, 1),
                time_s=sum(r["ms"] for r in records) / n / 1e3,
                cond=sum(conds) / len(conds) if conds else None,
                max_lit_step=max(r["krylov_its"] / max(r["newton_its"], 1) for r in records),
                failed=sum(1 for r in records if r["reason"] != 0))


def update_maps(maps, v, t, threshold):
    """Activation (first v >= threshold) and recovery (first v < threshold after it) times."""
    act, rec = maps["activation"], maps["recovery"]
    rec[~np.isnan(act) & np.isnan(rec) & (v < threshold)] = t
    act[np.isnan(act) & (v >= threshold)] = t


def activation_summary(maps):
    """Time by which every node has activated (NaN if some never did), the fraction of
    nodes activated and the mean activation-recovery interval of the nodes that recovered."""
    act, rec = maps["activation"], maps["recovery"]
    done = ~np.isnan(rec)
    return dict(all_active_ms=float(np.max(act)) if not np.isnan(act).any() else float("nan"),
                active_fraction=float(np.mean(~np.isnan(act))),
                mean_ari_ms=float(np.mean(rec[done] - act[done])) if done.any() else float("nan"))


# solver options a checkpoint records; a resumed run must use the same ones
CHECKPOINT_KEYS = ("method", "krylov", "precision", "scaling", "primal")


def _run_meta(w, s, opt):
    meta = {k: str(opt.get(k, "")) for k in CHECKPOINT_KEYS}
    meta["primal"] = str(opt.get("primal", w.get("primal", "")))
    meta.update(workload=str(w.get("name", "")), n_node=str(s.N))
    return meta


def save_checkpoint(path, s, step, maps, meta=None):
    """State, step count, maps and the run's description (workload, node count, solver
    options) to ``path`` (.npz), replaced atomically."""
    ui, ue, wg, t = s.get_state()
    extra = {k: v for k, v in (maps or {}).items()}
    extra.update({"meta_" + k: np.array(v) for k, v in (meta or {}).items()})
    tmp = path + ".tmp.npz"
    np.savez(tmp, ui=np.asarray(ui), ue=np.asarray(ue), w=np.asarray(wg), t=t, step=step, **extra)
    os.replace(tmp, path)


def check_resume(z, meta, record):
    """Refuse a checkpoint written by a different run: another workload, node count or
    solver options, or one without activation maps when this run records them."""
    for k, v in meta.items():
        key = "meta_" + k
        if key not in z.files:
            raise ValueError(f"checkpoint has no {k!r}: written by an older runner, cannot verify it")
        if str(z[key]) != v:
            raise ValueError(f"checkpoint {k} = {str(z[key])!r}, this run {k} = {v!r}")
    if record and not all(k in z.files for k in ("activation", "recovery")):
        raise ValueError("checkpoint holds no activation / recovery maps but this run records them: "
                         "resume with record_every = 0 or restart the run")


def run(w, steps, seed=0, maps=None, record_every=0, threshold=50.0, checkpoint=None, checkpoint_every=0,
        resume=None, **opt):
    """Yield one record per time step of workload ``w`` (a synth workload dict), for the
    steps up to ``steps`` (a resumed run starts after its checkpoint's step).

    maps: a dict that receives "activation" and "recovery" (ms per node, NaN where the
    event was not seen) when record_every > 0."""
    if (checkpoint or resume) and (opt.get("learned_guess") or opt.get("precond_every", 1) > 1):
        raise ValueError("checkpoints hold the state only: no learned guess, precond_every = 1")
    s = binding.Solver(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, **opt)
    try:
        record = bool(record_every) and maps is not None
        meta = _run_meta(w, s, opt)
        if record:
            maps["activation"] = np.full(s.N, np.nan)
            maps["recovery"] = np.full(s.N, np.nan)
        start = 0
        if resume:
            z = np.load(resume)
            check_resume(z, meta, record)
            s.set_state(z["ui"], z["ue"], z["w"], float(z["t"]))
            start = int(z["step"])
            if record:
                for k in ("activation", "recovery"):
                    maps[k][:] = z[k]
        else:
            ui, ue, wg = synth.initial_state(s.N, seed)
            s.set_state(ui, ue, wg, 0.0)
        stim = synth.stimulus(w)
        for n in range(start, steps):
            t0 = time.perf_counter()
            try:
                st = s.step(stim)
            except binding.BidomainError as e:  # a failed step: its record ends the run
                st = dict(e.stats or {}, reason=e.code)
            ms = (time.perf_counter() - t0) * 1e3
            yield dict(step=n + 1, t=(n + 1) * synth.TAU, newton_its=st.get("newton_its", 0),
                       krylov_its=st.get("krylov_its", 0), reason=st["reason"], ms=ms,
                       res0=st.get("res0"), res_final=st.get("res_final"), cond_max=st.get("cond_max"))
            if st["reason"] != 0:
                return
            if record and (n + 1) % record_every == 0:
                gui, gue, _, t = s.get_state()
                update_maps(maps, np.asarray(gui) - np.asarray(gue), t, threshold)
            if checkpoint and checkpoint_every and (n + 1) % checkpoint_every == 0:
                save_checkpoint(checkpoint, s, n + 1, maps if record else None, meta)
    finally:
        s.close()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="beat_slab_half")
    ap.add_argument("--steps", type=int, default=None, help="default: the workload's own step count")
    ap.add_argument("--method", default="bddc", choices=("bddc", "fetidp"))
    ap.add_argument("--krylov", default="pcg", choices=("pcg", "gmres"))
    ap.add_argument("--precision", default="mixed", choices=("fp64", "mixed"))
    ap.add_argument("--scaling", default="deluxe", choices=("deluxe", "rho"))
    ap.add_argument("--precond-every", type=int, default=1)
    ap.add_argument("--primal", default=None, choices=("V", "VE", "VEF"), help="override the workload's primal space")
    ap.add_argument("--graphs", type=int, default=1)
    ap.add_argument("--out", default=None, help="JSONL file: one line per step, then the summary")
    ap.add_argument("--record-every", type=int, default=0,
                    help="read the state back every k steps for activation / recovery times (0: off)")
    ap.add_argument("--checkpoint", default=None, help=".npz file the run saves its state to")
    ap.add_argument("--checkpoint-every", type=int, default=0)
    ap.add_argument("--resume", default=None, help=".npz checkpoint to continue from")
    a = ap.parse_args(argv)
    w = synth.workload(a.workload)
    if a.primal:
        w["primal"] = a.primal
    steps = a.steps if a.steps is not None else w["steps"]
    build.build()
    expected = steps - (int(np.load(a.resume)["step"]) if a.resume else 0)
    records, maps = [], {}
    out = open(a.out, "w") if a.out else None
    try:
        for r in run(w, steps, maps=maps, record_every=a.record_every, checkpoint=a.checkpoint,
                     checkpoint_every=a.checkpoint_every, resume=a.resume, method=a.method, krylov=a.krylov,
                     precision=a.precision, scaling=a.scaling, precond_every=a.precond_every,
                     use_graphs=a.graphs):
            records.append(r)
            if out:
                out.write(json.dumps(r) + "\n")
        summary = dict(summarize(records), workload=a.workload, method=a.method, precision=a.precision,
                       scaling=a.scaling, primal=w["primal"], precond_every=a.precond_every)
        if maps:
            summary.update(activation_summary(maps))
        if out:
            out.write(json.dumps(dict(summary=summary)) + "\n")
    finally:
        if out:
            out.close()
    print(json.dumps(summary))
    return 0 if summary["failed"] == 0 and summary["steps"] == expected else 1


if __name__ == "__main__":
    raise SystemExit(main())
