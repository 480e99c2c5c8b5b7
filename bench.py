#!/usr/bin/env python
"""Throughput benchmark of the fused D2Q9 multiphase time step on GB300.

Workload (one bench "step" = one pass of the whole hot path over one batch): a
4096 x 4096 periodic D2Q9 lattice, Carnahan-Starling EOS (a = 0.25, b = 4, R = 1)
at Tr = 0.85, tau = 0.8, spinodal decomposition from rho = (rho_l + rho_v)/2 (1 +
U(-0.01, 0.01)) (seed 2403), 2000 FP32 time steps of the pseudopotential model and
2000 of the free-energy model, each started from f = f^eq(rho0).

Prints one JSON line.  ``value`` is MLUPS with the initial density already in HBM;
``e2e`` is the same metric through the public C ABI with the FP64 initial density
in pinned host memory, host->device copy, time stepping and observables read-back
inside the timed region.  ``--impl reference`` times the FP64 CPU oracle instead.
Multi-GPU (torchrun): independent replicas, one lattice per rank (weak scaling).
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D2Q9 multiphase MLUPS & HBM-roofline fraction; sweep runs/s batched vs plain"
# Algorithmic bytes per FP32 cell update: the state each step must read and write once, 9 FP32
# populations and the int16 extension of the rest population (compensated f_0), in and out:
# 2 x (36 + 2) = 76 B for both models.
BYTES_PER_CELL = {0: 76, 1: 76}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--lbm-steps", type=int, default=2000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the batched-vs-plain calibration sweep")
    ap.add_argument("--sweep-lattices", type=int, default=512)
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned calibration surrogate")
    ap.add_argument("--surrogate-sets", type=int, default=8000)
    ap.add_argument("--no-walls", action="store_true", help="skip the walled-channel measurement")
    ap.add_argument("--ref-seconds", type=float, default=None,
                    help="reference arm: seconds of oracle work per timed step (default: ~1 min in total)")
    ap.add_argument("--plain-sets", type=int, default=6, help="held-out sets also calibrated one lattice at a time")
    ap.add_argument("--profile", choices=["pp", "fe"], default=None,
                    help="profiler workload: --steps single-step launches of one model's FP32 step on the "
                         "--size^2 spinodal lattice (for ncu -k regex:<model>_step), no JSON line")
    ap.add_argument("--A", type=float, default=0.0, help="--profile fe with A != 0 runs the full-model kernel")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device="cpu") -> float:
    """The largest of every rank's x (the job takes as long as its slowest rank); x itself when
    the job has one rank.  Collective over the default process group (NCCL on GPUs, gloo in
    the CPU tests)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ws: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return ws * units_per_rank / seconds


def workload_config(args):
    return {
        "workload": f"spinodal decomposition, {args.size}x{args.size} periodic D2Q9, Carnahan-Starling a=0.25 "
                    f"Tr=0.85, tau=0.8, {args.lbm_steps} steps each of the pseudopotential and free-energy models",
        "nx": args.size, "ny": args.size, "lbm_steps_per_model": args.lbm_steps,
        "models": ["pseudopotential (MP-LBM)", "free energy (IWB-FE-LBM)"],
        "precision": "fp32 populations", "parallelism": "replicas",
        "l2": "inputs larger than L2 (1.2 GB of populations per model)",
    }


def make_rho0(size, rho_v, rho_l):
    """The workload's initial density from the coexistence densities of its parameters."""
    from paper_2403_11167_gb300 import inputs

    return inputs.spinodal_noise(size, size, 0.5 * (rho_l + rho_v), 0.01, seed=2403)


# --------------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline).  Everything on this leg -- the temperature,
# the coexistence densities, sigma^Li and the default relaxation times (tau_nu = tau; P:
# tau_e = tau_zeta = tau, tau_q = 1/1.99; FE: tau_e = 1/4 + tau/2) -- comes from the oracle
# package; the product library is not loaded.

def oracle_workload():
    """(rho_v, rho_l, [oracle parameters of the P and FE models]) of the throughput workload
    (Carnahan-Starling a = 0.25, b = 4, R = 1, Tr = 0.85, tau = 0.8, kappa = 0.5)."""
    import oracle as O
    from oracle import thermo

    a, b, R, Tr, tau = 0.25, 4.0, 1.0, 0.85, 0.8
    T = thermo.temperature(a, b, R, Tr)
    rho_v, rho_l, _ = thermo.maxwell(a, b, R, Tr)
    sigma_li = thermo.sigma_li(a, b, R, Tr)[0]
    pp = O.make_params(a=a, b=b, R=R, T=T, tau_e=tau, tau_zeta=tau, tau_q=1.0 / 1.99, tau_j=1.0, tau_nu=tau,
                       kappa_P=1.0, kappa_Li=0.0, sigma_Li=sigma_li)
    fe = O.make_params(a=a, b=b, R=R, T=T, tau_e=0.25 + 0.5 * tau, tau_zeta=1.0, tau_q=1.0, tau_j=1.0,
                       tau_nu=tau, kappa=0.5)
    return rho_v, rho_l, [pp, fe]


def oracle_mlups(size, seconds, crop=512):
    """Time the FP64 oracle, as it stands, on a crop of the workload: both models, the
    number of steps grown until about ``seconds`` of CPU work.  Returns (MLUPS, threads,
    sample description, seconds of oracle work)."""
    import numpy as np

    import oracle as O

    rho_v, rho_l, cfgs = oracle_workload()
    sub = np.ascontiguousarray(make_rho0(size, rho_v, rho_l)[:crop, :crop])
    updates, elapsed, steps = 0, 0.0, 1
    while elapsed < seconds:
        for model in (0, 1):
            f = O.init(model, sub)
            t = time.perf_counter()
            O.run(model, cfgs[model], f, steps)
            elapsed += time.perf_counter() - t
            updates += sub.size * steps
        steps *= 2
    return updates / elapsed / 1e6, O.num_threads(), f"{crop}x{crop} crop of the workload, both models, " \
        f"{updates // sub.size} lattice steps in total, FP64", elapsed


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    per_step = args.ref_seconds or max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_mlups(args.size, per_step / 4)
    vals, secs, cores, sample = [], [], 1, ""
    for _ in range(args.steps):
        v, cores, sample, sec = oracle_mlups(args.size, per_step)
        vals.append(v)
        secs.append(sec)
    value = sum(vals) / len(vals)
    cell_updates = 2 * args.lbm_steps * args.size * args.size
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        # a timed step is one bounded sample of the workload (see cpu_baseline.sample)
        "ms_per_step": 1e3 * sum(secs) / len(secs),
        "ms_per_step_extrapolated_full_workload": cell_updates / (value * 1e6) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# --------------------------------------------------------------------------------------
# GPU arm

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_sweep(args):
    """Calibration sweep of 512 seeded pseudopotential lattices (uneven sizes 64x4 .. 512x512,
    flat slabs and droplets, Tr ~ U[0.5, 0.95], kappa_P in {0.4, 0.7, 1}, tau ~ U[0.6, 1.2],
    5e3 .. 2e4 steps), FP32: runs/s of one batched sweep (lbm_batch_run + observables) against
    the same lattices solved one at a time through the single-lattice API (set_density +
    step + observables on pre-created contexts).  Allocation and autotuning are outside both
    timed regions."""
    import torch

    from paper_2403_11167_gb300 import inputs, lbm

    entries = inputs.calibration_sweep(args.sweep_lattices, seed=11167)
    specs, rhos = lbm.sweep_specs(entries)
    cells = sum(s["nx"] * s["ny"] * s["nsteps"] for s in specs)
    b = lbm.Batch(specs, rhos)
    info = b.info()
    torch.cuda.synchronize()
    t = time.perf_counter()
    b.run()
    obs = b.observables()
    t_batch = time.perf_counter() - t
    diverged = sum(1 for o in obs if o["status"] != 0)
    b.close()
    # floor of the tiled path's per-step launches (graph replays of one launch per step): a
    # single tiled lattice too small to do measurable work, 2e4 steps
    e = inputs.calibration_sweep(1, seed=5)[0]
    e.update(geometry=0, nx=512, ny=12, radius=0.0, nsteps=20000, Tr=0.8, kappa_P=1.0)
    fspecs, frhos = lbm.sweep_specs([e])
    fb = lbm.Batch(fspecs, frhos)
    assert fb.info()["n_resident"] == 0
    torch.cuda.synchronize()
    t = time.perf_counter()
    fb.run()
    fb.observables()
    floor_s = (time.perf_counter() - t) / 20000
    fb.close()
    # lattices of more than 4452 cells run tiled (lbm_batch_create's residency rule)
    max_tiled = max((s["nsteps"] for s in specs if s["nx"] * s["ny"] > 4452), default=0)
    ctxs = [lbm.Context(s["params"], s["nx"], s["ny"]) for s in specs]
    torch.cuda.synchronize()
    t = time.perf_counter()
    for ctx, s, r in zip(ctxs, specs, rhos):
        ctx.set_density(r)
        ctx.step(s["nsteps"])
        ctx.observables(s["geometry"])
    t_plain = time.perf_counter() - t
    for ctx in ctxs:
        ctx.close()
    n = len(specs)
    ok = n - diverged
    return {"lattices": n, "cell_updates": cells, "batched_s": t_batch, "plain_s": t_plain,
            # every lattice runs all its steps on both paths (a diverged one is only flagged at
            # the end), so runs/s counts all of them; the completed (non-diverged) runs per
            # second are reported beside them
            "batched_runs_per_s": n / t_batch, "plain_runs_per_s": n / t_plain, "speedup": t_plain / t_batch,
            "completed_lattices": ok, "diverged_lattices": diverged,
            "batched_completed_runs_per_s": ok / t_batch, "plain_completed_runs_per_s": ok / t_plain,
            "batched_mlups": cells / t_batch / 1e6, "plain_mlups": cells / t_plain / 1e6,
            "tiled_step_floor_us": floor_s * 1e6, "tiled_steps": max_tiled,
            # upper bound of what one persistent launch could save over the per-step replays
            "tiled_launch_floor_fraction": floor_s * max_tiled / t_batch,
            "resident_lattices": info["n_resident"],
            "tiled_work_items": info["n_items"], "resident_threads": info["resident_threads"],
            "strip_rows": info["strip_rows"],
            "workload": "512 seeded pseudopotential calibration lattices (64x4..512x512 slabs and droplets, "
                        "5e3-2e4 steps), FP32"}


def run_walls(args, peak):
    """Walled channel (no-slip walls on rows 0 and ny-1, body force): FP32 step throughput of
    both models (periodic strip kernel on the whole lattice, then the wall bands recomputed by
    the wall kernel; two launches per step) on a size x size plate channel (vapour below, liquid above, sine-perturbed
    interface, F_x = 1e-6), CUDA events around 500 steps on the launching stream; and the
    wall-clock rate of the 101 x 50 FP64 channel of Sec. 5.3 (steps/s over 2e4 steps); and the
    droplet-collision drive of Sec. 5.4: steps/s of the 200 x 100 FP64 pair (a domain-mean
    reduction plus a direct step per step), and FP32 throughput of a size x size pair (the
    driven strip kernels, rho_ave from the masses the previous step stored; one reduction per
    64-step graph)."""
    import numpy as np
    import torch

    from paper_2403_11167_gb300 import inputs, lbm

    size, nsteps = args.size, 500
    out = {"workload": f"{size}x{size} plate channel, FP32, 500 steps per model; 101x50 Sec. 5.3 channel, FP64"}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for model, key in ((0, "pseudopotential"), (1, "free_energy")):
            p = lbm.lbm_params_default(model, precision=lbm.LBM_F32, a=0.25, Tr=0.8, tau_nu=1.0, tau_e=1.0,
                                       body_fx=1e-6)
            ctx = lbm.Context(p, size, size, stream=stream, walls=True)
            _, th = ctx.derived()
            ctx.set_density(inputs.plate_channel(size, size, th.rho_v, th.rho_l, amp=8.0))
            ctx.step(64)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            ctx.step(nsteps)
            e1.record(stream)
            torch.cuda.synchronize()
            s = e0.elapsed_time(e1) * 1e-3 / nsteps
            gbs = BYTES_PER_CELL[model] * size * size / s / 1e9
            out[key] = {"mlups": size * size / s / 1e6, "us_per_launch": s * 1e6,
                        "algorithmic_bytes_per_cell": BYTES_PER_CELL[model], "gbs": gbs,
                        "frac_of_hbm": gbs / peak,
                        "kernels": ("pp_step_pair + pp_step_ext (wall bands, 2 rows)",
                                    "fe_step_pair + fe_step_ext (wall bands, 3 rows)")[model]}
            ctx.close()
        rates = {}
        for model, key in ((0, "pseudopotential"), (1, "free_energy")):
            kw = dict(a=0.25, Tr=0.8, tau_nu=1.0, tau_e=1.0, body_fx=1e-6)
            kw.update({"match_kappa": 0.5} if model == 0 else {"kappa": 0.5})
            p = lbm.lbm_params_default(model, precision=lbm.LBM_F64, **kw)
            ctx = lbm.Context(p, 101, 50, stream=stream, walls=True)
            _, th = ctx.derived()
            ctx.set_density(inputs.plate_channel(101, 50, th.rho_v, th.rho_l))
            ctx.step(640)
            torch.cuda.synchronize()
            t = time.perf_counter()
            ctx.step(20000)
            torch.cuda.synchronize()
            rates[key] = 20000 / (time.perf_counter() - t)
            ctx.close()
        out["sec53_channel_f64_steps_per_s"] = rates
        # Sec. 5.4: droplet pair driven together (FP64: reduction + direct step; FP32: driven strip kernels)
        col = {}
        for model, key in ((0, "pseudopotential"), (1, "free_energy")):
            kw = dict(a=0.25, Tr=0.8, tau_nu=1.0)
            kw.update({"match_kappa": 0.5, "tau_e": 1.0} if model == 0 else {"tau_e": 0.75, "kappa": 0.5})
            for prec, pk in ((lbm.LBM_F64, "f64_200x100_steps_per_s"), (lbm.LBM_F32, "f32_4096_mlups")):
                nx, ny = (200, 100) if prec == lbm.LBM_F64 else (size, size)
                p = lbm.lbm_params_default(model, precision=prec, **kw)
                ctx = lbm.Context(p, nx, ny, stream=stream)
                _, th = ctx.derived()
                ctx.set_density(inputs.two_droplets(nx, ny, [(nx / 4, ny / 2), (3 * nx / 4, ny / 2)], ny / 4,
                                                    th.rho_v, th.rho_l))
                ctx.set_drive(5e-6, -5e-6, nx // 2, 0)
                ctx.step(128)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                n = 20000 if prec == lbm.LBM_F64 else 256
                torch.cuda.synchronize()
                e0.record(stream)
                ctx.step(n)
                e1.record(stream)
                torch.cuda.synchronize()
                sec = e0.elapsed_time(e1) * 1e-3
                col.setdefault(key, {})[pk] = n / sec if prec == lbm.LBM_F64 else nx * ny * n / sec / 1e6
                if prec == lbm.LBM_F32:
                    col[key]["f32_4096_frac_of_hbm"] = BYTES_PER_CELL[model] * nx * ny * n / sec / 1e9 / peak
                ctx.close()
        out["collision_sec54"] = col
        # full free-energy model (A != 0: strain rate of u at the neighbours), FP32 droplet
        p = lbm.lbm_params_default(1, precision=lbm.LBM_F32, a=0.25, Tr=0.8, tau_nu=1.0, tau_e=0.9, A=0.15)
        ctx = lbm.Context(p, size, size, stream=stream)
        _, th = ctx.derived()
        ctx.set_density(inputs.droplet(size, size, size / 4, th.rho_v, th.rho_l))
        ctx.step(64)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.step(256)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3 / 256
        out["free_energy_A_f32"] = {"kernel": "fe_iwb_pair", "mlups": size * size / sec / 1e6,
                                    "frac_of_hbm": BYTES_PER_CELL[1] * size * size / sec / 1e9 / peak}
        ctx.close()
    return out


def run_surrogate(args):
    """Learned calibration surrogate: label seeded parameter sets (Tr, a, b, kappa_P) with the
    batched solver (flat slab + three width-scaled droplets each), train the MLP on the GPU,
    and measure it against the calibration runs of 256 held-out sets (batched; a sample of them
    also through the plain one-lattice-at-a-time API, which must agree bitwise).  Reports the
    per-set cost of a plain calibration, of a batched one, and of a surrogate query (4096
    queries per fused BF16 launch, CUDA events), held-out errors, and the gain over the
    no-network theory (Maxwell densities) at Tr <= 0.6."""
    import torch

    from paper_2403_11167_gb300 import calibration as C
    from paper_2403_11167_gb300 import inputs

    tr = inputs.surrogate_sets(args.surrogate_sets, seed=4032)
    ho = inputs.surrogate_sets(256, seed=1116)
    r = C.calibrate_batched(tr)
    rh = C.calibrate_batched(ho)
    k = args.plain_sets
    rp = C.calibrate_plain(ho[:k])
    plain_equal = bool(np.array_equal(rp["Y"], rh["Y"][:k], equal_nan=True))
    X, ok = C.features(tr), r["ok"]
    m, loss, t_train = C.fit_surrogate(X[ok], r["Y"][ok])
    Xh, okh = C.features(ho), rh["ok"]
    P = m.predict(Xh)
    err = C.relative_errors(P[okh], rh["Y"][okh])
    sig = np.isfinite(err[:, 3])
    # inference: 4096 queries resident on the device, one fused launch each, events on the stream
    q = torch.from_numpy(C.features(inputs.surrogate_sets(4096, seed=777)).astype(np.float32)).cuda()
    out = torch.empty_like(q)
    stream = torch.cuda.current_stream()
    for _ in range(5):
        m.predict_device(q, out, stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 200
    e0.record(stream)
    for _ in range(reps):
        m.predict_device(q, out, stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    infer_us = e0.elapsed_time(e1) * 1e3 / reps
    e0.record(stream)
    for _ in range(reps):
        m.predict_device(q, out, stream.cuda_stream, mode=1)
    e1.record(stream)
    torch.cuda.synchronize()
    infer_single_us = e0.elapsed_time(e1) * 1e3 / reps
    T = C.theory(ho)
    low = okh & (Xh[:, 0] <= 0.6)
    e_th = np.abs(T[low, 1] / rh["Y"][low, 1] - 1)
    e_nn = np.abs(P[low, 1] / rh["Y"][low, 1] - 1)
    m.close()
    plain_per_set = rp["seconds"] / k
    return {
        "training_sets": len(tr), "training_sets_valid": int(ok.sum()),
        "training_sets_with_sigma": int(np.isfinite(r["Y"][ok, 3]).sum()),
        "label_seconds_batched": r["seconds"], "label_lattice_updates": r["updates"],
        "label_glups": r["updates"] / r["seconds"] / 1e9,
        "train_seconds": t_train, "train_final_loss": loss,
        "held_out_sets": len(ho), "held_out_valid": int(okh.sum()), "held_out_with_sigma": int(sig.sum()),
        "max_rel_err": {"rho_l": float(err[:, 0].max()), "rho_v": float(err[:, 1].max()),
                        "width": float(err[:, 2].max()), "sigma": float(err[sig, 3].max())},
        # per width factor: sets with a sigma label and their largest sigma error (sigma's domain
        # is kappa_P >= 0.7; kappa_P = 0.4 calibration droplets mostly diverge)
        "sigma_by_kappa_P": {f"{k:g}": {"held_out_valid": int((Xh[okh, 3] == k).sum()),
                                        "with_sigma": int((sig & (Xh[okh, 3] == k)).sum()),
                                        "max_rel_err": (float(err[sig & (Xh[okh, 3] == k), 3].max())
                                                        if (sig & (Xh[okh, 3] == k)).any() else None)}
                             for k in (0.4, 0.7, 1.0)},
        "mean_rel_err": {"rho_l": float(err[:, 0].mean()), "rho_v": float(err[:, 1].mean()),
                         "width": float(err[:, 2].mean()), "sigma": float(err[sig, 3].mean())},
        "gain_rho_v_Tr_le_0.6": {"sets": int(low.sum()), "theory_mean_rel_err": float(e_th.mean()),
                                 "surrogate_mean_rel_err": float(e_nn.mean())},
        "seconds_per_set": {"plain_calibration": plain_per_set, "batched_calibration": rh["seconds"] / len(ho),
                            "surrogate_query": infer_us * 1e-6 / 4096},
        "plain_sample_sets": k, "plain_equals_batched_bitwise": plain_equal,
        "inference_us_per_4096_queries": infer_us, "inference_mode": "split-BF16 operands, FP32 accumulation",
        "inference_us_per_4096_queries_single_bf16": infer_single_us,
        "workload": f"{len(tr)} training + 256 held-out seeded pseudopotential parameter sets (Tr U[0.5,0.95], "
                    "a U[0.25,0.5], b U[3,5], kappa_P in {0.4,0.7,1}); per set a 256x4 slab (4e4 and 5e4 steps) "
                    "and three droplets R = 3l, 4l, 5l on 16l lattices, l = max(W_theory, 4)",
    }


KERNEL_SOURCES = ("lbm_kernels.cuh", "ring.cuh", "step_pair.cuh")


def kernel_source_hash():
    """First 12 hex digits of the SHA-256 of the step kernels' sources (per-cell arithmetic, the
    row ring and the strip kernels), concatenated in KERNEL_SOURCES order."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2403_11167_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def profiled_traffic(kernel):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary, if it was taken
    on the current kernel source (matching hash); else None."""
    path = os.path.join(ROOT, "profiles", "step_kernels_ncu.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"kernel_source_sha256_12:\s*([0-9a-f]{12})", text)
    if not m or m.group(1) != kernel_source_hash():
        return None
    m = re.search(rf"traffic_per_launch_4096\[{kernel}\]:\s*([0-9.eE+]+)", text)
    return float(m.group(1)) if m else None


def measured_peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    if ws > 1:
        torch.distributed.barrier()
    from paper_2403_11167_gb300 import lbm

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    size, nsteps = args.size, args.lbm_steps
    ncell = size * size
    _, th = lbm.lbm_resolve_params(lbm.lbm_params_default(0, a=0.25, Tr=0.85, tau_nu=0.8))
    rho0 = make_rho0(size, th.rho_v, th.rho_l)
    stream = torch.cuda.Stream()
    ctxs = []
    for model in (0, 1):
        p = lbm.lbm_params_default(model, precision=lbm.LBM_F32, a=0.25, Tr=0.85, tau_nu=0.8)
        ctxs.append(lbm.Context(p, size, size, stream=stream))
    rho0_dev = torch.from_numpy(rho0.astype(np.float32)).cuda()
    rho0_pinned = torch.from_numpy(rho0).pin_memory()
    rho0_pinned_np = rho0_pinned.numpy()

    def one_step(events=None):
        for m, ctx in enumerate(ctxs):
            ctx.set_density_device(rho0_dev)
            if events is not None:
                events[m][0].record(stream)
            ctx.step(nsteps)
            if events is not None:
                events[m][1].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
        barrier()
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.3)
        barrier()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kev = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(2)]
               for _ in range(args.steps)]
        t0.record(stream)
        for k in range(args.steps):
            one_step(kev[k])
        t1.record(stream)
        barrier()
        clocks = sampler.stop()
        elapsed_ms = t0.elapsed_time(t1)
        per_model_ms = [sum(kev[k][m][0].elapsed_time(kev[k][m][1]) for k in range(args.steps)) for m in range(2)]

    elapsed_ms = max_over_ranks(elapsed_ms, ws, device="cuda")
    updates_per_rank = args.steps * 2 * nsteps * ncell
    updates = ws * updates_per_rank
    value = job_rate(updates_per_rank, ws, elapsed_ms * 1e-3) / 1e6

    # end to end through the public API: pinned host rho0 -> H2D -> steps -> observables D2H
    e2e = None
    if not args.no_e2e:
        barrier()
        t = time.perf_counter()
        for _ in range(args.steps):
            for ctx in ctxs:
                ctx.set_density(rho0_pinned_np)
                ctx.step(nsteps)
                ctx.observables(0)
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t, ws, device="cuda")
        e2e = {"value": job_rate(updates_per_rank, ws, e2e_s) / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": 2 * ncell * 8,
               "d2h_bytes_per_step": 2 * 8 * 8}

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    names = ["pp_step_pair", "fe_step_pair"]
    per_launch_s = [ms * 1e-3 / (args.steps * nsteps) for ms in per_model_ms]
    dom = int(np.argmax(per_model_ms))
    peak, peak_kind = measured_peak_gbs()
    achieved = BYTES_PER_CELL[dom] * ncell / per_launch_s[dom] / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profiled_traffic(names[dom]), "kernel": names[dom], "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": BYTES_PER_CELL[dom] * ncell}
    per_model = {}
    for m, key in enumerate(("pseudopotential", "free_energy")):
        per_model[key] = {"mlups": ncell / per_launch_s[m] / 1e6, "us_per_launch": per_launch_s[m] * 1e6,
                          "algorithmic_bytes_per_cell": BYTES_PER_CELL[m],
                          "gbs": BYTES_PER_CELL[m] * ncell / per_launch_s[m] / 1e9,
                          "frac_of_hbm": BYTES_PER_CELL[m] * ncell / per_launch_s[m] / 1e9 / peak}
    sweep = None
    if not args.no_sweep:
        sweep = run_sweep(args)
    surrogate = None
    if not args.no_surrogate:
        surrogate = run_surrogate(args)
    walls = None
    if not args.no_walls:
        walls = run_walls(args, peak)
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        v, cores, sample, _ = oracle_mlups(size, args.cpu_seconds)
        cpu = {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample}
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": args.steps * (2 + 2 * nsteps), "clocks": clocks, "per_model": per_model,
        "sweep": sweep, "surrogate": surrogate, "walls": walls,
        "kernel_source_sha256_12": kernel_source_hash(),
    }
    print(json.dumps(line))
    for ctx in ctxs:
        ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_profile(args):
    """Small fixed workload for ncu captures of one step kernel (see --profile)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2403_11167_gb300 import inputs, lbm

    model = lbm.LBM_PSEUDOPOTENTIAL if args.profile == "pp" else lbm.LBM_FREE_ENERGY
    p = lbm.lbm_params_default(model, precision=lbm.LBM_F32, a=0.25, Tr=0.85, tau_nu=0.8, A=args.A)
    ctx = lbm.Context(p, args.size, args.size)
    _, th = ctx.derived()
    ctx.set_density(inputs.spinodal_noise(args.size, args.size, 0.5 * (th.rho_l + th.rho_v), 0.01, seed=2403))
    for _ in range(args.steps):
        ctx.step(1)
    ctx.synchronize()
    torch.cuda.synchronize()
    print("profile workload done:", args.profile, args.size, args.steps)
    ctx.close()


def main():
    args = parse()
    if args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
