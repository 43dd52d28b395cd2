"""Benchmark of the MHD + H/H2 chemistry time step (arXiv:1608.08748) on GB300.

Workload (one "step" = one full time step of the method over the whole box):
  decaying supersonic MHD turbulence with hydrogen chemistry, 128^3 periodic cells, FP64,
  n = 100 cm^-3, T = 100 K, rms Mach 5, beta 1, seed 1, CFL 0.4 (synthetic initial state).
Metric: Mcell-updates/s = cells x steps / device time of the timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank advances its own box (independent replicas, no collective on the
data path) and the line reports the sum over ranks with the slowest rank's time.
`--impl reference` times the FP64 CPU oracle (the plain implementation the tests check against) on
the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CFL = 0.4
N_GRID = 128
WORKLOAD = "mhd_turbulence_h2chem_128^3_fp64"
METRIC = "Mcell-updates/s"
# FP64 peak of a GB300: 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz (max SM clock); the
# FMA-chain peak measured in the run (mhd_probe_fma_peak) is reported beside it
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 peak: 152 SMs x 128 FP32 FMA lanes x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# algorithmic HBM bytes of one cell-update of the unfused substage model (129 field accesses with
# chemistry: each of the six RK substages reads its inputs and the RK register and writes its
# outputs once; the post pass reads the face fields), FP64 and FP32 bulk
BYTES_PER_CELL_UPDATE = {8: 1032, 4: 516}
# the copy bandwidth used when the measured peaks are not available
HBM_FALLBACK_GBS = 6800.0
# algorithmic FP64 flops of one Eulerian face, counted from the kernel source with an FMA as two
# flops and a division, square root or reciprocal square root as one (compares and selects not
# counted): the parabolas of the six primitives of one new cell, streamed along the pencil (6 x 32:
# differences, halved slope, edge value and second difference 11, Steps 2-5 18, the Step 4 test 3),
# the Riemann solve (Roe average, speeds and eigenvector rows 116; the three wave pairs'
# domain-of-dependence averages with L q and R s 244) and the fluxes (25)
FLOPS_PER_EULER_FACE = 577
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one Eulerian face launch at 128^3,
# the mean of the x, y and z launches of one ncu capture of this kernel (358.1, 256.2, 260.9 MB;
# profiles/kb_metrics_turbulence_128_fp64.md; set to None whenever the kernel changes)
EULER_FACE_TRAFFIC_BYTES = 291.7e6
# FP32 bulk: FP32 flops of one Eulerian face (fadd + fmul + 2 ffma executed per face, 795-796 in
# the three directions of one ncu capture of kb_euler_pencil<float> at 128^3) and the DRAM bytes of
# one 256^3 launch: the mean of the 128^3 capture's x, y, z launches (175.7, 110.0, 114.0 MB) times
# 8, the ratio of the faces processed (profiles/kb_metrics_turbulence_128_fp32bulk.md)
FP32_FLOPS_PER_EULER_FACE = 796
EULER_FACE_TRAFFIC_BYTES_FP32 = 133.2e6 * 8


def hbm_peak():
    """(GB/s, source) of the HBM roofline: the measured copy bandwidth of the GB300s when
    the measured-peaks file is present, else the fallback figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        if v > 0:
            return v, "measured (STREAM-style copy)"
    except (OSError, ValueError, KeyError, TypeError):
        pass
    return HBM_FALLBACK_GBS, "fallback"


def hbm_roofline(bytes_per_update, cells, ms_per_step):
    """Whole-step HBM roofline: algorithmic bytes of one step over its time, against the peak."""
    peak, src = hbm_peak()
    achieved = bytes_per_update * cells / (ms_per_step * 1e-3) / 1e9
    return {"bound": "hbm", "scope": "whole step (algorithmic bytes / step time)",
            "bytes_per_cell_update": bytes_per_update, "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "peak_source": src}


def reduce_max(x, dist=None, device="cpu"):
    """Largest value of x over all ranks (the slowest rank's time); x itself without a group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, cells_per_rank, steps, seconds):
    """Whole-job Mcell-updates/s: every rank advances its own box of cells_per_rank cells."""
    return world * cells_per_rank * steps / seconds / 1e6


def rank_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def sample_clocks(stop, out):
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return
    def reader():
        for line in p.stdout:
            out.append(line.strip())
    th = threading.Thread(target=reader, daemon=True)
    th.start()
    stop.wait()
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    th.join(timeout=5)


def summarize_clocks(lines, gpu_index):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9 or f[0] != str(gpu_index):
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
            "samples": len(sm)}


def oracle_rate(n, steps, warm=1, threads=None):
    """Oracle Mcell-updates/s on an n^3 box of the same turbulence set-up (all host cores, or
    `threads` OpenMP threads); returns (rate, cores, seconds)."""
    from oracle import oracle as O
    from paper_1608_08748_gb300 import inputs as I
    ic = I.turbulence(n, mach=5.0, beta=1.0, seed=1)
    opts = {} if threads is None else {"threads": threads}
    s = O.run(ic, **opts)
    for _ in range(warm):
        s.step(CFL)
    t0 = time.perf_counter()
    for _ in range(steps):
        s.step(CFL)
    dt = time.perf_counter() - t0
    cores = os.cpu_count() if threads is None else threads
    return n ** 3 * steps / dt / 1e6, cores, dt


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1608_08748_gb300 import inputs as I
    n = 64  # bounded sample of the 128^3 workload: same set-up on a 64^3 box
    ic = I.turbulence(n, mach=5.0, beta=1.0, seed=1)
    s = O.run(ic)
    for _ in range(args.warmup):
        s.step(CFL)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step(CFL)
    dt = time.perf_counter() - t0
    value = n ** 3 * args.steps / dt / 1e6
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "grid": [N_GRID] * 3, "cfl": CFL,
                                        "sample": f"{n}^3 box of the same set-up"},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                         "sample": f"{n}^3 turbulence box, {args.steps} steps after {args.warmup} warm-up"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def rel_l1_fields(a, b):
    """Per-field relative L1 of state a against reference b (scales as in the parity tests)."""
    rho = b["rho"]
    vscale = np.sqrt(max(np.mean(2.0 * np.abs(b["E"]) / rho), 1e-300))
    brms = np.sqrt(np.mean(b["B"] ** 2))
    sc = {"rho": rho.mean(), "E": np.abs(b["E"]).mean(), "mom": rho.mean() * vscale,
          "B": brms if brms > 0 else 1.0, "rho_h2": rho.mean()}
    f = lambda x, y, s: float(np.abs(x - y).sum() / max(np.abs(y).sum(), y.size * s))
    out = {k: f(a[k], b[k], sc[k]) for k in ["rho", "E", "rho_h2"]}
    for c, ax in enumerate("xyz"):
        out["m" + ax] = f(a["mom"][c], b["mom"][c], sc["mom"])
        out["B" + ax] = f(a["B"][c], b["B"][c], sc["B"])
    return out


def timed_steps(torch, sim, steps, warm):
    stream = torch.cuda.Stream()
    sim.set_stream(stream.cuda_stream)
    for _ in range(warm):
        sim.step(CFL, sync=False)
    sim.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        sim.step(CFL, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    sim.sync()
    return e0.elapsed_time(e1)


def fp32_leg(M, I, torch, n=256, steps=10, warm=3, err_steps=100):
    """Config 3: the same turbulence set-up at n^3 with the FP32-bulk path.  Per-field error
    against the FP64 GPU path from the same initial state after err_steps steps (the FP64 path
    matches the FP64 oracle element by element; the oracle itself is checked against the FP32 path
    at 64^3 over the same 100 steps in the GPU tests)."""
    ic = I.turbulence(n, mach=5.0, beta=1.0, seed=1)
    s32 = M.from_ic(ic, precision=1)
    ms = timed_steps(torch, s32, steps, warm)
    prof = M.profile(s32, CFL, 2)
    del s32
    a = M.from_ic(ic, precision=1)
    b = M.from_ic(ic, precision=0)
    for _ in range(err_steps):
        a.step(CFL, sync=False)
        b.step(CFL, sync=False)
    a.sync()
    b.sync()
    err = rel_l1_fields(a.get_state(), b.get_state())
    t32, t64 = a.diagnostics()["t"], b.diagnostics()["t"]
    del a, b
    ms_step = ms / steps
    kernels = {k: v["ms_total"] / 2 for k, v in prof.items()}
    dominant = max((k for k in kernels if k != "small"), key=lambda k: kernels[k])
    roof = None
    if FP32_FLOPS_PER_EULER_FACE:
        faces = (n + 1) * n * n
        launch_s = prof["euler_face"]["ms_total"] / prof["euler_face"]["launches"] * 1e-3
        measured = M.probe_fma_peak(fp64=False)
        achieved = FP32_FLOPS_PER_EULER_FACE * faces / launch_s / 1e12
        roof = {"bound": "alu", "kernel": "kb_euler_pencil (FP32)", "achieved": achieved,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                "traffic": EULER_FACE_TRAFFIC_BYTES_FP32, "flops_per_face": FP32_FLOPS_PER_EULER_FACE,
                "peak_source": "derived: 152 SM x 128 FP32 FMA/clk x 2 flop x 2.07 GHz",
                "peak_measured": measured, "frac_of_measured": achieved / measured,
                "share_of_step": kernels["euler_face"] / sum(kernels.values())}
    return {"workload": f"mhd_turbulence_h2chem_{n}^3_fp32bulk", "value": n ** 3 * steps / (ms * 1e-3) / 1e6,
            "unit": METRIC, "ms_per_step": ms_step, "steps": steps, "warmup": warm,
            "roofline_hbm": hbm_roofline(BYTES_PER_CELL_UPDATE[4], n ** 3, ms_step),
            "roofline": roof, "dominant_kernel": dominant,
            "rel_l1_vs_fp64_100steps": err, "error_steps": err_steps,
            "t_after_error_steps": {"fp32": t32, "fp64": t64},
            "kernels": kernels}


def heatcool_leg(M, I, torch, n=128, steps=10, warm=3):
    """The heating/cooling stage (Sec. 2.8) on the FP64 128^3 turbulence box with 5 % of the
    hydrogen molecular: Mcell-updates/s with the stage on and off, and the post kernel (chemistry,
    heating/cooling, regularisation, CFL) per step."""
    ic = I.turbulence(n, mach=5.0, beta=1.0, seed=1)
    ic["rho_h2"] = 0.05 * ic["rho"]
    out = {"workload": f"mhd_turbulence_h2chem_heatcool_{n}^3_fp64", "unit": METRIC, "steps": steps,
           "warmup": warm}
    for on in (1, 0):
        s = M.from_ic(ic, heatcool=on)
        ms = timed_steps(torch, s, steps, warm)
        prof = M.profile(s, CFL, 2)
        key = "on" if on else "off"
        out[key] = {"value": n ** 3 * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps,
                    "post_ms_per_step": prof["post"]["ms_total"] / 2}
        del s
    out["value"] = out["on"]["value"]
    return out


def ions_leg(M, I, torch, n=128, steps=10, warm=3):
    """The ionisation network (reactions 5-8 with H+ and e, Sec. 4.3 / App. D) with heating/cooling
    (Gamma_1-Lambda_8) on the FP64 128^3 turbulence box with 5 % of the hydrogen molecular and an
    ion fraction of 1e-3: Mcell-updates/s with the ions on and off (heating/cooling on in both), and
    the post kernel per step."""
    ic = I.turbulence(n, mach=5.0, beta=1.0, seed=1)
    ic["rho_h2"] = 0.05 * ic["rho"]
    ic["rho_hp"] = 1e-3 * ic["rho"]
    out = {"workload": f"mhd_turbulence_h2chem_ions_heatcool_{n}^3_fp64", "unit": METRIC, "steps": steps,
           "warmup": warm}
    for on in (1, 0):
        s = M.from_ic(ic, heatcool=1, ions=on)
        ms = timed_steps(torch, s, steps, warm)
        prof = M.profile(s, CFL, 2)
        out["on" if on else "off"] = {"value": n ** 3 * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps,
                                      "post_ms_per_step": prof["post"]["ms_total"] / 2,
                                      "lag_face_ms_per_step": prof["lag_face"]["ms_total"] / 2}
        del s
    out["value"] = out["on"]["value"]
    return out


def gravity_leg(M, I, torch, n=128, steps=10, warm=3):
    """Self-gravity (Sec. 2.10 Poisson solve by cuFFT each step, gravity terms in the Eulerian stage)
    on the FP64 128^3 turbulence box with G in code units (pc, km/s, m_H cm^-3): Mcell-updates/s
    with and without it."""
    G_CODE = 6.6743e-8 * 1.6735575e-24 * (3.0856775814913673e18 / 1e5) ** 2
    ic = I.turbulence(n, mach=5.0, beta=1.0, seed=1)
    out = {"workload": f"mhd_turbulence_h2chem_gravity_{n}^3_fp64", "unit": METRIC, "steps": steps,
           "warmup": warm, "G_code": G_CODE}
    for on in (1, 0):
        s = M.from_ic(ic, grav_g=G_CODE if on else 0.0)
        ms = timed_steps(torch, s, steps, warm)
        out["on" if on else "off"] = {"value": n ** 3 * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps}
        del s
    out["value"] = out["on"]["value"]
    return out


def batched_leg(M, I, torch, steps=20, warm=3):
    """Config 4: 64 turbulence boxes, axes from {16..96}, FP32 bulk, one launch per kernel class
    per step (CUDA graph), launch shapes autotuned first."""
    sims = []
    for b in I.ensemble_boxes():
        ic = I.turbulence(8, mach=b["mach"], beta=b["beta"], seed=b["seed"], shape=b["shape"])
        sims.append(M.from_ic(ic, precision=1))
    cells = sum(int(np.prod(s.shape)) for s in sims)
    batch = M.Batch(sims)
    tuned = batch.tune(CFL, reps=1)
    shapes = {k: batch.shape(k) for k in M.mhd.KERNEL_CLASSES[:7]}
    for _ in range(warm):
        batch.step(CFL)
    batch.sync()
    t0 = time.perf_counter()
    for _ in range(steps):
        batch.step(CFL)
    batch.sync()
    dt = time.perf_counter() - t0
    prof = batch.profile(CFL, 2)
    batch.close()
    return {"workload": "ensemble_64_boxes_fp32bulk", "boxes": len(sims), "cells": cells,
            "value": cells * steps / dt / 1e6, "unit": METRIC, "ms_per_step": dt / steps * 1e3,
            "steps": steps, "tuned_ms_per_step": tuned, "tuned_shapes": shapes,
            "kernels": {k: v["ms_total"] / 2 for k, v in prof.items()}}


def serving_leg(M, I, torch, duration=10.0, big=True, policy="fifo", rate=20.0):
    """Config 5: Poisson arrivals (20 requests/s, seed 5) of turbulence runs, cubic n in
    {32..192} and 512 with probability 0.005 (when big), 20-200 steps, FP32 bulk, submitted in real
    time to the continuous-batching server.  Velocity fields: one cached solenoidal field per size,
    shifted periodically per request.  Besides p50/p99 time-to-result it reports the service time
    (admission to result) and the queueing delay (submission to admission) per size class, and the
    admission log's summary."""
    arr = [r for r in I.serving_arrivals(rate=rate, big_prob=0.005 if big else 0.0) if r["t"] < duration]
    base = {}
    for n in sorted({r["n"] for r in arr}):
        base[n] = I.solenoidal_field((n, n, n), seed=n)
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * 0.6)
    srv = M.Server(budget, max_active=64)
    srv.set_policy(policy)
    rng = np.random.default_rng(5)
    ids = []
    t0 = time.perf_counter()
    for r in arr:
        ic = I.turbulence_from_field(base[r["n"]], mach=r["mach"], beta=r["beta"],
                                     shift=rng.integers(0, r["n"], 3))
        while time.perf_counter() - t0 < r["t"]:
            time.sleep(0.001)
        ids.append((srv.submit(ic, nsteps=r["steps"], precision=1), r))
    srv.drain(3600)
    wall = time.perf_counter() - t0
    lat, work, first, last = [], 0, None, None
    failed = {}
    classes = {}
    for rid, r in ids:
        rc, res = srv.poll(rid)
        if rc != 0:
            key = f"status {rc} (n={r['n']}, mach={r['mach']:.1f}, beta={r['beta']:.2f})"
            failed[key] = failed.get(key, 0) + 1
            continue
        lat.append(res["t_done"] - res["t_submit"])
        work += res["cells"] * res["steps_done"]
        first = res["t_submit"] if first is None else min(first, res["t_submit"])
        last = res["t_done"] if last is None else max(last, res["t_done"])
        n = r["n"]
        cls = "512" if n == 512 else ("32-64" if n <= 64 else ("72-128" if n <= 128 else "136-192"))
        c = classes.setdefault(cls, {"service_s": [], "queue_s": [], "rate": []})
        svc = res["t_done"] - res["t_admit"]
        c["service_s"].append(svc)
        c["queue_s"].append(res["t_admit"] - res["t_submit"])
        c["rate"].append(res["cells"] * res["steps_done"] / max(svc, 1e-9) / 1e6)
    st = srv.stats()
    srv.close()
    lat = np.array(lat)
    table = {k: {"requests": len(v["service_s"]), "service_p50_s": float(np.median(v["service_s"])),
                 "service_p99_s": float(np.percentile(v["service_s"], 99)),
                 "queue_p50_s": float(np.median(v["queue_s"])),
                 "per_request_mcell_updates_s_p50": float(np.median(v["rate"]))}
             for k, v in sorted(classes.items())}
    return {"workload": f"serving_poisson_{rate:g}rps_fp32bulk", "requests": len(ids), "completed": len(lat),
            "stream_s": duration, "big_512": bool(big), "requests_512": sum(1 for _, r in ids if r["n"] == 512),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "value": work / (last - first) / 1e6, "unit": METRIC, "wall_s": wall,
            "by_size": table,
            "admission": {"hbm_budget_bytes": budget, "peak_bytes": st["peak_bytes"],
                          "peak_active": st["peak_active"], "scheduler_iterations": st["iterations"],
                          "max_active": 64},
            "failed": failed, "policy": policy}


def steps_leg(M, I, torch, grid=128, precision=0, nsteps=4, graph=1):
    """A plain run of nsteps steps of the turbulence box at grid^3 (no timing): the case the ncu
    captures of profiles/ run, small enough for a multi-pass capture."""
    ic = I.turbulence(grid, mach=5.0, beta=1.0, seed=1)
    s = M.from_ic(ic, precision=precision, graph=graph)
    for _ in range(nsteps):
        s.step(CFL, sync=False)
    s.sync()
    return {"workload": f"mhd_turbulence_h2chem_{grid}^3_{'fp32bulk' if precision else 'fp64'}",
            "steps": nsteps, "t": s.diagnostics()["t"]}


def run_leg(args):
    """One secondary leg alone (profiling): prints its JSON object."""
    import torch
    from paper_1608_08748_gb300 import build as B
    B.build()
    import paper_1608_08748_gb300 as M
    from paper_1608_08748_gb300 import inputs as I
    if args.leg == "steps":
        print(json.dumps({"steps": steps_leg(M, I, torch, args.grid, args.precision, args.nsteps,
                                             args.graph)}), flush=True)
        return
    fn = {"fp32": fp32_leg, "batched": batched_leg, "serving": serving_leg, "heatcool": heatcool_leg,
          "gravity": gravity_leg, "ions": ions_leg}[args.leg]
    kw = {"policy": args.serve_policy, "big": not args.no_serving_big} if args.leg == "serving" else {}
    print(json.dumps({args.leg: fn(M, I, torch, **kw)}), flush=True)


def run_ours(args):
    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1608_08748_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if dist:
        dist.barrier()
    import paper_1608_08748_gb300 as M
    from paper_1608_08748_gb300 import inputs as I

    ic = I.turbulence(N_GRID, mach=5.0, beta=1.0, seed=1 + rank)
    cells = N_GRID ** 3
    sim = M.from_ic(ic)
    stream = torch.cuda.Stream()
    sim.set_stream(stream.cuda_stream)
    for _ in range(args.warmup):
        sim.step(CFL, sync=False)
    sim.sync()

    stop = threading.Event()
    clk = []
    th = threading.Thread(target=sample_clocks, args=(stop, clk), daemon=True)
    th.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        sim.step(CFL, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    stop.set()
    th.join(timeout=10)
    sim.sync()
    ms = reduce_max(e0.elapsed_time(e1), dist, "cuda")
    value = job_rate(world, cells, args.steps, ms * 1e-3)
    launches = sim.L.mhd_launches_per_step(sim.h) * args.steps

    # end to end through the C-ABI with host buffers: per step, upload the state from pinned host
    # memory, one step, read the state back
    host = {k: torch.empty((3,) + ic["rho"].shape if k in ("mom", "B") else ic["rho"].shape,
                           dtype=torch.float64).pin_memory() for k in ["rho", "mom", "E", "B", "rho_h2"]}
    st0 = sim.get_state()
    for k in host:
        host[k].copy_(torch.from_numpy(st0[k]))
    hnp = {k: v.numpy() for k, v in host.items()}
    e2e_steps = max(3, min(args.steps, 10))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sim.set_state(hnp["rho"], hnp["mom"], hnp["E"], hnp["B"], hnp["rho_h2"])
        sim.step(CFL, sync=False)
        sim.get_state(out=hnp)
    torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, dist, "cuda")
    field_bytes = 9 * cells * 8
    e2e = {"value": job_rate(world, cells, e2e_steps, e2e_s), "unit": METRIC,
           "h2d_bytes_per_step": field_bytes, "d2h_bytes_per_step": field_bytes}

    # per-kernel device times (event pairs around each launch, separate pass, same workload)
    import ctypes
    prof_steps = 4
    kms = (ctypes.c_double * 8)()
    kn = (ctypes.c_int64 * 8)()
    sim.L.mhd_profile.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    rc = sim.L.mhd_profile(sim.h, CFL, prof_steps, kms, kn)
    names = ["prim", "euler_face", "edges", "euler_update", "lag_face", "lag_update", "post", "small"]
    kernels = {nm: {"ms_total": kms[c], "launches": int(kn[c])} for c, nm in enumerate(names)} if rc == 0 else {}
    tot = sum(v["ms_total"] for v in kernels.values()) or 1.0
    for v in kernels.values():
        v["share"] = v["ms_total"] / tot
    roofline = None
    if kernels:
        faces_per_launch = (N_GRID + 1) * N_GRID * N_GRID
        avg_launch_s = kernels["euler_face"]["ms_total"] / kernels["euler_face"]["launches"] * 1e-3
        achieved = FLOPS_PER_EULER_FACE * faces_per_launch / avg_launch_s / 1e12
        measured = M.probe_fma_peak(fp64=True)
        roofline = {"bound": "alu", "kernel": "kb_euler_pencil (FP64)", "achieved": achieved,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                    "traffic": EULER_FACE_TRAFFIC_BYTES,
                    "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                    "peak_measured": measured, "frac_of_measured": achieved / measured,
                    "peak_measured_source": "FP64 FMA chains timed here (mhd_probe_fma_peak)"}

    if rank != 0:
        return
    del sim
    extras = {}
    if world == 1 and not args.no_extras:
        extras["fp32_bulk"] = fp32_leg(M, I, torch)
        extras["batched"] = batched_leg(M, I, torch)
        extras["serving"] = serving_leg(M, I, torch, big=not args.no_serving_big, policy=args.serve_policy)
        # the same stream at a tenth of the rate, which the GPU sustains: latency is then service
        # time, not queueing
        extras["serving_sustained"] = serving_leg(M, I, torch, big=False, policy=args.serve_policy, rate=2.0)
        extras["heatcool"] = heatcool_leg(M, I, torch)
        extras["gravity"] = gravity_leg(M, I, torch)
        extras["ions"] = ions_leg(M, I, torch)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rate, cores, secs = oracle_rate(48, 8)
        rate1, _, secs1 = oracle_rate(32, 4, threads=1)
        cpu = {"value": rate, "unit": METRIC, "cores": cores, "kind": "oracle",
               "sample": f"48^3 box of the same turbulence set-up, 8 steps ({secs:.1f} s)",
               "one_core": {"value": rate1, "unit": METRIC, "cores": 1,
                            "sample": f"32^3 box of the same set-up, 4 steps ({secs1:.1f} s)"}}
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [N_GRID] * 3, "cfl": CFL, "chemistry": True,
                   "l2": "inputs larger than L2 (about 0.9 GB of fields and scratch per box)",
                   "parallelism": f"replicas x{world}"},
        "clocks": summarize_clocks(clk, local),
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": roofline,
        "roofline_hbm": hbm_roofline(BYTES_PER_CELL_UPDATE[8], cells, ms / args.steps),
        "cpu_baseline": cpu,
        "kernels": kernels,
    }
    line.update(extras)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP32-bulk (256^3), batched-ensemble, serving, heating/cooling and gravity legs")
    ap.add_argument("--leg", choices=["main", "fp32", "batched", "serving", "heatcool", "gravity", "ions", "steps"],
                    default="main",
                    help="run one secondary leg alone (for profiling); 'steps' runs --nsteps plain steps "
                         "of the turbulence box at --grid^3 in --precision (the ncu capture case)")
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--precision", type=int, choices=[0, 1], default=0)
    ap.add_argument("--nsteps", type=int, default=4)
    ap.add_argument("--graph", type=int, choices=[0, 1], default=1,
                    help="steps leg: 1 replays the captured graph, 0 launches kernel by kernel")
    ap.add_argument("--serve-policy", choices=["fifo", "smallest_work"], default="fifo",
                    help="admission order of the serving leg")
    ap.add_argument("--no-serving-big", action="store_true",
                    help="leave the 512^3 request class (probability 0.005) out of the serving leg")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.leg != "main":
        run_leg(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
