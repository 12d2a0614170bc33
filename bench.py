"""Benchmark of the multiphase LBM hot path on GB300.

Workload (N = 1): 2048 x 1024 lattice, cylinder R = 300 centred on the bottom boundary, drop
r = 150 resting on it, body force 1e-6 toward the cylinder (sessile), wall wetting drawn from
seed 0, FP32 populations with FP64 reductions; one bench step = one time step (fused step kernel),
the contact angle measured on the device every 500 steps inside the timed region.

Metric: MLUPS (million lattice-node updates per second, all nx * ny nodes), higher is better.
The device-timed region uses CUDA events on the library's stream; the working set (2 x 75.5 MB of
populations + 2 x 8 MB of density + geometry, 170 MB) is larger than the 126 MB L2, so no L2
flush is inserted between steps. ``e2e`` repeats the run through the C ABI from host buffers:
geometry and a host initial density in, angles and the final density out.

N > 1 (torchrun): every rank runs an independent instance (seed = rank) with no data-path
collective; value = all ranks' node updates / the slowest rank's time (weak scaling). The
batched, sweep and warm-start workloads instead split their independent instances over the
ranks in contiguous ranges (paper_2202_06516_gb300/shard.py) and gather the per-instance results
on rank 0 (strong scaling of a fixed instance set).

--impl reference: the FP64 CPU oracle on the host cores on the same workload, for a bounded
number of steps.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURE_EVERY = 500
# sources of the step kernel: a committed ncu summary applies only while these are unchanged
STEP_KERNEL_SRCS = [os.path.join(ROOT, "paper_2202_06516_gb300", "csrc", f)
                    for f in ("lbm_step.cu", "lbm_step_body.cuh", "lbm_internal.cuh")]
PROFILE = os.path.join(ROOT, "profiles", "k_step_fp32_2048x1024.md")
BYTES_PER_FLUID_NODE = 80  # 9 x 4 B populations read + written, 4 B density read + written


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _src_hash():
    h = hashlib.sha256()
    for p in STEP_KERNEL_SRCS:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _profiled_traffic():
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if it was taken
    on the current kernel source (None otherwise)."""
    try:
        txt = open(PROFILE).read()
    except OSError:
        return None
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not h or not b or h.group(1) != _src_hash():
        return None
    return float(b.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 6:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[2 + k]
                          and "Not" not in r[2 + k]})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(rows[0][1]) if rows[0][1].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(value: float, dist, device) -> float:
    """The slowest rank's time (barrier-synchronised max-reduction); value itself at N = 1."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def rank_workload(rank: int):
    """Each rank runs its own independent instance: the 2048 x 1024 workload seeded by rank."""
    from paper_2202_06516_gb300 import workloads as W
    return W.plain_large(seed=rank)


def _resolve(w, lbm_mod):
    m = w.model
    co = lbm_mod.lbm_coexistence(m["eos"], m["Tr"])
    neutral = m["k2"] * co["mu_sat"]
    return co, neutral


def _make_lattice(lbm, w, stream=None, tile=(0, 0), min_blocks=0):
    m = w.model
    co, neutral = _resolve(w, lbm)
    lat = lbm.Lattice(w.nx, w.ny, eos=m["eos"], Tr=m["Tr"], k2=m["k2"], kappa=m["kappa"],
                      tau=m["tau"], s_e=m["s_e"], s_eps=m["s_eps"], s_q=m["s_q"], gx=w.g[0],
                      gy=w.g[1], stream=stream, tile=tile, min_blocks=min_blocks,
                      g_rho_ref=co["rho_g"] if w.buoyant else 0.0)
    geo = dict(circle=w.circle, mu_circle=neutral + w.mu_rel_circle,
               mu_bottom=neutral + w.mu_rel_bottom, mu_top=neutral + w.mu_rel_top, drop=w.drop,
               stripes=(w.stripes[0], neutral + w.stripes[1]) if w.stripes else None,
               concave=w.concave)
    return lat, geo


def run_cuda(args, rank, world, dist):
    import torch
    from paper_2202_06516_gb300 import lbm, workloads as W

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    w = rank_workload(rank)
    stream = torch.cuda.Stream(device=dev)
    lat, geo = _make_lattice(lbm, w, stream=stream, tile=args.tile, min_blocks=args.min_blocks)
    lat.set_geometry(**geo)
    tune = None
    if args.tile == (0, 0) and args.min_blocks == 0:
        tune = lat.autotune(20)   # picks the step-kernel variant on this workload's own state
    tile = (lat.info().tile_x, lat.info().tile_y, lat.info().min_blocks)
    n_nodes = w.nx * w.ny
    n_fluid = int(lat.info().n_fluid)

    def run(k):
        left = k
        done = 0
        nmeas = 0
        while left > 0:
            chunk = min(left, MEASURE_EVERY - (done % MEASURE_EVERY))
            lat.step(chunk)
            done += chunk
            left -= chunk
            if done % MEASURE_EVERY == 0:
                lat.measure()
                nmeas += 1
        return nmeas

    run(args.warmup)
    lat.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        t0.record(stream)
        nmeas = run(args.steps)
        t1.record(stream)
        t1.synchronize()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    # step kernel alone (graph-replayed back-to-back launches) for the roofline
    k2 = max(256, min(args.steps, 4000))
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    lat.step(k2)
    k1.record(stream)
    k1.synchronize()
    kernel_us = k0.elapsed_time(k1) * 1e3 / k2
    st, mres = lbm.lbm_mass(lat.ctx, allow_unstable=True)
    stable = st == lbm.LBM_OK
    angles = lat.measure()
    lat.close()
    ms = max_over_ranks(ms, dist, f"cuda:{dev}")

    # end to end through the C ABI from host buffers (rank-local, not part of the device timing)
    e2e = None
    if rank == 0:
        co, _ = _resolve(w, lbm)
        j, i = np.mgrid[0:w.ny, 0:w.nx].astype(np.float64)
        d = np.sqrt((i - w.drop[0]) ** 2 + (j - w.drop[1]) ** 2)
        # the step's input and result live in pinned host memory (the copies run at full speed
        # and no page is first touched inside the timed region)
        rho0 = torch.empty((w.ny, w.nx), dtype=torch.float64, pin_memory=True).numpy()
        rho0[:] = 0.5 * (co["rho_g"] + co["rho_l"]) + 0.5 * (co["rho_g"] - co["rho_l"]) * \
            np.tanh(2.0 * (d - w.drop[2]) / w.drop[3])
        rho_out = torch.zeros((w.ny, w.nx), dtype=torch.float64, pin_memory=True).numpy()
        lat2, geo2 = _make_lattice(lbm, w, stream=stream, tile=tile[:2], min_blocks=tile[2])
        lat2.set_geometry(**geo2)
        lat2.step(max(3, args.warmup))
        lat2.synchronize()
        ke = args.steps
        tt = time.perf_counter()
        lat2.set_geometry(**geo2, rho0=rho0)
        nm = 0
        done = 0
        while done < ke:
            c = min(ke - done, MEASURE_EVERY - (done % MEASURE_EVERY))
            lat2.step(c)
            done += c
            if done % MEASURE_EVERY == 0:
                lat2.measure()
                nm += 1
        lat2.rho(out=rho_out)
        te = time.perf_counter() - tt
        lat2.close()
        ang_bytes = 2 * 104
        e2e = {"value": n_nodes * ke / te / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": rho0.nbytes / ke,
               "d2h_bytes_per_step": (rho_out.nbytes + nm * ang_bytes) / ke,
               "what": "lbm_set_geometry(pinned host rho0) + lbm_step + "
                       "lbm_measure_contact_angle every 500 steps + lbm_read_fields(rho into "
                       "pinned host memory), host wall clock"}

    peak, peak_kind = _peaks()
    achieved = BYTES_PER_FLUID_NODE * n_fluid / (kernel_us * 1e-6) / 1e9
    traffic = _profiled_traffic()
    line = {
        "metric": "MLUPS", "value": n_nodes * args.steps * world / (ms * 1e-3) / 1e6,
        "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name.rsplit("-s", 1)[0], "nx": w.nx, "ny": w.ny,
                   "fluid_nodes": n_fluid, "measure_every": MEASURE_EVERY,
                   "value_counts": "all nx*ny nodes (the disc's solid nodes included); the "
                                   "roofline counts fluid nodes only",
                   "fluid_mlups": n_fluid * args.steps * world / (ms * 1e-3) / 1e6,
                   "precision": "FP32 populations (deviation form), FP64 reductions/angles",
                   "l2": "working set 170 MB > L2, no flush", "parallelism": f"replicas{world}",
                   "eos": "Peng-Robinson Tr=0.7", "seed": "rank",
                   "autotune_us_per_step": None if tune is None else {
                       f"{r['tile'][0]}x{r['tile'][1]}/{r['min_blocks']}": round(r["us_per_step"], 2)
                       for r in tune}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": f"k_step<float,{tile[0]},{tile[1]}> min_blocks={tile[2]}",
                     "kernel_us_per_launch": kernel_us,
                     "bytes_per_launch": BYTES_PER_FLUID_NODE * n_fluid},
        "e2e": e2e,
        "gpu_launches": args.steps + 4 * nmeas,
        "clocks": clk.summary(),
        "stable": stable,
        "angles_deg": [round(angles[0].theta, 3), round(angles[1].theta, 3)],
    }
    return line


def cpu_baseline(steps: int = 400, warmup: int = 2):
    """The oracle as it stands on the host cores: the same 2048 x 1024 workload, `warmup`
    untimed steps, then `steps` timed time steps (a bounded sample of the 50k-step run)."""
    import oracle as O
    from paper_2202_06516_gb300 import workloads as W
    w = W.plain_large(0)
    m = w.model
    mx = O.maxwell(m["eos"], m["Tr"])
    neutral = m["k2"] * mx["mu_sat"]
    cfg = O.Config(nx=w.nx, ny=w.ny, **{k: m[k] for k in ("eos", "Tr", "k2", "kappa", "tau", "s_e",
                                                           "s_eps", "s_q")},
                   gx=w.g[0], gy=w.g[1], rho_g=mx["rho_g"], rho_l=mx["rho_l"], has_circle=1,
                   cx=w.circle[0], cy=w.circle[1], R=w.circle[2],
                   mu_circle=neutral + w.mu_rel_circle, mu_bottom=neutral, mu_top=neutral,
                   drop_x=w.drop[0], drop_y=w.drop[1], drop_r=w.drop[2], drop_W=w.drop[3])
    s = O.Sim(cfg)
    if warmup > 0:
        s.step(warmup)
    t = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t
    return {"value": w.nx * w.ny * steps / dt / 1e6, "unit": "MLUPS", "cores": O.threads(),
            "kind": "oracle", "sample": f"{steps} FP64 oracle steps of the 2048x1024 workload",
            "seconds": dt}


def run_reference(args):
    """--impl reference: the oracle on the host cores, bounded so the run ends in minutes."""
    from paper_2202_06516_gb300 import workloads as W
    w = W.plain_large(0)
    steps = max(1, min(args.steps, 200))
    warm = max(0, min(args.warmup, 3))
    cb = cpu_baseline(steps, warm)
    return {"metric": "MLUPS", "value": cb["value"], "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": cb["seconds"] * 1e3 / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name.rsplit("-s", 1)[0], "nx": w.nx, "ny": w.ny,
                       "device": "host cores (FP64 oracle), rank 0 only"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_batched(args, rank=0, world=1, dist=None):
    """256-instance sweep (domains 128..768 x 128..512, R 20..200, r 15..90, target angle 30..150
    degrees): all instances advance together in the batched kernel (grid mode and tile from the
    autotuner); value = all instances' node updates per second over args.steps steps (no early
    exit in the timed run), then (--converge) a convergence run (residual < 1e-6 per 500 steps
    or the angle rule, at most 40k steps) reports steps and angles per instance.
    Under torchrun the instances are split over the ranks in contiguous ranges balanced by
    lattice nodes, each rank runs its own batch, and the per-instance results are gathered on
    rank 0; the timed region is the slowest rank's."""
    import torch
    from paper_2202_06516_gb300 import lbm, shard, workloads as W
    ws_all = W.batched(args.instances, seed=0)
    lo, hi = shard.partition([w.nx * w.ny for w in ws_all], world, rank)
    ws = ws_all[lo:hi]
    m = ws_all[0].model
    co = lbm.lbm_coexistence(m["eos"], m["Tr"])
    neutral = m["k2"] * co["mu_sat"]

    def make():
        bb = lbm.Batch([(w.nx, w.ny) for w in ws], eos=m["eos"], Tr=m["Tr"], k2=m["k2"],
                       kappa=m["kappa"], tau=m["tau"], s_e=m["s_e"], s_eps=m["s_eps"],
                       s_q=m["s_q"])
        for i, w in enumerate(ws):
            bb.set_geometry(i, circle=w.circle, mu_circle=neutral + w.mu_rel_circle,
                            mu_bottom=neutral, mu_top=neutral, drop=w.drop)
        return bb

    b = make() if ws else None
    fluid_local = sum(lbm.lbm_get_info(lbm.lbm_batch_instance(b.b, i)).n_fluid
                      for i in range(len(ws))) if ws else 0
    tune = b.autotune(20) if ws else []
    if ws:
        b.run(max(4, args.warmup // 2 * 2), check_every=max(2, args.warmup // 2 * 2), tol=0.0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t = time.perf_counter()
    if ws:
        b.run(args.steps, check_every=500, tol=0.0)
    torch.cuda.synchronize()
    dt_local = time.perf_counter() - t
    dt = shard.max_over_ranks(dt_local, dist)
    fluid = sum(shard.gather([fluid_local], dist) or [fluid_local]) if dist else fluid_local
    nodes = sum(w.nx * w.ny for w in ws_all)
    line = {"metric": "MLUPS", "value": nodes * args.steps / dt / 1e6, "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched-{args.instances}-instances", "total_nodes": nodes,
                       "fluid_nodes": fluid,
                       "parallelism": f"instances split over {world} rank(s), contiguous ranges "
                                      "balanced by nodes, results gathered on rank 0",
                       "timing": "host wall clock around the synchronous batch run, slowest rank",
                       "autotune_us_per_step": {
                           f"{r['tile'][0]}x{r['tile'][1]}/{r['min_blocks']}"
                           f"{' persistent' if r['persistent'] else ' per-tile'}":
                           round(r["us_per_step"], 2) for r in tune}}}
    peak, kind = _peaks()
    ach = BYTES_PER_FLUID_NODE * fluid * args.steps / dt / 1e9
    line["roofline"] = {"bound": "hbm", "achieved": ach / world, "peak": peak, "unit": "GB/s",
                        "frac": ach / world / peak, "traffic": None, "peak_kind": kind,
                        "kernel": "k_batch_step (autotuned tile)",
                        "note": "80 B per fluid node over host wall time per GPU, residual "
                                "checks every 500 steps included"}
    if b is not None:
        b.close()
    if args.converge:
        rows = []
        t = time.perf_counter()
        if ws:
            b2 = make()
            steps, conv, res = b2.run(40000, check_every=500, tol=1e-6, angle_tol=0.05)
            ang = b2.measure()
            rows = [(lo + i, int(steps[i]), bool(conv[i]),
                     ang[i][0].status == 0 and ang[i][1].status == 0,
                     [ang[i][0].theta, ang[i][1].theta]) for i in range(len(ws))]
            b2.close()
        dt2 = shard.max_over_ranks(time.perf_counter() - t, dist)
        rows = shard.gather(rows, dist)
        if rows is not None:
            assert [r[0] for r in rows] == list(range(len(ws_all)))
            line["converge"] = {"seconds": dt2, "converged": sum(r[2] for r in rows),
                                "steps_mean": float(np.mean([r[1] for r in rows])),
                                "steps_max": max(r[1] for r in rows),
                                "angles_ok": sum(r[3] for r in rows)}
    return line


def _sweep_one(args, Tr, rank=0, world=1, dist=None):
    """One temperature of the curvature sweep: returns (node updates, seconds, summary); None
    on ranks other than 0 under torchrun (instances split over the ranks, rows gathered)."""
    import torch
    from paper_2202_06516_gb300 import lbm, shard, workloads as W, contact_mechanics as CM
    ws_all = W.curvature_sweep()
    lo, hi = shard.partition([w.nx * w.ny for w in ws_all], world, rank)
    ws = ws_all[lo:hi]
    m = dict(ws_all[0].model, Tr=Tr)
    co = lbm.lbm_coexistence(m["eos"], m["Tr"])
    neutral = m["k2"] * co["mu_sat"]
    rows = []
    if dist:
        dist.barrier()
    t = time.perf_counter()
    if ws:
        b = lbm.Batch([(w.nx, w.ny) for w in ws], eos=m["eos"], Tr=m["Tr"], k2=m["k2"],
                      kappa=m["kappa"], tau=m["tau"], s_e=m["s_e"], s_eps=m["s_eps"],
                      s_q=m["s_q"], tile_auto=True)
        for i, w in enumerate(ws):
            b.set_geometry(i, circle=w.circle, mu_circle=neutral + w.mu_rel_circle,
                           mu_bottom=neutral, mu_top=neutral, drop=w.drop, concave=w.concave)
        torch.cuda.synchronize()
        t = time.perf_counter()
        steps, conv, res = b.run(args.sweep_steps, check_every=1000, tol=0.0, angle_tol=0.05)
        torch.cuda.synchronize()
    dt = shard.max_over_ranks(time.perf_counter() - t, dist)
    if ws:
        ang = b.measure()
        for i, w in enumerate(ws):
            l, r = ang[i]
            row = {"name": w.name, "concave": w.concave, "R": w.circle[2], "r": w.drop[2],
                   "target": float(w.name.rsplit("theta", 1)[1]), "steps": int(steps[i]),
                   "converged": bool(conv[i]), "ok": l.status == 0 and r.status == 0,
                   "updates": w.nx * w.ny * int(steps[i])}
            if row["ok"]:
                row.update(left=l.theta, right=r.theta, theta=0.5 * (l.theta + r.theta),
                           alpha=0.5 * (l.alpha + r.alpha), beta=0.5 * (l.beta + r.beta))
                ctx = lbm.lbm_batch_instance(b.b, i)
                _, pd = lbm.lbm_read_candidates(ctx, w.nx, w.ny)
                try:
                    row["cap"] = CM.cap_angle(pd[:, :2], pd[:, 2], w.circle,
                                              concave=w.concave)["theta"]
                except ValueError:
                    row["cap"] = None
            rows.append(row)
        b.close()
    rows = shard.gather(rows, dist)
    if rows is None:
        return None
    assert [r["name"] for r in rows] == [w.name for w in ws_all]
    ws = ws_all
    steps = np.array([r["steps"] for r in rows])
    conv = np.array([r["converged"] for r in rows])
    updates = sum(r.pop("updates") for r in rows)
    groups = {}
    for row in rows:
        if row["ok"]:
            groups.setdefault(("cavity" if row["concave"] else "cylinder", row["target"]),
                              []).append(row)
    by_group = {}
    for (kind, target), g in sorted(groups.items()):
        th = np.array([x["theta"] for x in g])
        by_group[f"{kind}-{target:g}"] = {"n": len(g), "mean": float(th.mean()),
                                          "std": float(th.std()), "min": float(th.min()),
                                          "max": float(th.max())}
    errs = {}
    for kind in ("cylinder", "cavity"):
        for subset in ("all", "converged"):
            pairs = [(x["theta"], x["cap"]) for x in rows
                     if x["ok"] and x.get("cap") is not None and
                     ("cavity" if x["concave"] else "cylinder") == kind and
                     (subset == "all" or x["converged"])]
            if pairs:
                a = np.array(pairs)
                errs[f"{kind}-{subset}"] = {
                    "n": len(a),
                    "E": float(np.sqrt(((a[:, 0] - a[:, 1]) ** 2).sum() / (a[:, 1] ** 2).sum())),
                    "mean_diff_deg": float((a[:, 0] - a[:, 1]).mean()),
                    "max_abs_deg": float(np.abs(a[:, 0] - a[:, 1]).max())}
    summary = {"seconds": dt, "converged": int(conv.sum()), "instances": len(ws),
               "angles_ok": int(sum(x["ok"] for x in rows)), "steps_mean": float(steps.mean()),
               "total_nodes": sum(w.nx * w.ny for w in ws), "by_group": by_group,
               "present_vs_cap": errs, "instances_detail": rows if args.sweep_detail else None}
    return updates, dt, summary


def run_sweep(args, rank=0, world=1, dist=None):
    """Grid-independence and curvature sweep (Sec. 4.1-4.2): drops of 30-100 lu on convex
    cylinders and in cavities of radius 150-400 lu for five wall potentials, all instances
    advanced together by the persistent batched kernel until their angles settle (two
    consecutive readings 1,000 steps apart within 0.05 degrees) or args.sweep_steps; then the
    device measurement against the spherical-cap method (Sec. 4.1) on the same fields. One
    batch per reduced temperature in args.sweep_tr."""
    temps = [float(t) for t in args.sweep_tr.split(",")]
    total_u, total_t, per = 0, 0.0, {}
    for Tr in temps:
        res = _sweep_one(args, Tr, rank, world, dist)
        if res is None:
            continue
        u, dt, summ = res
        total_u += u
        total_t += dt
        per[f"Tr={Tr:g}"] = summ
    if rank != 0:
        return None
    n_inst = next(iter(per.values()))["instances"]
    return {"metric": "MLUPS", "value": total_u / total_t / 1e6, "unit": "MLUPS", "n_gpus": world,
            "steps": args.sweep_steps, "warmup": 0, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"curvature-sweep-{n_inst}-instances",
                       "temperatures": temps,
                       "parallelism": f"instances split over {world} rank(s), rows gathered",
                       "timing": "host wall clock around each synchronous batch run (autotune, "
                                 "angle checks every 1,000 steps included)"},
            "sweep": per}


def run_gravity(args):
    """Gravity independence of the microscopic angle (Sec. 4.3): the same drops (radius 20-120 on
    a cylinder of radius 150, three wall potentials) without body force, sessile and pendent, each
    setting one persistent batched run until the angles settle; per instance the device
    measurement and the spherical-cap estimate of the same field."""
    import torch
    from paper_2202_06516_gb300 import lbm, workloads as W, contact_mechanics as CM
    sw = W.gravity_sweep()
    ws = sw["instances"]
    m = ws[0].model
    co = lbm.lbm_coexistence(m["eos"], m["Tr"])
    neutral = m["k2"] * co["mu_sat"]
    per, t_all, upd = {}, 0.0, 0
    for gname, g in sw["g"].items():
        b = lbm.Batch([(w.nx, w.ny) for w in ws], eos=m["eos"], Tr=m["Tr"], k2=m["k2"],
                      kappa=m["kappa"], tau=m["tau"], s_e=m["s_e"], s_eps=m["s_eps"],
                      s_q=m["s_q"], gx=g[0], gy=g[1], tile_auto=True)
        for i, w in enumerate(ws):
            b.set_geometry(i, circle=w.circle, mu_circle=neutral + w.mu_rel_circle,
                           mu_bottom=neutral, mu_top=neutral, drop=w.drop)
        torch.cuda.synchronize()
        t = time.perf_counter()
        steps, conv, res = b.run(args.gravity_steps, check_every=1000, tol=0.0, angle_tol=0.05)
        torch.cuda.synchronize()
        t_all += time.perf_counter() - t
        upd += sum(w.nx * w.ny * int(s) for w, s in zip(ws, steps))
        ang = b.measure()
        rows = []
        for i, w in enumerate(ws):
            l, r = ang[i]
            row = {"target": float(w.name.rsplit("theta", 1)[1]), "r": w.drop[2],
                   "steps": int(steps[i]), "converged": bool(conv[i]),
                   "contact": l.status == 0 and r.status == 0}
            if row["contact"]:
                row["theta"] = 0.5 * (l.theta + r.theta)
                _, pd = lbm.lbm_read_candidates(lbm.lbm_batch_instance(b.b, i), w.nx, w.ny)
                try:
                    row["cap"] = CM.cap_angle(pd[:, :2], pd[:, 2], w.circle)["theta"]
                except ValueError:
                    row["cap"] = None
            rows.append(row)
        b.close()
        per[gname] = rows
    summary = {}
    for gname, rows in per.items():
        for t in sorted({x["target"] for x in rows}):
            sel = [x for x in rows if x["target"] == t and x["contact"]]
            th = np.array([x["theta"] for x in sel])
            cp = np.array([x["cap"] for x in sel if x.get("cap") is not None])
            summary[f"{gname}-{t:g}"] = {
                "drops_with_contact": len(sel),
                "present_mean": float(th.mean()) if th.size else None,
                "present_range": float(th.max() - th.min()) if th.size else None,
                "cap_mean": float(cp.mean()) if cp.size else None,
                "cap_range": float(cp.max() - cp.min()) if cp.size else None,
                "by_radius": {f"{x['r']:g}": [round(x["theta"], 2),
                                              None if x.get("cap") is None else round(x["cap"], 2)]
                              for x in sel}}
    return {"metric": "MLUPS", "value": upd / t_all / 1e6, "unit": "MLUPS", "n_gpus": 1,
            "steps": args.gravity_steps, "warmup": 0, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"gravity-sweep-{len(ws)}-drops-x3",
                       "g": {k: list(v) for k, v in sw["g"].items()},
                       "timing": "host wall clock around the three synchronous batch runs"},
            "gravity": summary}


def run_boundary(args):
    """Staircase sensitivity of the equilibrium angle under the two curved-wall schemes: the same
    drop (r = 40) on cylinders whose radius (R, R + 1/2) and centre (offsets of 0 or 1/2 in x and
    y) change only how the circle falls on the lattice; the spread of the measured angle over
    these discretisations, with half-way and with interpolated bounce-back."""
    import torch
    from paper_2202_06516_gb300 import lbm, workloads as W, contact_mechanics as CM
    m = W.MODEL
    out, t0 = {}, time.perf_counter()
    for name, bnd in (("halfway", lbm.LBM_BB_HALFWAY), ("interpolated", lbm.LBM_BB_INTERP)):
        for target in (70.0, 110.0):
            th, failed = [], []
            for R in (100.0, 100.5):
                for off in ((0.0, 0.0), (0.5, 0.0), (0.0, 0.5), (0.5, 0.5)):
                    try:
                        res = CM.intrinsic_angle(m, W.mu_rel_for_angle(target), R=R, r=40.0,
                                                 steps=args.boundary_steps, samples=5,
                                                 every=1000, boundary=bnd, offset=off)
                        th.append(res["theta"])
                    except RuntimeError:
                        failed.append([R, *off])
            th = np.array(th)
            out[f"{name}-{target:g}"] = {"n": len(th), "mean": float(th.mean()),
                                         "std": float(th.std()),
                                         "range": float(th.max() - th.min()),
                                         "values": [round(float(v), 3) for v in th],
                                         "no_contact": failed}
    torch.cuda.synchronize()
    return {"metric": "angle spread over discretisations", "value": None, "unit": "deg",
            "n_gpus": 1, "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "staircase-sensitivity-R100-r40",
                       "steps": args.boundary_steps, "seconds": time.perf_counter() - t0},
            "boundary": out}


def unet_flops(H, Wd, base):
    """Multiply-add FLOPs of one forward pass (2 per MAC) of the U-Net."""
    from paper_2202_06516_gb300 import workloads as W
    res = [1, 1, 2, 2, 4, 4, 8, 8, 4, 4, 4, 2, 2, 2, 1, 1, 1]  # downsampling factor per conv
    f = 0
    for (ci, co), d in zip(W.unet_layers(base), res):
        f += 2 * (H // d) * (Wd // d) * 9 * ci * co
    return f + 2 * H * Wd * base


def _young_summary(mech, tension, skip, theta_c, stripes, scatter):
    """Eq. 17 force statistics per contact line and wall region (after `skip` samples)."""
    names = {0: "theta_%g" % theta_c, 1: "theta_%g" % stripes[1] if stripes else "-", 2: "border"}
    out = {"gamma": tension["gamma"], "laplace_spread": tension["spread"],
           "interface_width_10_90": tension["width_10_90"],
           "equilibrium_angles": {"circle": theta_c, "stripes": stripes[1] if stripes else None},
           "equilibrium_angle_scatter": scatter}
    for side, label in (("right", "advancing"), ("left", "receding")):
        f, reg = mech[side]["force"][skip:], mech[side]["region"][skip:]
        d = {}
        for k, nm in names.items():
            v = f[reg == k]
            if v.size:
                d[nm] = {"samples": int(v.size), "mean": float(v.mean()),
                         "min": float(v.min()), "max": float(v.max())}
        out[label] = d
    return out


def run_hysteresis(args):
    """Dynamic contact-angle hysteresis on the striped (or uniform) 4096 x 1024 cylinder: the
    drop is driven along the surface and the advancing (right) and receding (left) angles are
    measured on the device every 100 steps. Reports the stepping rate including the measurements
    and the angle statistics once the initial cap has relaxed (after 10k steps)."""
    import torch
    from paper_2202_06516_gb300 import lbm, workloads as W, contact_mechanics as CM
    w = W.hysteresis(heterogeneous=not args.homogeneous)
    steps, every = args.hyst_steps, w.measure_every
    # Eq. 17-18 inputs, untimed: liquid-gas tension (free drops) and the intrinsic angle of each
    # wall wettability (uniform-wall equilibrium drops)
    tension = CM.laplace_tension(w.model)
    R_c, r_d = w.circle[2], w.drop[2]
    intrinsic = [CM.intrinsic_angle(w.model, w.mu_rel_circle, R=R_c, r=r_d)]
    if w.stripes:
        intrinsic.append(CM.intrinsic_angle(w.model, w.stripes[1], R=R_c, r=r_d))
    stream = torch.cuda.Stream()
    lat, geo = _make_lattice(lbm, w, stream=stream, tile=(lbm.LBM_TILE_AUTO, 0))
    lat.set_geometry(**geo)
    lat.step(max(2, args.warmup // 2 * 2))   # autotunes, then a few steps
    m0 = lat.mass()
    rows, diverged = [], None
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    with ClockSampler(0) as clk:
        try:
            for k in range(steps // every):
                lat.step(every)
                st, (l, r) = lbm.lbm_measure_contact_angle(lat.ctx)
                m = lat.mass()
                rows.append((l.status, l.theta_deg, r.status, r.theta_deg, l.contact_x,
                             r.contact_x, l.contact_y, r.contact_y, m["mass"], m["cx"],
                             m["cy"]))
        except lbm.LbmError as e:
            diverged = {"after_step": (len(rows) + 1) * every, "error": str(e)}
        t1.record(stream)
        t1.synchronize()
    ms = t0.elapsed_time(t1)
    lat.close()
    arr = np.array(rows, dtype=np.float64).reshape(-1, 11)
    theta_c = intrinsic[0]["theta"]
    stripes = (w.stripes[0], intrinsic[1]["theta"]) if w.stripes else None
    mech = CM.analyse_series(arr[:, :8], w.circle, theta_c, stripes, tension["gamma"],
                             tension["width_10_90"])
    if args.series:
        step = (np.arange(len(rows)) + 1) * every
        cols = [step, arr]
        for side in ("left", "right"):
            cols += [mech[side]["theta_eq"], mech[side]["phi_d"], mech[side]["force"]]
        np.savetxt(args.series, np.column_stack(cols), delimiter=",", fmt="%.6f",
                   header="step,left_status,theta_left,right_status,theta_right,"
                          "contact_x_left,contact_x_right,contact_y_left,contact_y_right,"
                          "mass,liquid_cx,liquid_cy,theta_eq_left,phi_d_left,force_x_left,"
                          "theta_eq_right,phi_d_right,force_x_right", comments="")
    steps = len(rows) * every
    # statistics after the initial 90-degree cap has relaxed (first 10k steps left out)
    late = arr[10000 // every:]
    ok = (late[:, 0] == 0) & (late[:, 2] == 0)
    adv, rec = late[ok, 3], late[ok, 1]

    def stats(v):
        if v.size == 0:
            return None
        p05, p50, p95 = np.percentile(v, [5, 50, 95])
        return {"mean": float(v.mean()), "min": float(v.min()), "p05": float(p05),
                "median": float(p50), "p95": float(p95), "max": float(v.max())}
    return {"metric": "MLUPS", "value": w.nx * w.ny * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS",
            "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": ms / max(steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "measure_every": every,
                       "g": list(w.g), "body_force": "(rho - rho_g) g",
                       "timing": "CUDA events around stepping plus one synchronous angle "
                                 "measurement and mass sum every 100 steps"},
            "clocks": clk.summary(),
            "hysteresis": {"samples": len(rows), "valid_after_10k_steps": int(ok.sum()),
                           "theta_advancing": stats(adv), "theta_receding": stats(rec),
                           "hysteresis": stats(adv - rec),
                           "no_contact_samples": int(((arr[:, 0] != 0) | (arr[:, 2] != 0)).sum()),
                           "liquid_centroid_travel_lu": (float(arr[-1, 9] - m0["cx"])
                                                         if len(rows) else None),
                           "mass_drift_rel": (float(arr[-1, 8] / m0["mass"] - 1.0)
                                              if len(rows) else None),
                           "diverged": diverged},
            "young_force": _young_summary(mech, tension, 10000 // every, theta_c, stripes,
                                          [t["scatter"] for t in intrinsic])}


def run_surrogate(args):
    """Warm-start U-Net alone (base 32, 256 x 256, batch args.batch, seeded synthetic inputs):
    args.steps training steps (forward, loss, backward, Adam) and as many forward passes, timed
    on the host around the library's synchronous calls."""
    import torch
    from paper_2202_06516_gb300 import lbm, workloads as W
    B, H = args.batch, 256
    sur = lbm.Surrogate(H, H, base=32, max_batch=B)
    sur.set_weights(W.unet_init(32, seed=0))
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand((B, H, H, 8), device="cuda", generator=g).to(torch.bfloat16)
    t = torch.rand((B, H, H), device="cuda", generator=g)
    m = (torch.rand((B, H, H), device="cuda", generator=g) > 0.2).to(torch.uint8)
    phi = torch.zeros((B, H, H), device="cuda")
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        sur.train_step(x.data_ptr(), t.data_ptr(), m.data_ptr(), B, 1e-4)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sur.train_step(x.data_ptr(), t.data_ptr(), m.data_ptr(), B, 1e-4)
    t_train = (time.perf_counter() - t0) / args.steps
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sur.forward(x.data_ptr(), B, phi.data_ptr())
    t_fwd = (time.perf_counter() - t0) / args.steps
    sur.close()
    f = unet_flops(H, H, 32) * B
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak, kind = float(json.load(fh)["bf16_tflops"]), "measured"
    except Exception:
        peak, kind = 1900.0, "fallback"
    ach = 3 * f / t_train / 1e12
    return {"metric": "TFLOP/s", "value": ach, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_train * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": f"unet-base32-256x256-batch{B}",
                       "flops_per_train_step": 3 * f, "timing": "host wall clock around the "
                       "synchronous training and forward calls"},
            "forward": {"ms": t_fwd * 1e3, "tflops": f / t_fwd / 1e12},
            "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak, "traffic": None, "peak_kind": kind,
                         "note": "whole training step; the 32-128-channel layers with short K "
                                 "leave the implicit-GEMM loaders, not the tensor cores, as "
                                 "the limit"}}


def time_to_angle_leg(args):
    """The second half of the metric on a bounded sample, so that every default run records it:
    a surrogate trained on args.tta_train solver-equilibrated 256 x 256 cases, then args.tta_cases
    held-out cases (the warm-start workload's seeds) run to args.tta_steps steps three ways: plain
    single-instance lattices one after another, the batched solver from the Eq. 16 start, and the
    batched solver from the network's prediction; steps and wall-clock seconds to the +-0.5 deg
    equilibrated angle of the plain run (see the warm-start workload). Not part of the timed
    region of the main line."""
    from paper_2202_06516_gb300 import lbm, warmstart as WS, workloads as W
    t0 = time.perf_counter()
    tr = W.warm_cases(args.tta_train, seed=1)
    ev = W.warm_cases(args.tta_cases, seed=10000)
    x, t, m = WS.generate(tr, steps=args.tta_steps)
    t_gen = time.perf_counter() - t0
    sur = lbm.Surrogate(256, 256, base=32, max_batch=8)
    sur.set_weights(W.unet_init(32, seed=0))
    losses, t_train = WS.train(sur, x, t, m, epochs=args.tta_epochs, batch=8, lr=args.lr)
    rows, extra = WS.evaluate(sur, ev, steps=args.tta_steps, every=250)
    sur.close()
    out = WS.summarise(rows, extra)
    out["config"] = {"train_cases": len(tr), "eval_cases": len(ev), "horizon_steps": args.tta_steps,
                     "epochs": args.tta_epochs, "lattice": "256x256", "network": "U-Net base 32",
                     "generation_seconds": round(t_gen, 2), "training_seconds": round(t_train, 2),
                     "loss_first_last": [losses[0], losses[-1]],
                     "criterion": "first check (every 250 steps, both sides) after which every later "
                                  "check stays within 0.5 deg of the plain run's final angle"}
    return out


def run_warmstart(args, rank=0, world=1, dist=None):
    """Learned warm start (256 x 256 cases) and the time to the equilibrated angle: generate
    equilibria with the batched solver, train the BF16 U-Net with the library's kernels, then on
    held-out seeds measure steps and wall-clock seconds to the +-0.5 degree equilibrated angle
    (the plain cold run's final angle) for the plain single-instance solver (one lattice per
    case, one after another), the batched solver from the Eq. 16 start, and the batched solver
    from the network's prediction. Under torchrun the training-case generation and the held-out
    evaluation are split over the ranks (contiguous ranges), the data and the per-case results
    gathered on rank 0, which trains; the trained weights are broadcast for the evaluation."""
    from paper_2202_06516_gb300 import lbm, shard, warmstart as WS, workloads as W
    log = (lambda msg: print(msg, file=sys.stderr, flush=True)) if rank == 0 else None
    t0 = time.perf_counter()
    tr = W.warm_cases(args.train_cases, seed=1)
    ev = W.warm_cases(args.eval_cases, seed=10000)
    lo, hi = shard.partition([1.0] * len(tr), world, rank)
    part = WS.generate(tr[lo:hi], steps=args.gen_steps) if hi > lo else None
    parts = shard.gather([part] if part is not None else [], dist)
    t_gen = shard.max_over_ranks(time.perf_counter() - t0, dist)
    weights = None
    info = {}
    if rank == 0:
        x = np.concatenate([p_[0] for p_ in parts])
        t = np.concatenate([p_[1] for p_ in parts])
        m = np.concatenate([p_[2] for p_ in parts])
        log(f"generated {len(tr)} cases in {t_gen:.1f}s")
        sur = lbm.Surrogate(256, 256, base=32, max_batch=args.batch)
        sur.set_weights(W.unet_init(32, seed=0))
        losses, t_train = WS.train(sur, x, t, m, epochs=args.epochs, batch=args.batch,
                                   lr=args.lr, log=log)
        steps_per_epoch = len(tr) // args.batch
        flops = 3 * unet_flops(256, 256, 32) * args.batch * steps_per_epoch * args.epochs
        weights = sur.weights()
        sur.close()
        info = {"loss_first_last": [losses[0], losses[-1]], "train_seconds": t_train,
                "train_tflops": flops / t_train / 1e12}
    weights = shard.broadcast(weights, dist)
    sur = lbm.Surrogate(256, 256, base=32, max_batch=args.batch)
    sur.set_weights(weights)
    lo, hi = shard.partition([1.0] * len(ev), world, rank)
    rows, extra = (WS.evaluate(sur, ev[lo:hi], steps=args.gen_steps, every=250,
                               plain=not args.no_plain) if hi > lo else ([], {}))
    sur.close()
    rows = shard.gather(rows, dist)
    extras = shard.gather([extra], dist)
    if rank != 0:
        return None
    tta = WS.summarise(rows, WS.merge_extra(extras))
    line = {"metric": "time to +-0.5 deg equilibrated angle (held-out 256x256 cases)",
            "impl": "cuda", "workload": "warm-start-256x256", "data": "synthetic",
            "n_gpus": world, "train_cases": len(tr), "eval_cases": len(ev),
            "epochs": args.epochs, "gen_seconds": t_gen, **info,
            "criterion": "first angle check (every 250 steps, both sides) after which every "
                         "later check lies within 0.5 deg of the plain cold run's final angle "
                         f"after {args.gen_steps} steps",
            "time_to_angle": tta}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=500)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=400)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile", type=lambda v: tuple(int(t) for t in v.split("x")), default=(0, 0),
                    help="step-kernel tile, e.g. 32x16 (default: the library's)")
    ap.add_argument("--workload", default="single", choices=["single", "batched", "warmstart", "surrogate",
                                                    "hysteresis", "sweep", "boundary",
                                                    "gravity"])
    ap.add_argument("--train-cases", type=int, default=1024)
    ap.add_argument("--eval-cases", type=int, default=64)
    ap.add_argument("--gen-steps", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--converge", action="store_true")
    ap.add_argument("--no-tta", action="store_true",
                    help="default workload: skip the bounded time-to-angle leg")
    ap.add_argument("--tta-train", type=int, default=1024)
    ap.add_argument("--tta-cases", type=int, default=64)
    ap.add_argument("--tta-steps", type=int, default=30000)
    ap.add_argument("--tta-epochs", type=int, default=20)
    ap.add_argument("--no-plain", action="store_true",
                    help="warmstart workload: skip the plain single-instance runs")
    ap.add_argument("--hyst-steps", type=int, default=200000)
    ap.add_argument("--sweep-steps", type=int, default=60000)
    ap.add_argument("--boundary-steps", type=int, default=30000)
    ap.add_argument("--gravity-steps", type=int, default=60000)
    ap.add_argument("--sweep-tr", default="0.7",
                    help="sweep workload: comma-separated reduced temperatures")
    ap.add_argument("--sweep-detail", action="store_true",
                    help="sweep workload: include every instance's angles in the JSON line")
    ap.add_argument("--series", default=None,
                    help="hysteresis workload: write the angle series to this CSV file")
    ap.add_argument("--homogeneous", action="store_true",
                    help="hysteresis workload on a uniform 120-degree wall")
    ap.add_argument("--min-blocks", type=int, default=0,
                    help="step-kernel CTAs per SM to fit registers to (0: none)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return

    dist = None
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        td.init_process_group("nccl")
        dist = td
    from paper_2202_06516_gb300 import _native
    if rank == 0:
        _native.build()
    if dist:
        dist.barrier()  # the other ranks load the library rank 0 has just built
    if args.workload == "batched":
        line = run_batched(args, rank, world, dist)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload == "warmstart":
        line = run_warmstart(args, rank, world, dist)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload == "surrogate":
        if rank == 0:
            print(json.dumps(run_surrogate(args)), flush=True)
        return
    if args.workload == "hysteresis":
        if rank == 0:
            print(json.dumps(run_hysteresis(args)), flush=True)
        return
    if args.workload == "sweep":
        line = run_sweep(args, rank, world, dist)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload == "boundary":
        if rank == 0:
            print(json.dumps(run_boundary(args)), flush=True)
        return
    if args.workload == "gravity":
        if rank == 0:
            print(json.dumps(run_gravity(args)), flush=True)
        return
    if dist:
        dist.barrier()
    line = run_cuda(args, rank, world, dist)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_steps)
        if world == 1 and not args.no_tta:
            line["time_to_angle"] = time_to_angle_leg(args)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
