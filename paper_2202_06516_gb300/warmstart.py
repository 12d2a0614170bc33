"""Learned warm start: data generation with the batched solver, training of the U-Net with the
library's kernels, and the time-to-equilibrated-angle comparison of warm and cold starts.

Inputs per case (H x W x 8, BF16): channel 0 the solid mask, channel 1 the wall chemical
potential relative to the neutral wall (divided by 0.1) on the wetting layers, channel 2 the
initial liquid area divided by H W (a constant plane); geometry encodings derived from the
substrate: channel 3 the height y / H, channel 4 the horizontal offset from the cylinder axis
divided by W, channel 5 the distance to the substrate surface divided by 64 (clipped to 1),
channel 6 the wetting value of channel 1 spread over all nodes (the drop sees one wall
chemical potential), channel 7 zero. Target: the
equilibrated phi = (rho - rho_g) / (rho_l - rho_g), clipped to [0, 1], on fluid nodes (the loss
mask). Orchestration only; every numerical step runs in the library (solver, geometry, network).
"""
from __future__ import annotations

import time

import numpy as np

from . import lbm, workloads as W

MU_SCALE = 0.1


def _model_kw(m):
    return dict(eos=m["eos"], Tr=m["Tr"], k2=m["k2"], kappa=m["kappa"], tau=m["tau"],
                s_e=m["s_e"], s_eps=m["s_eps"], s_q=m["s_q"])


def _geometry(w, neutral):
    return dict(circle=w.circle, mu_circle=neutral + w.mu_rel_circle, mu_bottom=neutral,
                mu_top=neutral, drop=w.drop)


def make_batch(ws, rho0=None):
    m = ws[0].model
    co = lbm.lbm_coexistence(m["eos"], m["Tr"])
    neutral = m["k2"] * co["mu_sat"]
    b = lbm.Batch([(w.nx, w.ny) for w in ws], **_model_kw(m))
    for i, w in enumerate(ws):
        b.set_geometry(i, **_geometry(w, neutral), rho0=None if rho0 is None else rho0[i])
    return b, co, neutral


def inputs_of(b, ws, neutral, co):
    """(n, H, W, 8) float32 network inputs from each instance's geometry and initial field."""
    n = len(ws)
    H, Wd = ws[0].ny, ws[0].nx
    x = np.zeros((n, H, Wd, 8), dtype=np.float32)
    jj, ii = np.mgrid[0:H, 0:Wd].astype(np.float64)
    for i, w in enumerate(ws):
        ctx = lbm.lbm_batch_instance(b.b, i)
        flags, muw, _ = lbm.lbm_read_geometry(ctx, w.nx, w.ny)
        f = flags[2:-2]
        x[i, :, :, 0] = f != 0
        layer = (f == 1) | (f == 2)
        x[i, :, :, 1] = np.where(layer, (muw[2:-2] - neutral) / MU_SCALE, 0.0)
        rho = lbm.lbm_read_fields(ctx, lbm.LBM_FIELD_RHO, w.nx, w.ny)[0]
        phi0 = np.clip((rho - co["rho_g"]) / (co["rho_l"] - co["rho_g"]), 0, 1) * (f == 0)
        x[i, :, :, 2] = phi0.sum() / (H * Wd)
        x[i, :, :, 3] = jj / H
        cx, cy, R = w.circle
        x[i, :, :, 4] = (ii - cx) / Wd
        dist = np.minimum(np.hypot(ii - cx, jj - cy) - (R + 0.5), jj + 0.5)
        x[i, :, :, 5] = np.clip(dist / 64.0, -1.0, 1.0)
        x[i, :, :, 6] = w.mu_rel_circle / MU_SCALE
    return x


def targets_of(b, ws, co):
    n = len(ws)
    H, Wd = ws[0].ny, ws[0].nx
    t = np.zeros((n, H, Wd), dtype=np.float32)
    mask = np.zeros((n, H, Wd), dtype=np.uint8)
    for i, w in enumerate(ws):
        ctx = lbm.lbm_batch_instance(b.b, i)
        flags, _, _ = lbm.lbm_read_geometry(ctx, w.nx, w.ny)
        rho = lbm.lbm_read_fields(ctx, lbm.LBM_FIELD_RHO, w.nx, w.ny)[0]
        fl = flags[2:-2] == 0
        t[i] = np.clip((rho - co["rho_g"]) / (co["rho_l"] - co["rho_g"]), 0, 1) * fl
        mask[i] = fl
    return t, mask


def generate(ws, steps=20000, chunk=512):
    """Equilibrated training data: inputs, targets, masks (numpy) for the cases."""
    xs, ts, ms = [], [], []
    for k in range(0, len(ws), chunk):
        part = ws[k:k + chunk]
        b, co, neutral = make_batch(part)
        xs.append(inputs_of(b, part, neutral, co))
        b.run(steps, check_every=500, tol=0.0, angle_tol=0.02)
        t, m = targets_of(b, part, co)
        ts.append(t)
        ms.append(m)
        b.close()
    return np.concatenate(xs), np.concatenate(ts), np.concatenate(ms)


def lr_at(step, total, lr, warmup=200, schedule="warmcos"):
    """Learning rate of step `step` of `total`: linear warm-up over `warmup` steps, then a cosine
    decay to zero ("warmcos"), or constant ("const")."""
    if schedule == "const":
        return lr
    w = min(1.0, (step + 1) / max(1, warmup))
    return lr * w * 0.5 * (1.0 + np.cos(np.pi * step / max(1, total)))


def train(sur, x, t, m, epochs=20, batch=8, lr=1e-3, seed=0, log=None, schedule="warmcos",
          warmup=200):
    """Adam on the masked MSE with the `lr_at` schedule; data held on the device (torch tensors
    as plain buffers)."""
    import torch
    n = x.shape[0]
    # start the head at the mean target (logit of the mean liquid fraction)
    w = sur.weights()
    pm = float(np.clip((t * m).sum() / max(m.sum(), 1), 1e-3, 1 - 1e-3))
    w[-1] = np.log(pm / (1 - pm))
    sur.set_weights(w)
    xd = torch.tensor(x).to(torch.bfloat16).cuda()
    td = torch.tensor(t).cuda()
    md = torch.tensor(m).cuda()
    rng = np.random.default_rng(seed)
    losses = []
    t0 = time.perf_counter()
    total = epochs * (n // batch)
    step = 0
    for ep in range(epochs):
        perm = rng.permutation(n)
        el = []
        for k in range(0, n - batch + 1, batch):
            idx = torch.tensor(perm[k:k + batch], device="cuda")
            xb, tb, mb = xd[idx].contiguous(), td[idx].contiguous(), md[idx].contiguous()
            el.append(sur.train_step(xb.data_ptr(), tb.data_ptr(), mb.data_ptr(), batch,
                                     lr_at(step, total, lr, warmup, schedule)))
            step += 1
        losses.append(float(np.mean(el)))
        if log:
            log(f"epoch {ep} loss {losses[-1]:.5f} ({time.perf_counter() - t0:.1f}s)")
    return losses, time.perf_counter() - t0


def predict(sur, x, batch=8):
    """phi for inputs x (n, H, W, 8) float32, `batch` cases per forward call; each chunk goes to
    the device as FP32 and is converted to BF16 there."""
    import torch
    n = x.shape[0]
    out = torch.zeros((n, x.shape[1], x.shape[2]), dtype=torch.float32, device="cuda")
    for k in range(0, n, batch):
        bb = min(batch, n - k)
        xb = torch.from_numpy(np.ascontiguousarray(x[k:k + bb])).cuda().to(torch.bfloat16)
        sur.forward(xb.contiguous().data_ptr(), bb, out[k:k + bb].data_ptr())
    return out.cpu().numpy()


def match_mass(phi, mask, target_mass, rho_g, rho_l, rtol=1e-12):
    """Shift phi by one constant (then clip to [0, 1]) so that the fluid nodes hold the mass of
    the cold start: the warm and cold runs then relax the same amount of liquid. The liquid
    content F(c) = sum clip(phi + c, 0, 1) is piecewise linear and non-decreasing in the shift c
    with slope = the number of nodes strictly inside (0, 1); Newton steps on it, kept inside a
    shrinking bracket (bisection where a step leaves it), find the shift in a few evaluations."""
    p = phi[mask].astype(np.float64)
    goal = (target_mass - rho_g * p.size) / (rho_l - rho_g)
    lo, hi = -1.0, 1.0
    c = 0.0
    for _ in range(100):
        v = p + c
        F = np.clip(v, 0.0, 1.0).sum()
        if abs(F - goal) <= rtol * max(1.0, abs(goal)):
            break
        if F < goal:
            lo = c
        else:
            hi = c
        slope = np.count_nonzero((v > 0.0) & (v < 1.0))
        nxt = c + (goal - F) / slope if slope else 0.5 * (lo + hi)
        c = nxt if lo < nxt < hi else 0.5 * (lo + hi)
    return np.clip(phi.astype(np.float64) + c, 0, 1)


def angle_histories(b, n, steps, every):
    """Angles (n, n_meas, 2) measured every `every` steps (NaN where a side had no contact) and
    the wall-clock seconds since the start at each measurement (the batch run and the
    measurement are synchronous)."""
    hist, times = [], []
    t0 = time.perf_counter()
    for _ in range(steps // every):
        b.run(every, check_every=every, tol=0.0)
        ang = b.measure()
        hist.append([[a.theta if a.status == 0 else np.nan for a in pair] for pair in ang])
        times.append(time.perf_counter() - t0)
    return np.transpose(np.array(hist), (1, 0, 2)), np.array(times)


def plain_histories(ws, steps, every, rho0=None):
    """The plain single-instance solver: one lattice per case, run one after another, angles
    every `every` steps. Returns the angles (n, n_meas, 2) and per case the wall-clock seconds
    since that case's first step at each measurement (n, n_meas)."""
    m = ws[0].model
    co = lbm.lbm_coexistence(m["eos"], m["Tr"])
    neutral = m["k2"] * co["mu_sat"]
    hist = np.full((len(ws), steps // every, 2), np.nan)
    times = np.zeros((len(ws), steps // every))
    for i, w in enumerate(ws):
        lat = lbm.Lattice(w.nx, w.ny, **_model_kw(m))
        lat.set_geometry(**_geometry(w, neutral), rho0=None if rho0 is None else rho0[i])
        lat.synchronize()
        t0 = time.perf_counter()
        for k in range(steps // every):
            lat.step(every)
            st, ang = lbm.lbm_measure_contact_angle(lat.ctx)
            hist[i, k] = [a.theta_deg if a.status == 0 else np.nan for a in ang]
            times[i, k] = time.perf_counter() - t0
        lat.close()
    return hist, times


def reach_index(hist, theta_final, tol=0.5):
    """Index of the first measurement after which every later measurement of both sides lies
    within tol of theta_final (None if never): the time-to-equilibrated-angle criterion."""
    ok = np.all(np.abs(hist - theta_final[None, :]) <= tol, axis=1)
    for k in range(len(ok)):
        if ok[k:].all():
            return k
    return None


def time_to_angle(hist, theta_final, every, tol=0.5):
    """First measured step after which every later measurement of both sides lies within tol of
    theta_final (None if never)."""
    k = reach_index(hist, theta_final, tol)
    return None if k is None else (k + 1) * every


def evaluate(sur, ws, steps=20000, every=250, log=None, plain=True):
    """Time to the equilibrated angle for held-out cases, three ways, all judged against the final
    angle theta_f of the plain cold run (Eq. 16 cap start) of the same case, criterion
    `reach_index` with tol 0.5 degrees:
      plain   one lattice per case, cases one after another (skipped with plain=False; the
              batched cold run then stands in for the reference, which it equals bit for bit);
      cold    all cases in one batch from the Eq. 16 start;
      warm    the network's prediction (shifted to the cold start's liquid mass) as the initial
              density, all cases in one batch; its clock includes the prediction.
    Returns one dict per case: the reference angle, steps and seconds to reach it per variant
    (None if not reached), the warm run's own final angle, and a class: 'ok', 'no_contact' (a
    side without contact at the end of the reference run: the drop lifted off or wet past the
    circle) or 'unsettled' (the reference run's last quarter strays more than 0.5 degrees from
    its final angle, so theta_f is no equilibrium)."""
    n_meas = steps // every
    hp = tp = None
    if plain:
        hp, tp = plain_histories(ws, steps, every)
    bc, co, neutral = make_batch(ws)
    x = inputs_of(bc, ws, neutral, co)
    masses, fluid = [], []
    for i, w in enumerate(ws):
        ctx = lbm.lbm_batch_instance(bc.b, i)
        masses.append(lbm.lbm_mass(ctx)[1]["mass"])
        fluid.append(lbm.lbm_read_geometry(ctx, w.nx, w.ny)[0][2:-2] == 0)
    hc, tc = angle_histories(bc, len(ws), steps, every)
    bc.close()
    # the warm batch's lattices exist before the clock starts, as the cold batch's did; the
    # clock covers the prediction, the mass matching and setting the predicted initial states
    bw, _, _ = make_batch(ws)
    t0 = time.perf_counter()
    phi = predict(sur, x).astype(np.float64)
    phi = np.stack([match_mass(phi[i], fluid[i], masses[i], co["rho_g"], co["rho_l"])
                    for i in range(len(ws))])
    rho0 = co["rho_g"] + phi * (co["rho_l"] - co["rho_g"])
    for i, w in enumerate(ws):
        bw.set_geometry(i, **_geometry(w, neutral), rho0=rho0[i])
    t_pred = time.perf_counter() - t0
    hw, tw = angle_histories(bw, len(ws), steps, every)
    bw.close()
    ref = hp if plain else hc
    rows = []
    for i in range(len(ws)):
        final = ref[i, -1]
        row = {"theta_f": final.tolist(), "plain_identical": None if hp is None else
               bool(np.array_equal(hp[i], hc[i], equal_nan=True))}
        if np.isnan(final).any():
            row["class"] = "no_contact"
        elif reach_index(ref[i], final) is None or reach_index(ref[i], final) > (3 * n_meas) // 4:
            row["class"] = "unsettled"
        else:
            row["class"] = "ok"
        for name, h, tt in (("plain", hp, tp), ("cold", hc, None), ("warm", hw, None)):
            if h is None or row["class"] == "no_contact":
                row[name] = None
                continue
            k = reach_index(h[i], final)
            if k is None:
                row[name] = None
            elif name == "plain":
                row[name] = ((k + 1) * every, float(tt[i, k]))
            elif name == "cold":
                row[name] = ((k + 1) * every, float(tc[k]))
            else:
                row[name] = ((k + 1) * every, float(t_pred + tw[k]))
        own = hw[i, -1]
        row["warm_final_gap"] = None if np.isnan(own).any() or np.isnan(final).any() else \
            float(np.abs(own - final).max())
        row["warm_self"] = None if np.isnan(own).any() else time_to_angle(hw[i], own, every)
        row["cold_self"] = None if np.isnan(final).any() else time_to_angle(hc[i], hc[i, -1], every)
        rows.append(row)
    extra = {"prediction_seconds": t_pred, "cold_batch_seconds": float(tc[-1]),
             "warm_batch_seconds": float(tw[-1]),
             "plain_seconds": None if tp is None else float(tp[:, -1].sum())}
    return rows, extra


def merge_extra(parts):
    """Per-rank `evaluate` timings combined: batches run side by side (the slowest rank's time),
    the prediction likewise, the plain runs' total is a sum over all cases."""
    parts = [p for p in parts if p]
    if not parts:
        return {}
    out = {k: max(p[k] for p in parts) for k in ("prediction_seconds", "cold_batch_seconds",
                                                 "warm_batch_seconds")}
    plain = [p["plain_seconds"] for p in parts]
    out["plain_seconds"] = None if any(v is None for v in plain) else float(sum(plain))
    return out


def summarise(rows, extra):
    """Aggregate the per-case rows of `evaluate` (possibly gathered from several ranks):
    per variant the cases that reach the reference angle, their median steps and seconds, and
    the time until every reaching case has reached it (the plain variant runs the cases one after
    another, so its total is the sum over cases)."""
    classes = {}
    for r in rows:
        classes[r["class"]] = classes.get(r["class"], 0) + 1
    ok = [r for r in rows if r["class"] == "ok"]
    out = {"cases": len(rows), "classes": classes, "judged": len(ok)}
    ran_plain = any(r["plain_identical"] is not None for r in rows)
    for name in ("plain", "cold", "warm"):
        if name == "plain" and not ran_plain:
            out[name] = None
            continue
        got = [r[name] for r in ok if r[name] is not None]
        steps = [g[0] for g in got]
        secs = [g[1] for g in got]
        out[name] = {"reached": len(got), "reached_fraction": len(got) / len(ok) if ok else None,
                     "median_steps": float(np.median(steps)) if got else None,
                     "median_seconds": float(np.median(secs)) if got else None,
                     "all_reached_seconds": (float(np.sum(secs)) if name == "plain"
                                             else float(np.max(secs))) if got else None}
    both = [(r["cold"][0], r["warm"][0]) for r in ok if r["cold"] and r["warm"]]
    out["warm_faster_fraction"] = float(np.mean([w < c for c, w in both])) if both else None
    gaps = [r["warm_final_gap"] for r in rows if r["warm_final_gap"] is not None]
    out["warm_final_gap_median_deg"] = float(np.median(gaps)) if gaps else None
    out["warm_settles_elsewhere"] = sum(1 for r in ok if r["warm"] is None and
                                        r["warm_final_gap"] is not None and
                                        r["warm_final_gap"] > 0.5)
    own = [(r["cold_self"], r["warm_self"]) for r in rows
           if r["cold_self"] is not None and r["warm_self"] is not None]
    out["own_final_angle"] = {"pairs": len(own),
                              "cold_median_steps": float(np.median([a for a, _ in own])) if own else None,
                              "warm_median_steps": float(np.median([b for _, b in own])) if own else None}
    ident = [r["plain_identical"] for r in rows if r["plain_identical"] is not None]
    out["plain_equals_batched_cold"] = all(ident) if ident else None
    out.update(extra)
    return out
