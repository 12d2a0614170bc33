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
    import torch
    n = x.shape[0]
    out = np.zeros((n, x.shape[1], x.shape[2]), dtype=np.float32)
    xd = torch.tensor(x).to(torch.bfloat16).cuda()
    phi = torch.zeros((batch, x.shape[1], x.shape[2]), dtype=torch.float32, device="cuda")
    for k in range(0, n, batch):
        bb = min(batch, n - k)
        xb = xd[k:k + bb].contiguous()
        sur.forward(xb.data_ptr(), bb, phi.data_ptr())
        out[k:k + bb] = phi[:bb].cpu().numpy()
    return out


def match_mass(phi, mask, target_mass, rho_g, rho_l):
    """Shift phi by one constant (then clip to [0, 1]) so that the fluid nodes hold the mass of
    the cold start: the warm and cold runs then relax the same amount of liquid. Bisection on
    the shift."""
    def mass(c):
        return (rho_g + np.clip(phi + c, 0, 1) * (rho_l - rho_g))[mask].sum()
    lo, hi = -1.0, 1.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if mass(mid) < target_mass:
            lo = mid
        else:
            hi = mid
    return np.clip(phi + 0.5 * (lo + hi), 0, 1)


def angle_histories(b, n, steps, every):
    """Angles (n, n_meas, 2) measured every `every` steps (NaN where a side had no contact)."""
    hist = []
    for _ in range(steps // every):
        b.run(every, check_every=every, tol=0.0)
        ang = b.measure()
        hist.append([[a.theta if a.status == 0 else np.nan for a in pair] for pair in ang])
    return np.transpose(np.array(hist), (1, 0, 2))


def time_to_angle(hist, theta_final, every, tol=0.5):
    """First measured step after which every later measurement of both sides lies within tol of
    theta_final (None if never)."""
    ok = np.all(np.abs(hist - theta_final[None, :]) <= tol, axis=1)
    for k in range(len(ok)):
        if ok[k:].all():
            return (k + 1) * every
    return None


def evaluate(sur, ws, steps=20000, every=250, log=None):
    """Cold start (Eq. 16 cap) vs warm start (prediction) for the held-out cases: steps to the
    +-0.5 degree equilibrated angle of the cold run's final angle."""
    bc, co, neutral = make_batch(ws)
    x = inputs_of(bc, ws, neutral, co)
    masses, fluid = [], []
    for i, w in enumerate(ws):
        ctx = lbm.lbm_batch_instance(bc.b, i)
        masses.append(lbm.lbm_mass(ctx)[1]["mass"])
        fluid.append(lbm.lbm_read_geometry(ctx, w.nx, w.ny)[0][2:-2] == 0)
    hc = angle_histories(bc, len(ws), steps, every)
    bc.close()
    phi = predict(sur, x).astype(np.float64)
    phi = np.stack([match_mass(phi[i], fluid[i], masses[i], co["rho_g"], co["rho_l"])
                    for i in range(len(ws))])
    rho0 = co["rho_g"] + phi * (co["rho_l"] - co["rho_g"])
    bw, _, _ = make_batch(ws, rho0=rho0)
    hw = angle_histories(bw, len(ws), steps, every)
    bw.close()
    rows = []
    for i in range(len(ws)):
        final = hc[i, -1]
        if np.isnan(final).any():
            rows.append((None, None, None, None, None))
            continue
        own = hw[i, -1]
        rows.append((time_to_angle(hc[i], final, every), time_to_angle(hw[i], final, every),
                     time_to_angle(hc[i], final, every),
                     None if np.isnan(own).any() else time_to_angle(hw[i], own, every),
                     None if np.isnan(own).any() else float(np.abs(own - final).max())))
    return rows, hc, hw
