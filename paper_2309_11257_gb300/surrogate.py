"""Column drag surrogate: training data from the ray tracer, the training loop and its evaluation.

The surrogate (gwam.Surrogate) maps the features of one column -- u, v, N^2, ln rho on the nz
levels and 8 source parameters -- to the column's drag du/dt, dv/dt on the nz levels.  Its
training data come from the FP64 ray tracer itself: an ensemble of spheres with different jets
and perturbations, the background source (Sec. 3c) with per-run parameters, and convective
spectral launches with per-column counts, stepped with the tracer; the targets are the drag
averaged over the last `avg` steps.  Every array stays on the GPU; the features and targets are
assembled by the library's kernels (gwam_column_features / gwam_column_targets).

Source features (per column): F_bg (f_w of the background source), z_launch, lambda_h, c_min,
c_max, F_conv (the column's convective flux), ln(1 + n_conv) (its convective ray count) and the
Coriolis parameter f = 2 Omega sin(phi) of the column's row.
"""
from __future__ import annotations

import math

import numpy as np

from . import gwam, synth

N_SRC = 8


def _source_table(grid, src, specs, members):
    """[members * ncol][8] float32 source features (host)."""
    nx, ny = grid["nx"], grid["ny"]
    ncol = nx * ny
    _, phi, _ = synth.node_coords(grid)
    f = (2.0 * grid["omega"] * np.sin(phi)).astype(np.float64)
    out = np.zeros((members, ncol, N_SRC), dtype=np.float32)
    out[:, :, 0] = src["f_w"]
    out[:, :, 1] = src["z_launch"]
    out[:, :, 2] = src["lambda_h"]
    out[:, :, 3] = src["c_min"]
    out[:, :, 4] = src["c_max"]
    out[:, :, 7] = np.repeat(f, nx)[None, :]
    for m, sp in enumerate(specs):
        if sp is None or len(sp) == 0:
            continue
        col = sp["j"].astype(np.int64) * nx + sp["i"]
        flux = np.bincount(col, weights=sp["flux"], minlength=ncol)
        cnt = np.bincount(col, minlength=ncol)
        out[m, :, 5] = flux
        out[m, :, 6] = np.log1p(cnt)
    return out.reshape(members * ncol, N_SRC)


def generate(members=16, nx=64, ny=32, nz=90, steps=120, avg=40, launch_every=5, tag=0, convection=True,
             src_overrides=None, max_rays=None, dt=180.0, conv_fraction=0.3, jet_member0=None):
    """Run the FP64 tracer on `members` backgrounds and return (X, Y, info): features
    [members * nx * ny][4 nz + 8] and drag targets [members * nx * ny][2 nz] as float32 CUDA
    tensors, member-major then column order (j, i).  The sources launch every `launch_every` steps
    (a quasi-continuous source), so the averaged drag approaches the columns' steady response."""
    import torch
    g = synth.rng(5000 + tag)
    grid = synth.sphere_grid(nx=nx, ny=ny, nz=nz, dz=1000.0)
    amps = g.uniform(30.0, 80.0, members)
    lats = g.uniform(30.0, 60.0, members)
    src = synth.background_source(
        z_launch=float(g.uniform(3e3, 7e3)), lambda_h=float(math.exp(g.uniform(math.log(60e3), math.log(200e3)))),
        c_min=float(g.uniform(3.0, 8.0)), c_max=float(g.uniform(35.0, 60.0)),
        f_w=float(g.uniform(4e-3, 12e-3)), f_s=2.4e-3)
    if src_overrides:
        src.update(src_overrides)
    ncol = nx * ny
    params = dict(synth.DEFAULT_PARAMS)
    if max_rays is None:
        max_rays = int(members * ncol * 32 * (steps // launch_every + 2) * 1.5 + (members * ncol * 60 if convection else 0))
    T = gwam.Tracer(grid, params, max_rays=max_rays, members=members)
    bgs = []
    if jet_member0 is not None:
        # member 0 on a given unperturbed jet background (e.g. 60 m/s at 45 deg)
        amps[0], lats[0] = jet_member0
    for m in range(members):
        bg = synth.jet_background(grid, amp=float(amps[m]), lat_deg=float(lats[m]))
        if not (m == 0 and jet_member0 is not None):
            bg = synth.perturbed(bg, tag=6000 + 97 * tag + m)
        bgs.append([torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in bg])
        T.set_member_background(m, *bgs[-1])
    specs = [None] * members
    if convection:
        allsp = []
        for m in range(members):
            sp = synth.convective_specs(grid, tag=7000 + 31 * tag + m, median=16.0, sigma=1.0, cap=512,
                                        z_launch=10e3, col_fraction=conv_fraction)
            sp["member"] = m
            specs[m] = sp
            allsp.append(sp)
        allsp = np.concatenate(allsp)
    du = torch.zeros((members, nz, ny, nx), dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    du_sum = torch.zeros_like(du)
    dv_sum = torch.zeros_like(du)
    step_ms = 0.0
    for s in range(steps):
        if s % launch_every == 0:
            T.launch_sources(src)
            if convection:
                T.launch_spectral(allsp)
        if s >= steps - avg:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            T.step(dt, du, dv)
            e1.record()
            du_sum += du
            dv_sum += dv
            e1.synchronize()
            step_ms += e0.elapsed_time(e1)
        else:
            T.step(dt, du, dv)
    nf = 4 * nz + N_SRC
    X = torch.empty((members * ncol, nf), dtype=torch.float32, device="cuda")
    Y = torch.empty((members * ncol, 2 * nz), dtype=torch.float32, device="cuda")
    srcf = torch.from_numpy(_source_table(grid, src, specs, members)).cuda()
    for m in range(members):
        sl = slice(m * ncol, (m + 1) * ncol)
        gwam.column_features(*bgs[m], srcf[sl].contiguous(), X[sl])
        gwam.column_targets(du_sum[m], dv_sum[m], 1.0 / avg, Y[sl])
    torch.cuda.synchronize()
    info = dict(grid=grid, members=members, ncol=ncol, src=src, amps=amps, lats=lats,
                rays=T.num_rays(), stats=T.stats(), tracer_ms_per_step=step_ms / max(1, min(avg, steps)))
    T.close()
    return X, Y, info


def train(S, X, Y, steps=2000, batch=4096, lr=1e-3, lr_end=1e-5, seed=1, log_every=0):
    """Adam with a cosine learning-rate decay from lr to lr_end; returns the loss history."""
    hist = []
    for it in range(steps):
        a = lr_end + 0.5 * (lr - lr_end) * (1.0 + math.cos(math.pi * it / max(1, steps - 1)))
        S.train_step(X, Y, batch, seed=seed * 1_000_003 + it, lr=a)
        if log_every and (it % log_every == 0 or it == steps - 1):
            hist.append((it, S.loss()))
    return hist


def generate_1m(nx=256, ny=128, nz=90, members_per_run=8, runs=4, steps=100, avg=30, launch_every=10, tag=10):
    """The surrogate's full data set: 1 048 576 columns (4 runs x 8 members of the 256 x 128 x 90
    sphere) from the FP64 tracer on the sphere workload's background (60 m/s jets at 45 deg: member 0
    of the first run, unperturbed) and the batched ensemble's (jets U[30, 80] m/s at U[30, 60] deg,
    seeded perturbations, convective launches in every column with lognormal counts, median 16, capped
    at 512, on top of the background source); sources relaunched every `launch_every` steps, targets
    averaged over the last `avg` steps.  Returns X, Y (member-major) and the per-run infos."""
    import torch
    Xs, Ys, infos = [], [], []
    for r in range(runs):
        X, Y, info = generate(members=members_per_run, nx=nx, ny=ny, nz=nz, steps=steps, avg=avg,
                              launch_every=launch_every, tag=tag + r, conv_fraction=1.0,
                              jet_member0=(60.0, 45.0) if r == 0 else None)
        Xs.append(X)
        Ys.append(Y)
        infos.append(info)
    X = torch.cat(Xs)
    Y = torch.cat(Ys)
    del Xs, Ys
    return X, Y, infos


def member_split(runs, members_per_run, ncol, test_member=-1, val_members=((0, -2), (2, -2))):
    """Boolean row masks (train, validation, test) of a member-major data set: the test set is
    member `test_member` of every run (unseen jets, perturbations and sources), the validation set
    the listed (run, member) pairs, the rest trains."""
    import torch
    n = runs * members_per_run * ncol
    test = torch.zeros(n, dtype=torch.bool, device="cuda")
    val = torch.zeros_like(test)
    for r in range(runs):
        m = test_member % members_per_run
        test[(r * members_per_run + m) * ncol:(r * members_per_run + m + 1) * ncol] = True
    for r, m in val_members:
        m = m % members_per_run
        val[(r * members_per_run + m) * ncol:(r * members_per_run + m + 1) * ncol] = True
    return ~(test | val), val, test


# training of the full data set: batches of 4096, Adam at 1e-3 with a cosine decay over at most 1500
# steps, validated every 50 (the validation error is lowest after about one epoch; the network then
# fits the columns' unpredictable convective part)
TRAIN_1M = dict(max_steps=1500, every=50, batch=4096, lr=1e-3, patience=6)


def train_early_stopping(S, Xtr, Ytr, Xva, Yva, nlev, max_steps=4000, every=250, batch=4096, lr=1e-3, lr_end=1e-5,
                         seed=1, patience=4):
    """Adam with a cosine learning-rate decay over max_steps; every `every` steps the drag relative
    L2 on the validation columns is measured and the weights with the lowest one are kept (early
    stopping after `patience` checks without improvement).  Returns (best validation error, step of
    the kept weights, history [(step, training loss, validation error)])."""
    best, best_params, best_step, bad, hist = float("inf"), None, 0, 0, []
    for it in range(max_steps):
        a = lr_end + 0.5 * (lr - lr_end) * (1.0 + math.cos(math.pi * it / max(1, max_steps - 1)))
        S.train_step(Xtr, Ytr, batch, seed=seed * 1_000_003 + it, lr=a)
        if (it + 1) % every == 0 or it == max_steps - 1:
            e = drag_error(S, Xva, Yva, nlev)["rel_l2"]
            hist.append((it + 1, S.loss(), e))
            if e < best:
                best, best_params, best_step, bad = e, S.params(), it + 1, 0
            else:
                bad += 1
                if bad >= patience:
                    break
    if best_params is not None:
        S.set_params(best_params)
    return best, best_step, hist


def drag_error(S, X, Y, nlev):
    """Surrogate drag on the columns X against the tracer's Y: relative L2 over all in-envelope
    columns and outputs, the same for the training-mean baseline, and the fallback count."""
    import torch
    ncol = X.shape[0]
    du = torch.zeros((nlev, ncol), dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    mask = torch.zeros(ncol, dtype=torch.int32, device="cuda")
    nfb = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.infer(X, du, dv, mask, nfb)
    S.status()
    inside = mask == 0
    pred = torch.cat([du.t(), dv.t()], dim=1)[inside]
    ref = Y.double()[inside]
    err = float(torch.linalg.norm(pred - ref) / torch.linalg.norm(ref))
    return dict(rel_l2=err, n_inside=int(inside.sum()), n_fallback=int(nfb.item()))
