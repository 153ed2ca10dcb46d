"""Training and evaluation of the learned troubled-cell indicator.

The solver itself makes the training data: seeded MHD blasts are advanced with
the plain TVB-characteristic limiter, and at every step the features of all
cells (dg_mhd_mlp_features) are recorded with the plain detector's decision
(the troubled flags of dg_mhd_limit) as the label. The network is trained on
the GPU by the library's own forward/backward/Adam kernels (dg_mhd_mlp_train).
Evaluation runs the same problem with the plain detector and with the network
gating the TVB procedure, and reports missed cells, false positives, positivity
activations, the L1 difference of the final states and the limiter time.

Everything numerical runs in the CUDA library; this module only orchestrates.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import workloads as W
from .binding import (DG_LIMIT_MLP, DG_LIMIT_TVB, DG_PREC_FP32MIX, DG_PREC_FP64, KIND_LIMIT, KIND_MLP,
                      KIND_POSITIVITY, Solver, mlp_loss_grad, mlp_train)

THRESHOLDS = (0.02, 0.05, 0.1, 0.2, 0.3, 0.5)

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS_DIR = os.path.join(HERE, "weights")


def n_params(nin):
    return 64 * nin + 64 + 64 * 64 + 64 + 64 + 1


def init_theta(nin, seed=0):
    import torch
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, math.sqrt(2.0 / nin), (64, nin))
    W2 = rng.normal(0, math.sqrt(2.0 / 64), (64, 64))
    w3 = rng.normal(0, math.sqrt(1.0 / 64), 64)
    th = np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), w3, [-2.0]])
    return torch.as_tensor(th, dtype=torch.float32, device="cuda")


def blast_state(sol, params, nvar, device="cuda"):
    """Projected blast start for a Solver on an n^3 box."""
    n = round(sol.ncell ** (1.0 / 3.0))
    fn = lambda x: W.blast_3d(x, nvar=nvar, **params)
    nodal = W.gauss_nodal(fn, n, sol.degree + 1, 3, sol.stride, device)
    w, wm = sol.alloc_state(device)
    sol.project(nodal, sol.degree + 1, w, wm)
    return w, wm


def turbulence_state(sol, seed, mach, nvar, device="cuda"):
    """Projected decaying-turbulence start (random-phase solenoidal velocity,
    E(k) ~ k^-2 on 2 <= |k| <= 8, rms Mach `mach`) for a Solver on an n^3 box."""
    n = round(sol.ncell ** (1.0 / 3.0))
    nodal = W.turbulence_nodal(n, sol.degree + 1, sol.stride, device, seed=seed, nvar=nvar, mach=mach)
    w, wm = sol.alloc_state(device)
    sol.project(nodal, sol.degree + 1, w, wm)
    del nodal
    return w, wm


def _record(sol, w, wm, keep, gen, device):
    """Features of the current state and the plain detector's decision on a
    copy of it; `keep` < 1 keeps a seeded random subset of the cells."""
    import torch
    nin = sol.n_features()
    ldx = (nin + 15) // 16 * 16
    X = torch.zeros((sol.ncell, ldx), dtype=torch.float32, device=device)
    flags = torch.zeros(sol.stride, dtype=torch.uint8, device=device)
    sol.mlp_features(w, wm, X, ldx)
    wc = w.clone()
    wmc = wm.clone() if wm is not None else None
    sol.limit(wc, wmc, flags)
    del wc, wmc
    y = flags[: sol.ncell]
    if keep < 1.0:
        # every troubled cell, and a random share `keep` of the others
        sel = (y > 0) | (torch.rand(sol.ncell, generator=gen, device=device) < keep)
        idx = torch.nonzero(sel).squeeze(1)
        return X[idx].contiguous(), y[idx].clone()
    return X, y.clone()


def generate(divb="powell", degree=2, n=64, seeds=(1, 2, 3, 4), steps=6, precision=DG_PREC_FP32MIX,
             Mtilde=5.0, device="cuda", turbulence=(), turb_steps=4, turb_every=1):
    """(X [samples][ldx] float32, y [samples] uint8, nin, src [samples] uint8)
    on the device. Blasts (src 0): `seeds` at n^3, `steps` states each.
    Turbulence (src 1): for each (n_t, mach, seed, keep) in `turbulence`,
    `turb_steps` states `turb_every` steps apart, a share `keep` of the
    untroubled cells kept."""
    import torch
    nvar = 9 if divb == "glm" else 8
    gen = torch.Generator(device=device)
    gen.manual_seed(12345)
    Xs, ys, srcs = [], [], []
    nin = None
    for sd in seeds:
        sol = Solver(3, (n, n, n), degree, divb, precision=precision, limiter=DG_LIMIT_TVB, positivity=1,
                     Mtilde=Mtilde)
        nin = sol.n_features()
        w, wm = blast_state(sol, W.blast_params(sd), nvar, device)
        sol.dt(w, wm)  # GLM: the labels' characteristic fields need c_h (a step sets it the same way)
        for _ in range(steps):
            X, y = _record(sol, w, wm, 1.0, gen, device)
            Xs.append(X)
            ys.append(y)
            srcs.append(torch.zeros_like(y))
            sol.step(w, wm)
        del sol, w, wm
    for (nt, mach, sd, keep) in turbulence:
        sol = Solver(3, (nt, nt, nt), degree, divb, precision=precision, limiter=DG_LIMIT_TVB, positivity=1,
                     Mtilde=Mtilde)
        nin = sol.n_features()
        w, wm = turbulence_state(sol, sd, mach, nvar, device)
        sol.dt(w, wm)
        for _ in range(turb_steps):
            X, y = _record(sol, w, wm, keep, gen, device)
            Xs.append(X)
            ys.append(y)
            srcs.append(torch.ones_like(y))
            for _ in range(turb_every):
                sol.step(w, wm)
        del sol, w, wm
        torch.cuda.empty_cache()
    return torch.cat(Xs), torch.cat(ys), nin, torch.cat(srcs)


def balance(X, y, neg_per_pos=20, seed=0, src=None):
    """All troubled samples plus a seeded random subset of the others
    (troubled cells are rare: ~0.2% of blast cells). With `src` (several
    sources), every source contributes at most as many troubled samples as
    source 0 (the blasts) has, and the untroubled samples are drawn in equal
    numbers from every source: no source's kind of discontinuity dominates."""
    import torch
    g = torch.Generator(device=X.device)
    g.manual_seed(seed)

    def pick(mask, k):
        idx = torch.nonzero(mask).squeeze(1)
        return idx[torch.randperm(len(idx), generator=g, device=X.device)[:min(k, len(idx))]]

    if src is None or len(torch.unique(src)) == 1:
        pos = torch.nonzero(y).squeeze(1)
        parts = [pos, pick(y == 0, max(1, neg_per_pos * len(pos)))]
    else:
        sources = torch.unique(src).tolist()
        npos = [int(((y > 0) & (src == s)).sum()) for s in sources]
        cap = npos[0] if npos[0] > 0 else max(npos)
        parts = [pick((y > 0) & (src == s), cap) for s in sources]
        k = max(1, neg_per_pos * cap) // len(sources)
        parts += [pick((y == 0) & (src == s), k) for s in sources]
    idx = torch.cat(parts)
    idx = idx[torch.randperm(len(idx), generator=g, device=X.device)]
    return X[idx].contiguous(), y[idx].contiguous()


def train(X, y, nin, epochs=8, batch=4096, lr=1e-3, pos_weight=4.0, seed=0, neg_per_pos=20, src=None):
    Xb, yb = balance(X, y, neg_per_pos, seed, src)
    theta = init_theta(nin, seed)
    l0, _ = mlp_loss_grad(Xb[:200000], yb[:200000], theta, nin, pos_weight)
    batch = min(batch, len(yb))
    last = mlp_train(Xb, yb, theta, nin, epochs, batch, lr, pos_weight, seed)
    return theta, {"loss_initial": l0, "loss_last_epoch": last, "train_samples": int(len(yb)),
                   "train_positives": int(yb.sum())}


def detection_rates(sol, w, wm, theta):
    """Per threshold: (missed, false positive, flagged, troubled) on one state:
    network flags versus the plain TVB decision on a copy of the state."""
    import torch
    sol.mlp_set_weights(theta, 0.5)
    prob = torch.zeros(sol.stride, dtype=torch.float32, device=w.device)
    sol.mlp_infer(w, wm, None, prob)
    f_tv = torch.zeros(sol.stride, dtype=torch.uint8, device=w.device)
    wc = w.clone()
    wmc = wm.clone() if wm is not None else None
    sol.limit(wc, wmc, f_tv)
    b = f_tv[: sol.ncell].bool()
    out = {}
    for th in THRESHOLDS:
        a = prob[: sol.ncell] > th
        out[th] = (int((b & ~a).sum()), int((a & ~b).sum()), int(a.sum()), int(b.sum()))
    return out


def evaluate(theta, nin, divb="powell", degree=2, n=128, steps=10, threshold=0.1, precision=DG_PREC_FP32MIX,
             Mtilde=5.0, device="cuda"):
    """Config-4 style evaluation on the p = 100 / 0.1 blast with
    B = (10/sqrt(4 pi), 0, 0): plain TVB detection against network gating."""
    import torch
    nvar = 9 if divb == "glm" else 8
    params = dict(center=(0.5, 0.5, 0.5), r0=0.1, p_in=100.0, p_out=0.1,
                  B0=(10.0 / math.sqrt(4.0 * math.pi), 0.0, 0.0))
    runs = {}
    for mode in ("plain", "mlp"):
        lim = DG_LIMIT_TVB if mode == "plain" else DG_LIMIT_MLP
        sol = Solver(3, (n, n, n), degree, divb, precision=precision, limiter=lim, positivity=1, Mtilde=Mtilde)
        w, wm = blast_state(sol, params, nvar, device)
        sol.dt(w, wm)  # GLM speeds of the start, as the first step sets them
        dt = torch.tensor([0.0], dtype=torch.float64, device=device)
        if mode == "mlp":
            sol.mlp_set_weights(theta, threshold)
        sol.counters(reset=True)
        rates = []
        sol.profile(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(steps):
            if mode == "plain":
                # detection quality measured on the plain run's own states
                probe = Solver(3, (n, n, n), degree, divb, precision=precision, limiter=DG_LIMIT_TVB,
                               positivity=0, Mtilde=Mtilde) if s == 0 else probe
                if divb == "glm":
                    # the plain decision of the running solver: its current GLM speeds
                    probe.set_glm(*sol.glm_speeds())
                rates.append(detection_rates(probe, w, wm, theta))
            sol.step(w, wm)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        tvb_ms, tvb_n = sol.profile_read(KIND_LIMIT)
        mlp_ms, _ = sol.profile_read(KIND_MLP)
        pos_ms, _ = sol.profile_read(KIND_POSITIVITY)
        sol.profile(False)
        cnt = sol.counters()
        runs[mode] = dict(w=w, wm=wm, wall_s=wall, limiter_ms=tvb_ms + mlp_ms, tvb_ms=tvb_ms, mlp_ms=mlp_ms,
                          pos_ms=pos_ms, limiter_launches=tvb_n, counters=cnt, rates=rates, status=sol.status())
        del sol
    plain, mlp = runs["plain"], runs["mlp"]
    ncell = n ** 3 * steps
    sweep = {}
    for th in THRESHOLDS:
        tot = sum(r[th][3] for r in plain["rates"])
        sweep[str(th)] = {"missed_cell_rate": sum(r[th][0] for r in plain["rates"]) / max(tot, 1),
                          "false_positive_rate": sum(r[th][1] for r in plain["rates"]) / max(ncell - tot, 1),
                          "flagged": sum(r[th][2] for r in plain["rates"])}
    key = min(THRESHOLDS, key=lambda t: abs(t - threshold))
    tot_tv = sum(r[key][3] for r in plain["rates"])
    missed = sum(r[key][0] for r in plain["rates"])
    fp = sum(r[key][1] for r in plain["rates"])
    flagged = sum(r[key][2] for r in plain["rates"])
    wp = plain["wm"] if plain["wm"] is not None else plain["w"]
    wq = mlp["wm"] if mlp["wm"] is not None else mlp["w"]
    # L1 difference of the final cell means per variable, relative to the plain run
    l1 = (torch.abs(wq[:, : n ** 3].double() - wp[:, : n ** 3].double()).sum(1) /
          torch.clamp(torch.abs(wp[:, : n ** 3].double()).sum(1), min=1e-300)).cpu().numpy()
    return {
        "cells": n ** 3, "steps": steps, "scheme": divb, "degree": degree, "threshold": threshold,
        "troubled_plain": tot_tv, "flagged_mlp": flagged,
        "missed_cell_rate": missed / max(tot_tv, 1),
        "false_positive_rate": fp / max(ncell - tot_tv, 1),
        "positivity_cells": {"plain": plain["counters"]["pos_cells"], "mlp": mlp["counters"]["pos_cells"]},
        "floor_injection": {"plain": [plain["counters"]["inj_mass"], plain["counters"]["inj_energy"]],
                            "mlp": [mlp["counters"]["inj_mass"], mlp["counters"]["inj_energy"]]},
        "l1_rel_final_means": [float(x) for x in l1],
        "threshold_sweep": sweep,
        "limiter_ms": {"plain": plain["limiter_ms"], "mlp": mlp["limiter_ms"]},
        "tvb_ms": {"plain": plain["tvb_ms"], "mlp": mlp["tvb_ms"]},
        "mlp_inference_ms": mlp["mlp_ms"],
        "positivity_ms": {"plain": plain["pos_ms"], "mlp": mlp["pos_ms"]},
        "limiter_launches": {"plain": plain["limiter_launches"], "mlp": mlp["limiter_launches"]},
        "wall_s": {"plain": plain["wall_s"], "mlp": mlp["wall_s"]},
        "status": {"plain": plain["status"], "mlp": mlp["status"]},
    }


def evaluate_turbulence(theta, nin, divb="glm", degree=2, n=256, steps=3, threshold=0.1, mach=2.0, seed=1234,
                        precision=DG_PREC_FP32MIX, Mtilde=5.0, device="cuda"):
    """Detection on the decaying-turbulence start (the n^3 workload of the
    benchmark): per step, cells flagged by the network against cells the plain
    TVB procedure changes, on the plain run's own states."""
    import torch
    nvar = 9 if divb == "glm" else 8
    sol = Solver(3, (n, n, n), degree, divb, precision=precision, limiter=DG_LIMIT_TVB, positivity=1,
                 Mtilde=Mtilde)
    w, wm = turbulence_state(sol, seed, mach, nvar, device)
    probe = Solver(3, (n, n, n), degree, divb, precision=precision, limiter=DG_LIMIT_TVB, positivity=0,
                   Mtilde=Mtilde)
    rates = []
    sol.dt(w, wm)
    for _ in range(steps):
        if divb == "glm":
            probe.set_glm(*sol.glm_speeds())
        rates.append(detection_rates(probe, w, wm, theta))
        sol.step(w, wm)
    del sol, probe, w, wm
    torch.cuda.empty_cache()
    key = min(THRESHOLDS, key=lambda t: abs(t - threshold))
    tot = sum(r[key][3] for r in rates)
    cells = n ** 3 * steps
    return {"cells": n ** 3, "steps": steps, "mach": mach, "threshold": threshold,
            "troubled_plain": tot, "flagged_mlp": sum(r[key][2] for r in rates),
            "missed_cell_rate": sum(r[key][0] for r in rates) / max(tot, 1),
            "false_positive_rate": sum(r[key][1] for r in rates) / max(cells - tot, 1),
            "flagged_fraction": sum(r[key][2] for r in rates) / cells}


def weights_path(divb, degree):
    return os.path.join(WEIGHTS_DIR, f"indicator_{divb}_d{degree}.npy")


def load_or_train(divb, degree, device="cuda", **kw):
    """Committed weights if present, else trained now on solver-generated data."""
    import torch
    p = weights_path(divb, degree)
    if os.path.exists(p):
        th = np.load(p)
        return torch.as_tensor(th, dtype=torch.float32, device=device), None
    X, y, nin, src = generate(divb, degree, **kw)
    theta, info = train(X, y, nin, src=src)
    return theta, info


if __name__ == "__main__":
    import argparse
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--divb", default="powell")
    ap.add_argument("--degree", type=int, default=2)
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--seeds", type=int, default=6)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--threshold", type=float, default=0.1)
    ap.add_argument("--neg-per-pos", type=int, default=20)
    ap.add_argument("--pos-weight", type=float, default=4.0)
    ap.add_argument("--eval-n", type=int, default=128)
    ap.add_argument("--eval-steps", type=int, default=10)
    ap.add_argument("--turb", default="64:1:11:1,64:2:12:1,64:4:13:1,128:2:14:0.25,128:4:15:0.25,256:2:16:0.02",
                    help="turbulence sources n:mach:seed:keep, comma separated ('' for none)")
    ap.add_argument("--turb-steps", type=int, default=4)
    ap.add_argument("--turb-every", type=int, default=8)
    ap.add_argument("--turb-eval-n", type=int, default=256)
    ap.add_argument("--save", default="")
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    t0 = time.perf_counter()
    turb = []
    for item in filter(None, args.turb.split(",")):
        nt, mach, sd, keep = item.split(":")
        turb.append((int(nt), float(mach), int(sd), float(keep)))
    X, y, nin, src = generate(args.divb, args.degree, args.n, tuple(range(1, args.seeds + 1)), args.steps,
                              turbulence=turb, turb_steps=args.turb_steps, turb_every=args.turb_every)
    t1 = time.perf_counter()
    theta, info = train(X, y, nin, epochs=args.epochs, src=src, neg_per_pos=args.neg_per_pos,
                        pos_weight=args.pos_weight)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    rep = {"args": vars(args), "samples": int(X.shape[0]), "positives": int(y.sum()),
           "samples_by_source": {"blast": int((src == 0).sum()), "turbulence": int((src == 1).sum())},
           "positives_by_source": {"blast": int(y[src == 0].sum()), "turbulence": int(y[src == 1].sum())},
           "turbulence_sources": turb, "gen_s": t1 - t0, "train_s": t2 - t1, **info}
    del X, y, src
    torch.cuda.empty_cache()
    rep["eval"] = evaluate(theta, nin, args.divb, args.degree, args.eval_n, args.eval_steps, args.threshold)
    if args.turb_eval_n:
        rep["eval_turbulence"] = evaluate_turbulence(theta, nin, args.divb, args.degree, args.turb_eval_n,
                                                     threshold=args.threshold)
    if args.save:
        os.makedirs(os.path.dirname(args.save), exist_ok=True)
        np.save(args.save, theta.cpu().numpy())
    js = json.dumps(rep, indent=1)
    print(js)
    if args.out:
        with open(args.out, "w") as f:
            f.write(js)
