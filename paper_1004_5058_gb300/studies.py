"""Runners of the workloads the library is measured on (all through the C ABI):

precision_study  one Couette cell run three ways (FP64, FP32, FP16-shifted
                 storage), compared with the FP64 run: max |d rho|, relative
                 sigma_xy error, and MLUPS of each.
flow_curve       many Couette cells (wall speeds x cross couplings G_AB) in one
                 batched, graph-captured launch per step; per G_AB the
                 Herschel-Bulkley fit sigma = sigma_Y + A S^beta; flow-curve
                 points per second.  With sequential=True the same cells run one
                 after another (no batching), the plain single-cell baseline of
                 the batched run.
kolmogorov       the paper's forced periodic flow: profiles, shear vs exact
                 stress scatter, Herschel-Bulkley fit, response R;
                 kolmogorov_rho0: R against rho0 and its VFT fit.
surrogate        LB flow-curve points -> training of the BF16 surrogate ->
                 held-out queries served with LB fallback: served fraction,
                 stress error against the LB, and queries per second of the
                 network vs. the LB.

python -m paper_1004_5058_gb300.studies precision|flow_curve [--quick]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs as I
from .lattice import Lattice, hb_fit


def _cuda_time(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def precision_study(n: int = 4096, u_wall: float = 1e-3, steps: int = 50000, every: int = 100,
                    precisions=("fp64", "fp32", "fp16", "fp16sr"), seed: int = 1004, g_ab: float = 0.405):
    """Same cell, same seeded start, each storage precision: MLUPS, the field
    difference from the FP64 run, the wall stress and shear rate against it,
    and the drift of each species' mass."""
    cell = I.make_cell("paper", nx=n, ny=n, g_ab=g_ab, bc=1, u_wall=u_wall)
    ra, rb = I.random_fields(n, n, seed=seed)
    ux, uy = I.couette_velocity(n, n, u_wall)
    res = {}
    for prec in precisions:
        with Lattice([cell], prec) as lat:
            lat.init_fields(ra, rb, ux, uy).set_sampling(steps // 2, every)
            lat.step(10)
            lat.sync()
            lat.init_fields(ra, rb, ux, uy).set_sampling(steps // 2, every)
            _, dt = _cuda_time(lambda: lat.step(steps).sync())
            a, b, _, _ = lat.fields()
            sigma, S, Sb = lat.shear_stress()
            mass, _ = lat.reductions()
            res[prec] = dict(rho_a=a[0], rho_b=b[0], sigma=float(sigma[0]), S=float(S[0]), S_bulk=float(Sb[0]),
                             mlups=n * n * steps / dt / 1e6, seconds=dt, kernel=lat.kernel(),
                             mass_drift=float(abs(mass[0, 0] - ra.sum()) / ra.sum()),
                             mass_drift_b=float(abs(mass[0, 1] - rb.sum()) / rb.sum()))
    ref = res.get("fp64")
    summary = {"n": n, "u_wall": u_wall, "steps": steps, "g_ab": g_ab}
    for prec, r in res.items():
        row = {"mlups": r["mlups"], "seconds": r["seconds"], "sigma_xy": r["sigma"], "shear_rate": r["S"],
               "kernel": r["kernel"], "mass_drift": r["mass_drift"], "mass_drift_b": r["mass_drift_b"]}
        if ref is not None and prec != "fp64":
            row["max_abs_drho"] = float(max(np.abs(r["rho_a"] - ref["rho_a"]).max(),
                                            np.abs(r["rho_b"] - ref["rho_b"]).max()))
            row["sigma_rel_err"] = abs(r["sigma"] - ref["sigma"]) / abs(ref["sigma"])
            row["shear_rate_rel_err"] = abs(r["S"] - ref["S"]) / abs(ref["S"])
        summary[prec] = row
    return summary


def flow_curve(L: int = 512, steps: int = 100000, every: int = 20, n_speeds: int = 16, u_lo: float = 1e-5,
               u_hi: float = 1e-2, g_abs=(0.3, 0.35, 0.405, 0.45), precision: str = "fp32",
               sequential: bool = False, seed: int = 1004):
    """Cells = wall speeds x G_AB values (paper couplings otherwise)."""
    speeds = I.log_spaced(u_lo, u_hi, n_speeds)
    cells = [I.make_cell("paper", nx=L, ny=L, g_ab=g, bc=1, u_wall=u) for g in g_abs for u in speeds]
    ra, rb = I.random_fields(L, L, n_cells=len(cells), seed=seed)
    ux, uy = I.couette_velocity(L, L, [c.u_wall for c in cells], n_cells=len(cells))
    if not sequential:
        with Lattice(cells, precision) as lat:
            lat.init_fields(ra, rb, ux, uy)
            kern = lat.autotune()
            lat.init_fields(ra, rb, ux, uy).set_sampling(steps // 2, every)
            _, dt = _cuda_time(lambda: lat.step(steps).sync())
            sigma, S, Sb = lat.shear_stress()
    else:
        # the same cells one at a time (no batching), each with its own tuned tile
        sig_l, S_l, Sb_l = [], [], []
        kern = None
        dt = 0.0
        for c, cell in enumerate(cells):
            with Lattice([cell], precision) as lat:
                lat.init_fields(ra[c:c + 1], rb[c:c + 1], ux[c:c + 1], uy[c:c + 1])
                kern = lat.autotune()
                lat.init_fields(ra[c:c + 1], rb[c:c + 1], ux[c:c + 1], uy[c:c + 1]).set_sampling(steps // 2, every)
                _, t = _cuda_time(lambda: lat.step(steps).sync())
                dt += t
                s, r, b = lat.shear_stress()
            sig_l.append(s[0])
            S_l.append(r[0])
            Sb_l.append(b[0])
        sigma, S, Sb = np.array(sig_l), np.array(S_l), np.array(Sb_l)
    out = {"L": L, "steps": steps, "cells": len(cells), "precision": precision, "kernel": kern,
           "seconds": dt, "mlups": len(cells) * L * L * steps / dt / 1e6, "points_per_s": len(cells) / dt,
           "curves": {}}
    for k, g in enumerate(g_abs):
        sl = slice(k * n_speeds, (k + 1) * n_speeds)
        s_, r_ = sigma[sl], S[sl]
        ok = np.isfinite(r_) & (r_ > 0) & np.isfinite(s_)
        fit = hb_fit(r_[ok], s_[ok]) if ok.sum() >= 3 else None
        out["curves"][str(g)] = {"u_wall": list(speeds), "sigma_xy": [float(v) for v in s_],
                                 "shear_rate": [float(v) for v in r_], "shear_bulk": [float(v) for v in Sb[sl]],
                                 "hb_fit": fit}
    return out


def kolmogorov(L: int = 512, steps: int = 1000000, every: int = 100, rho0s=(0.83, 0.81),
               u0s=(0.1, 0.2, 0.25, 0.3, 0.35, 0.4, 0.5, 0.6), g_ab: float = 0.405, precision: str = "fp32",
               noise: float = 1e-3, seed: int = 1004, r_flow: float = 0.05):
    """The paper's own workload (section "Numerical Results"): a fully periodic
    L x L box, body force F_x(y) = F0 sin(k y), k = 2 pi / L, with F0 tuned so
    that the laminar flow would peak at U0 (F0 = rho nu k^2 U0), the paper's
    sinusoidal initial densities, footnote couplings (G_AB read as 0.405).
    Per cell: the time- and line-averaged profile U(y), the shear S(y) = dU/dy
    (central difference), the exact stress sigma(y) = (F0/k) cos(k y) of the
    momentum balance, the response R = U_hat / U0 with
    U_hat = 2/L sum_y U(y) sin(k y), and the Herschel-Bulkley fit of the
    (S, sigma) scatter where both are positive.

    noise: relative seeded perturbation of the initial densities that breaks
    their invariance under x translations (without it the lamellae of the
    sinusoidal start stay lamellae, parallel to the flow, and R = 1).  Per cell
    the final state is summarised by the spread of rho_A (std over the box) and
    its mean spread along x (droplets: comparable to the total; lamellae: 0).

    Per rho0, the (S(y), sigma(y)) points of all runs that flow (R > r_flow)
    are pooled into one scatter, the paper's master curve, and fitted with the
    Herschel-Bulkley law; the largest forcing amplitude sigma0 = F0/k of the runs
    that do not flow bounds the yield stress from below."""
    k = 2.0 * np.pi / L
    cells = []
    for r0 in rho0s:
        for u0 in u0s:
            cells.append(I.make_cell("paper", nx=L, ny=L, rho0=r0, g_ab=g_ab, f0=I.kolmogorov_f0(u0, L)))
    ra, rb = I.sine_fields(L, L, n_cells=len(cells), noise=noise, seed=seed)
    with Lattice(cells, precision) as lat:
        lat.init_fields(ra, rb)
        kern = lat.autotune()
        lat.init_fields(ra, rb).set_sampling(steps // 2, every)
        _, dt = _cuda_time(lambda: lat.step(steps).sync())
        ub, ns = lat.profile()
        fa = lat.fields()[0]
    y = np.arange(L)
    out = {"L": L, "steps": steps, "cells": len(cells), "noise": noise, "kernel": kern, "seconds": dt,
           "mlups": len(cells) * L * L * steps / dt / 1e6, "samples": ns, "runs": []}
    for c, cell in enumerate(cells):
        u0 = u0s[c % len(u0s)]
        U = ub[c]
        S = (np.roll(U, -1) - np.roll(U, 1)) / 2.0
        sig = cell.f0 / k * np.cos(k * y)
        R = 2.0 / L * np.sum(U * np.sin(k * y)) / u0
        ok = (S > 0) & (sig > 0)
        fit = hb_fit(S[ok], sig[ok]) if ok.sum() >= 3 else None
        out["runs"].append({"rho0": cell.rho0, "u0": u0, "f0": cell.f0, "sigma0": cell.f0 / k, "R": float(R),
                            "u_max": float(np.max(np.abs(U))), "hb_fit": fit,
                            "rho_a_std": float(np.std(fa[c])), "rho_a_std_x": float(np.mean(np.std(fa[c], axis=1))),
                            "profile": [float(v) for v in U]})
    out["master"] = {}
    for r0 in rho0s:
        runs = [(c, r) for c, r in enumerate(out["runs"]) if r["rho0"] == r0]
        pts_S, pts_s = [], []
        for c, r in runs:
            if r["R"] <= r_flow:
                continue
            U = np.array(r["profile"])
            S = (np.roll(U, -1) - np.roll(U, 1)) / 2.0
            sig = r["f0"] / k * np.cos(k * y)
            ok = (S > 0) & (sig > 0)
            pts_S.extend(S[ok])
            pts_s.extend(sig[ok])
        arrested = [r["sigma0"] for _, r in runs if r["R"] <= r_flow]
        pts_S, pts_s = np.array(pts_S), np.array(pts_s)
        out["master"][str(r0)] = {
            "flowing_runs": int(sum(1 for _, r in runs if r["R"] > r_flow)), "points": int(pts_S.size),
            "largest_arrested_sigma0": float(max(arrested)) if arrested else None,
            "hb_fit": hb_fit(pts_S, pts_s) if pts_S.size >= 3 else None}
    return out


def vft_fit(rho0, inv_r, rho_c_hi: float = 1.2):
    """Vogel-Fulcher-Tammann law 1/R = A exp(B / (rho_c - rho0)) (the paper's fit of
    the reciprocal response): for fixed rho_c, ln(1/R) is linear in (ln A, B);
    rho_c > max(rho0) minimises the residual (scan + refinement)."""
    x = np.asarray(rho0, dtype=np.float64)
    yl = np.log(np.asarray(inv_r, dtype=np.float64))

    def solve(rc):
        X = np.stack([np.ones_like(x), 1.0 / (rc - x)], axis=1)
        coef, *_ = np.linalg.lstsq(X, yl, rcond=None)
        r = yl - X @ coef
        return float(r @ r), coef

    lo = x.max() + 1e-4
    grid = np.linspace(lo, rho_c_hi, 4001)
    vals = [solve(rc)[0] for rc in grid]
    k = int(np.argmin(vals))
    a, b = grid[max(k - 1, 0)], grid[min(k + 1, len(grid) - 1)]
    for _ in range(100):  # golden section
        c1, c2 = b - 0.618033988749895 * (b - a), a + 0.618033988749895 * (b - a)
        if solve(c1)[0] < solve(c2)[0]:
            b = c2
        else:
            a = c1
    rc = 0.5 * (a + b)
    rss, coef = solve(rc)
    return {"A": float(np.exp(coef[0])), "B": float(coef[1]), "rho_c": float(rc), "rss": rss}


def kolmogorov_rho0_sweep(L: int = 512, steps: int = 1000000, u0: float = 0.1,
                          rho0s=(0.70, 0.72, 0.74, 0.75, 0.76, 0.77, 0.78, 0.79, 0.80, 0.81, 0.83, 0.85),
                          g_ab: float = 0.405, r_floor: float = 0.02):
    """Response R = U_hat / U0 against rho0 at fixed forcing (U0 = 0.1), and the
    VFT fit of 1/R (the paper's arrest analysis) over the runs whose response is
    above the floor r_floor (below it the box has arrested and the time-averaged
    profile is residual motion)."""
    out = kolmogorov(L=L, steps=steps, rho0s=rho0s, u0s=(u0,), g_ab=g_ab)
    R = np.array([r["R"] for r in out["runs"]])
    ok = R > r_floor
    out["vft_points"] = int(ok.sum())
    out["vft"] = vft_fit(np.array(rho0s)[ok], 1.0 / R[ok]) if ok.sum() >= 4 else None
    return out


def belt_scale_stability(L: int = 128, steps: int = 20000, chunk: int = 500, scale: float = 3.0,
                         taus=(1.0, 0.8, 0.7, 0.6), g_ab: float = 0.405, seed: int = 1004):
    """The other reading of the interaction weights' overall scale (both belts
    with sum w c_x^2 = 1 instead of 1/3 = c_s^2): forces scale with G w, so it is
    the paper's couplings times `scale`.  Runs the sine start under each
    relaxation time and reports the first step at which the watchdog finds a
    non-finite or non-positive density (None: stable for all `steps`)."""
    from ._lib import LBError
    base = I.make_cell("paper", nx=L, ny=L, g_ab=g_ab)
    out = {"L": L, "steps": steps, "scale": scale, "g_ab": g_ab, "runs": []}
    ra, rb = I.sine_fields(L, L, noise=1e-3, seed=seed)
    for tau in taus:
        cell = I.make_cell("paper", nx=L, ny=L, tau=tau, g_aa1=scale * base.g_aa1, g_aa2=scale * base.g_aa2,
                           g_bb1=scale * base.g_bb1, g_bb2=scale * base.g_bb2, g_ab=scale * g_ab)
        blew = None
        with Lattice([cell], "fp32") as lat:
            lat.init_fields(ra, rb)
            done = 0
            while done < steps:
                try:
                    lat.step(chunk).sync()
                except LBError:
                    blew = done + chunk
                    break
                done += chunk
            spread = None if blew else float(np.std(lat.fields()[0][0]))
        out["runs"].append({"tau": tau, "unstable_by_step": blew, "rho_a_std": spread})
    return out


def kolmogorov_readings(L: int = 512, steps: int = 1000000, u0s=(0.1, 0.2, 0.25, 0.3, 0.35, 0.4, 0.5, 0.6),
                        rho0s=(0.83, 0.81), g_abs=(0.405, 0.045),
                        sweep_rho0s=(0.70, 0.72, 0.74, 0.76, 0.78, 0.80, 0.83, 0.85)):
    """The paper's Kolmogorov experiment under each reading of what it does not
    print unambiguously: the cross coupling (the footnote's G_AB = 0.045 against
    0.405) with the D2Q9-scale interaction weights, and the belt-weight scale
    (sum w c_x^2 = 1, the paper's couplings times 3) by its stability.  Per
    G_AB: the master-curve Herschel-Bulkley fit per rho0, the largest arrested
    forcing, and the response R(rho0) at U0 = 0.1 with its VFT fit."""
    out = {"L": L, "steps": steps, "readings": {}}
    for g in g_abs:
        # a mixture that stays mixed flows with R ~ 1, i.e. at the laminar peak
        # speed U0 itself; above U0 ~ 0.3 (a Mach number above one half) the
        # update blows up, which the watchdog reports: forcings up to 0.3 only
        u0s_g = u0s if g >= 0.1 else tuple(u for u in u0s if u <= 0.3)
        fc = kolmogorov(L=L, steps=steps, rho0s=rho0s, u0s=u0s_g, g_ab=g)
        sw = kolmogorov_rho0_sweep(L=L, steps=steps, rho0s=sweep_rho0s, g_ab=g)
        out["readings"]["g_ab=%g" % g] = {
            "master": fc["master"], "seconds": fc["seconds"] + sw["seconds"], "u0s": list(u0s_g),
            "runs": [{k: r[k] for k in ("rho0", "u0", "sigma0", "R", "rho_a_std", "rho_a_std_x")} for r in fc["runs"]],
            "R_of_rho0": [{"rho0": r["rho0"], "R": r["R"], "rho_a_std": r["rho_a_std"]} for r in sw["runs"]],
            "vft": sw["vft"]}
    out["belt_scale_x3"] = belt_scale_stability(L=128, steps=20000)
    return out


def surrogate_study(n_train: int = 600, n_test: int = 64, n_speeds: int = 16, L: int = 64, steps: int = 20000,
                    epochs: int = 300, batch: int = 256, lr: float = 2e-3, seed: int = 11):
    """Train on n_train x n_speeds LB points, score on n_test x n_speeds held-out points."""
    import time as _t
    import torch
    from . import surrogate as S
    speeds = I.log_spaced(2e-4, 2e-2, n_speeds)
    t0 = _t.perf_counter()
    x, sig, lab, _ = S.flow_curve_dataset(n_train, speeds, L_side=L, steps=steps, seed=seed)
    t_data = _t.perf_counter() - t0
    xt, st, lt, _ = S.flow_curve_dataset(n_test, speeds, L_side=L, steps=steps, seed=seed + 1000)
    t0 = _t.perf_counter()
    sg, hist = S.train(x, sig, lab, epochs=epochs, batch=batch, lr=lr, logit_margin=0.5)
    torch.cuda.synchronize()
    t_train = _t.perf_counter() - t0
    # error budget of serving: 10% of the largest training stress, per log S bin
    budget = 0.1 * float(np.max(np.abs(sig)))
    table = sg.calibrate_error_budget(x, sig, budget, n_bins=8)
    inside = np.all(np.abs(xt - sg.box.center) <= sg.box.half_range, axis=1)
    q, qs, ql = xt[inside], st[inside], lt[inside]
    X = torch.tensor(q, dtype=torch.float32, device="cuda")
    stress, logit, fb = sg.serve(X)
    stress, logit, fb = stress.cpu().numpy(), logit.cpu().numpy(), fb.cpu().numpy().astype(bool)
    # serving rate on batches of 4096 queries (the held-out queries repeated)
    X4k = X.repeat((4096 + len(q) - 1) // len(q), 1)[:4096].contiguous()
    outs = sg.serve(X4k)  # a serving loop reuses its output buffers
    torch.cuda.synchronize()
    reps = 50
    t0 = _t.perf_counter()
    for _ in range(reps):
        sg.serve(X4k, out=outs)
    torch.cuda.synchronize()
    t_serve = (_t.perf_counter() - t0) / reps
    served = ~fb
    err = np.abs(stress - qs)
    scale = float(np.max(np.abs(st)))
    # the method without the network: one LB cell run per point, batched (data generation rate)
    return {"train_points": int(len(x)), "test_points": int(len(q)), "cell": L, "steps": steps,
            "data_seconds": t_data, "lb_points_per_s": len(x) / t_data, "train_seconds": t_train,
            "loss_first": hist[0], "loss_last": hist[-1], "served_fraction": float(served.mean()),
            "error_budget": budget, "error_table_by_logS_bin": [float(v) for v in table],
            "stress_scale": scale, "median_abs_err_served": float(np.median(err[served])) if served.any() else None,
            "p90_abs_err_served": float(np.quantile(err[served], 0.9)) if served.any() else None,
            "median_rel_err_served": float(np.median(err[served]) / scale) if served.any() else None,
            "yield_agreement_served": float(np.mean((logit[served] > 0) == (ql[served] > 0.5))) if served.any() else None,
            "network_queries_per_s": 4096 / t_serve, "network_seconds_per_4096_batch": t_serve,
            "gain_queries_per_s": (4096 / t_serve) / (len(x) / t_data)}


def two_time_flow_curve(L: int = 256, steps: int = 500000, every: int = 50, n_speeds: int = 16,
                        u_lo: float = 1e-5, u_hi: float = 1e-2, tau_bs=(0.7, 1.0, 1.5), g_ab: float = 0.405,
                        precision: str = "fp32", seed: int = 1004):
    """The Couette flow curve with a relaxation time per species (the
    coupling-dependent relaxation time the paper leaves unexplored): species A
    keeps tau = 1, species B takes each tau_b in turn; cells = tau_b values x
    wall speeds in one batch, the second half of the steps sampled, a
    Herschel-Bulkley fit per tau_b.  The default 256^2 cells run 5e5 steps,
    longer than the viscous time L^2/nu of every mixture here."""
    speeds = I.log_spaced(u_lo, u_hi, n_speeds)
    cells = [I.make_cell("paper", nx=L, ny=L, g_ab=g_ab, bc=1, u_wall=u, tau=1.0, tau_b=tb)
             for tb in tau_bs for u in speeds]
    ra, rb = I.random_fields(L, L, n_cells=len(cells), seed=seed)
    ux, uy = I.couette_velocity(L, L, [c.u_wall for c in cells], n_cells=len(cells))
    with Lattice(cells, precision) as lat:
        lat.init_fields(ra, rb, ux, uy)
        kern = lat.autotune()
        lat.init_fields(ra, rb, ux, uy).set_sampling(steps // 2, every)
        _, dt = _cuda_time(lambda: lat.step(steps).sync())
        sigma, S, Sb = lat.shear_stress()
    out = {"L": L, "steps": steps, "cells": len(cells), "precision": precision, "g_ab": g_ab, "kernel": kern,
           "seconds": dt, "mlups": len(cells) * L * L * steps / dt / 1e6, "curves": {}}
    for k, tb in enumerate(tau_bs):
        sl = slice(k * n_speeds, (k + 1) * n_speeds)
        s_, r_ = sigma[sl], S[sl]
        ok = np.isfinite(r_) & (r_ > 0) & np.isfinite(s_) & (s_ > 0)
        out["curves"][str(tb)] = {"u_wall": list(speeds), "sigma_xy": [float(v) for v in s_],
                                  "shear_rate": [float(v) for v in r_], "shear_bulk": [float(v) for v in Sb[sl]],
                                  "hb_fit": hb_fit(r_[ok], s_[ok]) if ok.sum() >= 3 else None}
    return out


def slab_throughput(n: int = 4096, steps: int = 400, worlds=(2, 4, 8), precision: str = "fp32",
                    u_wall: float = 1e-3, seed: int = 1004):
    """One Couette cell of n x n as the whole cell and as `world` horizontal
    slabs on this one device, all on one stream with the stream-ordered
    exchange (slabs.StreamExchange): site updates per second of each, timed
    with CUDA events around `steps` steps after a warm-up, and whether the slabs'
    final populations equal the whole cell's bit for bit.  The slabs' kernels
    are those of a multi-device split; what one device cannot show is the
    transfer between devices."""
    import torch
    from .slabs import SlabLattice, StreamExchange, split_rows
    cell = I.make_cell("paper", nx=n, ny=n, g_ab=0.405, bc=1, u_wall=u_wall)
    ra, rb = I.random_fields(n, n, seed=seed)
    ux, uy = I.couette_velocity(n, n, u_wall)
    fields = (ra, rb, ux, uy)
    stream = torch.cuda.Stream()

    def timed(run):
        run(10)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        run(steps)
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) * 1e-3

    out = {"n": n, "steps": steps, "precision": precision, "runs": []}
    with Lattice([cell], precision, stream=stream) as lat:
        lat.init_fields(*fields)
        dt = timed(lambda k: lat.step(k))
        whole = lat.get_populations()[0]
        out["whole"] = {"seconds": dt, "mlups": n * n * steps / dt / 1e6, "kernel": lat.kernel()}
    for world in worlds:
        parts = split_rows(n, world)
        slabs = [SlabLattice([cell], y0, rows, precision, stream=stream) for y0, rows in parts]
        try:
            for s_, (y0, rows) in zip(slabs, parts):
                s_.lat.init_fields(*[a[:, y0:y0 + rows] for a in fields])
            ex = StreamExchange(slabs, periodic=False)
            dt = timed(lambda k: ex.step(k))
            got = np.concatenate([s_.lat.get_populations()[0] for s_ in slabs], axis=2)
            out["runs"].append({"world": world, "seconds": dt, "mlups": n * n * steps / dt / 1e6,
                                "relative_to_whole": out["whole"]["seconds"] / dt,
                                "launches_per_step": sum(s_.lat.kernel_launches for s_ in slabs) / (steps + 10),
                                "bitwise_equal_to_whole": bool(np.array_equal(got, whole))})
        finally:
            for s_ in slabs:
                s_.close()
    return out


MRT_CONFIGS = (("BGK, G_AB 0.30", 0.30, {}), ("MRT s_nu 1.6, G_AB 0.30", 0.30, {"s_nu": 1.6}),
               ("BGK, G_AB 0.405", 0.405, {}), ("MRT s_q 1.2, G_AB 0.405", 0.405, {"s_q": 1.2}))


def mrt_flow_curve(L: int = 128, steps: int = 400000, every: int = 50, n_speeds: int = 16, u_lo: float = 1e-5,
                   u_hi: float = 1e-2, configs=MRT_CONFIGS, precision: str = "fp32", seed: int = 1004):
    """Couette flow curves with the multiple-relaxation-time collision (a method
    variant) beside the paper's BGK one, all cells in one batch: per
    configuration (label, G_AB, rates; tau = 1) n_speeds wall speeds, the second
    half of the steps sampled.  Reports the Newtonian ratio sigma/S (rho nu),
    the Herschel-Bulkley fit and the spread of rho_A (the demixing) per
    configuration.  The default 128^2 cells run 4e5 steps, beyond the viscous
    time L^2/nu of the least viscous configuration (nu = 1/24)."""
    speeds = I.log_spaced(u_lo, u_hi, n_speeds)
    cells = [I.make_cell("paper", nx=L, ny=L, g_ab=g, bc=1, u_wall=u, tau=1.0, **rates)
             for _, g, rates in configs for u in speeds]
    ra, rb = I.random_fields(L, L, n_cells=len(cells), seed=seed)
    ux, uy = I.couette_velocity(L, L, [c.u_wall for c in cells], n_cells=len(cells))
    with Lattice(cells, precision) as lat:
        lat.init_fields(ra, rb, ux, uy)
        kern = lat.autotune()
        lat.init_fields(ra, rb, ux, uy).set_sampling(steps // 2, every)
        _, dt = _cuda_time(lambda: lat.step(steps).sync())
        sigma, S, Sb = lat.shear_stress()
        rho_a = lat.fields()[0]
    out = {"L": L, "steps": steps, "cells": len(cells), "precision": precision, "kernel": kern,
           "seconds": dt, "mlups": len(cells) * L * L * steps / dt / 1e6, "curves": {}}
    for k, (label, g, rates) in enumerate(configs):
        sl = slice(k * n_speeds, (k + 1) * n_speeds)
        s_, r_ = sigma[sl], S[sl]
        ok = np.isfinite(r_) & (r_ > 0) & np.isfinite(s_) & (s_ > 0)
        out["curves"][label] = {"g_ab": g, "rates": rates, "u_wall": list(speeds),
                                "sigma_xy": [float(v) for v in s_], "shear_rate": [float(v) for v in r_],
                                "shear_bulk": [float(v) for v in Sb[sl]],
                                "sigma_over_S": [float(a / b) if b != 0 else None for a, b in zip(s_, r_)],
                                "rho_a_std": [float(np.std(rho_a[c])) for c in range(sl.start, sl.stop)],
                                "hb_fit": hb_fit(r_[ok], s_[ok]) if ok.sum() >= 3 else None}
    return out


def couette_flow_curve(n: int = 1024, n_speeds: int = 8, steps: int = 200000, every: int = 10, g_ab: float = 0.405,
                       precision: str = "fp32", seed: int = 1004):
    """The benchmark's configuration run to its end: n_speeds Couette cells of
    n x n, wall speeds U = 10^(-4 + 2k/(n_speeds-1)), linear-profile start, the
    second half of the steps sampled; per cell the wall stress and shear rate,
    and the Herschel-Bulkley fit of the curve."""
    speeds = I.log_spaced(1e-4, 1e-2, n_speeds)
    cells = [I.make_cell("paper", nx=n, ny=n, g_ab=g_ab, bc=1, u_wall=u) for u in speeds]
    ra, rb = I.random_fields(n, n, n_cells=n_speeds, seed=seed)
    ux, uy = I.couette_velocity(n, n, speeds, n_cells=n_speeds)
    with Lattice(cells, precision) as lat:
        lat.init_fields(ra, rb, ux, uy)
        kern = lat.autotune()
        lat.init_fields(ra, rb, ux, uy).set_sampling(steps // 2, every)
        _, dt = _cuda_time(lambda: lat.step(steps).sync())
        sigma, S, Sb = lat.shear_stress()
        ub, ns = lat.profile()
    ok = np.isfinite(S) & (S > 0) & np.isfinite(sigma) & (sigma > 0)
    return {"n": n, "steps": steps, "cells": n_speeds, "precision": precision, "g_ab": g_ab, "kernel": kern,
            "seconds": dt, "mlups": n_speeds * n * n * steps / dt / 1e6, "points_per_s": n_speeds / dt,
            "samples": ns, "u_wall": list(speeds), "sigma_xy": [float(v) for v in sigma],
            "shear_rate": [float(v) for v in S], "shear_bulk": [float(v) for v in Sb],
            "nominal_rate": [2.0 * u / n for u in speeds],
            "hb_fit": hb_fit(S[ok], sigma[ok]) if ok.sum() >= 3 else None}


# surrogate layers (inputs, outputs): 5 -> 128 -> 128 -> 128 -> 2
SURROGATE_LAYERS = ((5, 128), (128, 128), (128, 128), (128, 2))


def surrogate_train_rate(batch: int = 10240, steps: int = 50, warmup: int = 5, seed: int = 0):
    """Training throughput of the surrogate's BF16 kernels at one batch size:
    Adam steps (forward, loss, backward, update; mlp_train_step) on seeded
    points inside a training box around the paper's couplings, timed with CUDA
    events on the handle's stream.  FLOPs per sample: the forward products
    2 sum(in*out), the weight gradients as many, and the input gradients of
    layers 2..4 (the network's input needs none)."""
    import torch
    from .surrogate import Box, Surrogate, init_params, N_IN
    center = np.array([math.log(1e-4), -9.0, 8.1, 0.405, 1.0])
    half = np.array([3.0, 1.35, 1.2, 0.06, 0.15])
    u = I.uniform01(seed, batch * N_IN).reshape(batch, N_IN)
    x = center + half * (2.0 * u - 1.0)
    t = 1e-4 * I.uniform01(seed + 1, batch)
    lab = (I.uniform01(seed + 2, batch) > 0.5).astype(np.float64)
    dev = torch.device("cuda")
    X = torch.tensor(x, dtype=torch.float32, device=dev)
    T = torch.tensor(t, dtype=torch.float32, device=dev)
    Y = torch.tensor(lab, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    sg = Surrogate(Box(center, half), 1e-4, max_batch=batch, lr=1e-3)
    try:
        sg.set_params(init_params(seed))
        for _ in range(warmup):
            sg.train_step(X, T, Y, loss)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            sg.train_step(X, T, Y, loss)
        e1.record(stream)
        e1.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3 / steps
        launches = sg.kernel_launches
        final_loss = float(loss.item())
    finally:
        sg.close()
    mac = sum(i * o for i, o in SURROGATE_LAYERS)
    flops = batch * (2 * mac + 2 * mac + 2 * sum(i * o for i, o in SURROGATE_LAYERS[1:]))
    return {"batch": batch, "steps": steps, "us_per_step": sec * 1e6, "samples_per_s": batch / sec,
            "flops_per_step": flops, "tflops": flops / sec / 1e12, "loss": final_loss,
            "kernel_launches": launches}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["precision", "precision_mixed", "flow_curve", "flow_curve_sequential",
                                      "flow_curve_long", "couette_1024", "surrogate", "kolmogorov",
                                      "kolmogorov_rho0", "two_time", "train_rate", "readings", "mrt", "slabs"])
    ap.add_argument("--batch", type=int, default=10240, help="train_rate: batch size")
    ap.add_argument("--quick", action="store_true", help="small sizes for a smoke run")
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    if a.study == "precision":
        r = precision_study(n=512, steps=2000) if a.quick else precision_study()
    elif a.study == "precision_mixed":  # the paper's footnote G_AB = 0.045: the mixture stays mixed
        r = precision_study(n=512, steps=2000, g_ab=0.045) if a.quick else precision_study(g_ab=0.045)
    elif a.study == "kolmogorov":
        r = kolmogorov(L=128, steps=20000, u0s=(0.05, 0.1)) if a.quick else kolmogorov()
    elif a.study == "kolmogorov_rho0":
        r = kolmogorov_rho0_sweep(L=128, steps=20000) if a.quick else kolmogorov_rho0_sweep()
    elif a.study == "couette_1024":  # the benchmark's 8 cells of 1024^2 for the full 2e5 steps
        r = couette_flow_curve(n=128, steps=4000) if a.quick else couette_flow_curve()
    elif a.study == "flow_curve_long":  # the batched 64 x 512^2 cells for 1e6 steps (steady state)
        r = flow_curve(L=128, steps=4000, n_speeds=4) if a.quick else flow_curve(steps=1000000, every=100)
    elif a.study == "two_time":  # relaxation time per species: flow curves for three tau_B
        r = two_time_flow_curve(L=64, steps=4000, n_speeds=4) if a.quick else two_time_flow_curve()
    elif a.study == "slabs":  # one cell as slabs on this device, stream-ordered exchange
        r = slab_throughput(n=256, steps=50, worlds=(2, 4)) if a.quick else slab_throughput()
    elif a.study == "mrt":  # multiple relaxation times beside BGK: Newtonian and demixing flow curves
        r = mrt_flow_curve(L=32, steps=4000, n_speeds=4) if a.quick else mrt_flow_curve()
    elif a.study == "readings":
        r = (kolmogorov_readings(L=64, steps=4000, u0s=(0.1, 0.3), sweep_rho0s=(0.7, 0.75, 0.8, 0.85))
             if a.quick else kolmogorov_readings())
    elif a.study == "train_rate":
        r = surrogate_train_rate(batch=a.batch, steps=10 if a.quick else 50)
    elif a.study == "surrogate":
        r = surrogate_study(n_train=48, n_test=12, n_speeds=8, L=32, steps=3000) if a.quick else surrogate_study()
    else:
        kw = dict(L=128, steps=2000, n_speeds=4) if a.quick else {}
        r = flow_curve(sequential=a.study.endswith("sequential"), **kw)
    s = json.dumps(r, default=lambda o: o.tolist() if hasattr(o, "tolist") else str(o))
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(s + "\n")
    print(s)


if __name__ == "__main__":
    main()
