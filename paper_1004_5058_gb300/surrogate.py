"""Learned surrogate of the Herschel-Bulkley flow curve, with the lattice
Boltzmann update as its fallback and its reference.

The network (include/lbhb_mlp.h) maps (log S, G_AA1, G_AA2, G_AB, tau) to the
wall stress sigma_xy and a yielded/arrested logit.  It is trained by the
library's BF16 kernels on points that batched Couette runs of the LB update
produce (flow_curve_dataset), and served in batches: a query outside the
training box, or whose yielded/arrested decision is not clear, is answered by
an LB run instead (serve_with_fallback).

Dataset recipe (one point per Couette cell):
  couplings drawn by a Latin hypercube within +-span around (G^a_AA, G^r_AA,
  G_AB, tau) = (-9, 8.1, 0.405, 1), with G^a_BB = G^a_AA + 1 and
  G^r_BB = G^r_AA - 1 (the offsets of the paper's footnote couplings);
  wall speeds U log-spaced; rho0 = 0.83; seeded random densities
  rho_s = 0.6 (1 +- 0.1 xi) and the linear Couette start; the time averages
  cover the second half of the run.  The label is 1 (yielded) when the bulk
  shear rate (least-squares slope of the central half of the profile) exceeds
  a tenth of the nominal rate 2U/ny.  All cells have one relaxation time tau
  for both species (the paper's model): the network does not cover cells with
  a relaxation time per species.
"""
from __future__ import annotations

import ctypes as C
import math
import time
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import _lib as L
from . import inputs as I

REFERENCE = dict(g_aa1=-9.0, g_aa2=8.1, g_ab=0.405, tau=1.0)
N_IN = 5
CUDA_STREAM_LEGACY = 0x1  # the cudaStream_t value of the legacy default stream


def param_count() -> int:
    return int(L.load().mlp_param_count())


def init_params(seed: int = 0) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), +1/sqrt(fan_in)) weights and biases from the
    SplitMix64 stream, flat in the library's order (W1, b1, ..., W4, b4)."""
    sizes = (5, 128, 128, 128, 2)
    parts, off = [], 0
    for l in range(4):
        fan_in, fan_out = sizes[l], sizes[l + 1]
        n = fan_out * fan_in + fan_out
        u = I.uniform01(seed, n, offset=off)
        off += n
        a = 1.0 / math.sqrt(fan_in)
        parts.append((2.0 * u - 1.0) * a)
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == param_count()
    return p


@dataclass
class Box:
    """Training box of the inputs (log S, G_AA1, G_AA2, G_AB, tau)."""
    center: np.ndarray
    half_range: np.ndarray

    @staticmethod
    def around(x: np.ndarray, pad: float = 0.02) -> "Box":
        lo, hi = x.min(axis=0), x.max(axis=0)
        c = 0.5 * (lo + hi)
        h = 0.5 * (hi - lo) * (1.0 + pad)
        h = np.where(h > 0, h, 1.0)
        return Box(c, h)


class Surrogate:
    """Handle of the BF16 surrogate kernels (mlp_create .. mlp_destroy)."""

    def __init__(self, box: Box, sigma_scale: float, max_batch: int = 4096, lam: float = 1.0, lr: float = 1e-3,
                 logit_margin: float = 1.0, stream="current"):
        """stream: "current" (default) enqueues on torch's current CUDA stream, so
        the kernels are ordered with torch's own work and with its caching
        allocator's reuse of the tensors passed in; or a torch stream / raw
        cudaStream_t value; None for a library-owned stream (the caller must
        then keep input tensors alive until the stream is done)."""
        self.lib = L.load()
        cfg = L.mlp_config()
        cfg.max_batch = int(max_batch)
        cfg.lam, cfg.lr, cfg.beta1, cfg.beta2, cfg.eps = lam, lr, 0.9, 0.999, 1e-8
        for i in range(N_IN):
            cfg.center[i] = float(box.center[i])
            cfg.half_range[i] = float(box.half_range[i])
        cfg.sigma_scale = float(sigma_scale)
        cfg.logit_margin = float(logit_margin)
        self.cfg, self.box, self.max_batch = cfg, box, int(max_batch)
        h = L._H()
        if isinstance(stream, str) and stream == "current":
            import torch
            s = int(torch.cuda.current_stream().cuda_stream) or CUDA_STREAM_LEGACY
        elif stream is None:
            s = None
        else:
            s = (stream if isinstance(stream, int) else int(stream.cuda_stream)) or CUDA_STREAM_LEGACY
        L.check(self.lib.mlp_create(C.byref(cfg), s, C.byref(h)))
        self.h = h
        self.n = param_count()

    def close(self):
        if getattr(self, "h", None):
            self.lib.mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        L.check(self.lib.mlp_set_params(self.h, p.ctypes.data_as(L._F), self.n))
        return self

    def get_params(self) -> np.ndarray:
        p = np.empty(self.n, dtype=np.float32)
        L.check(self.lib.mlp_get_params(self.h, p.ctypes.data_as(L._F), self.n))
        return p

    @staticmethod
    def _ptr(t):
        return C.c_void_p(t.data_ptr())

    def forward(self, x):
        """x: torch float32 cuda [B,5] -> [B,2] (stress, logit)."""
        import torch
        out = torch.empty((x.shape[0], 2), dtype=torch.float32, device=x.device)
        L.check(self.lib.mlp_forward(self.h, self._ptr(x), int(x.shape[0]), self._ptr(out)))
        return out

    def gradients(self, x, target, label):
        g = np.empty(self.n, dtype=np.float32)
        loss = C.c_double()
        L.check(self.lib.mlp_gradients(self.h, self._ptr(x), self._ptr(target), self._ptr(label), int(x.shape[0]),
                                       g.ctypes.data_as(L._F), C.byref(loss)))
        return g, loss.value

    def train_step(self, x, target, label, loss_out=None):
        L.check(self.lib.mlp_train_step(self.h, self._ptr(x), self._ptr(target), self._ptr(label), int(x.shape[0]),
                                        self._ptr(loss_out) if loss_out is not None else None))

    def serve(self, x, out=None):
        """(stress, logit, fallback) for queries x [B,5] (mlp_serve, one kernel).
        out: optional preallocated (stress, logit, fallback) tensors."""
        import torch
        B = int(x.shape[0])
        if out is None:
            stress = torch.empty(B, dtype=torch.float32, device=x.device)
            logit = torch.empty(B, dtype=torch.float32, device=x.device)
            fb = torch.empty(B, dtype=torch.int32, device=x.device)
        else:
            stress, logit, fb = out
        L.check(self.lib.mlp_serve(self.h, self._ptr(x), B, self._ptr(stress), self._ptr(logit), self._ptr(fb)))
        return stress, logit, fb

    def set_error_budget(self, bin_error, log_s_lo: float, log_s_hi: float, budget: float):
        """Queries whose log S bin showed a held-out stress error above `budget`
        are sent to the LB by serve()."""
        e = np.ascontiguousarray(bin_error, dtype=np.float32)
        L.check(self.lib.mlp_set_error_budget(self.h, e.ctypes.data_as(L._F), int(e.size), float(log_s_lo),
                                              float(log_s_hi), float(budget)))
        return self

    def calibrate_error_budget(self, x_val, stress_val, budget: float, n_bins: int = 8):
        """Per-bin median absolute stress error on held-out LB points (x_val,
        stress_val), uploaded as the serving error budget; returns the table."""
        import torch
        X = torch.tensor(np.asarray(x_val), dtype=torch.float32, device="cuda")
        pred = np.concatenate([self.forward(X[k:k + self.max_batch].contiguous())[:, 0].cpu().numpy()
                               for k in range(0, X.shape[0], self.max_batch)]).astype(np.float64)
        ls = np.asarray(x_val)[:, 0]
        lo, hi = self.box.center[0] - self.box.half_range[0], self.box.center[0] + self.box.half_range[0]
        k = np.clip(np.floor((ls - lo) / (hi - lo) * n_bins).astype(int), 0, n_bins - 1)
        err = np.abs(pred - np.asarray(stress_val))
        table = np.array([np.median(err[k == b]) if np.any(k == b) else np.nan for b in range(n_bins)])
        self.set_error_budget(table, lo, hi, budget)
        return table

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.mlp_kernel_launches(self.h))


# ------------------------------------------------------------------ data --
def couplings_lhs(n: int, span: float = 0.15, seed: int = 7):
    """Latin hypercube of n coupling sets (g_aa1, g_aa2, g_ab, tau) within
    +-span of the reference values (SplitMix64 draws)."""
    keys = ("g_aa1", "g_aa2", "g_ab", "tau")
    cols = []
    for j, k in enumerate(keys):
        u = I.uniform01(seed + 101 * j, 2 * n)
        perm = np.argsort(u[:n])
        strata = (perm + u[n:]) / n  # one point per stratum, strata shuffled
        ref = REFERENCE[k]
        cols.append(ref + span * abs(ref) * (2.0 * strata - 1.0))
    return np.stack(cols, axis=1)


def cells_for(couplings: np.ndarray, speeds, L_side: int, rho0: float = 0.83):
    cells = []
    for g_aa1, g_aa2, g_ab, tau in couplings:
        for u in speeds:
            cells.append(I.CellParams(nx=L_side, ny=L_side, tau=float(tau), rho0=rho0, g_aa1=float(g_aa1),
                                      g_aa2=float(g_aa2), g_bb1=float(g_aa1) + 1.0, g_bb2=float(g_aa2) - 1.0,
                                      g_ab=float(g_ab), u_wall=float(u), bc=1))
    return cells


def run_cells(cells, steps: int, seed: int = 1004, precision: str = "fp32", chunk: int = 4096):
    """Batched Couette runs; returns (sigma, S, S_bulk) per cell (time averages
    over the second half of the run)."""
    from .lattice import Lattice
    sig, S, Sb = [], [], []
    for k in range(0, len(cells), chunk):
        part = cells[k:k + chunk]
        nx, ny = part[0].nx, part[0].ny
        ra, rb = I.random_fields(nx, ny, n_cells=len(part), seed=seed + k)
        ux, uy = I.couette_velocity(nx, ny, [c.u_wall for c in part], n_cells=len(part))
        with Lattice(part, precision) as lat:
            lat.init_fields(ra, rb, ux, uy).set_sampling(steps // 2, 10).step(steps)
            s, r, b = lat.shear_stress()
        sig.append(s)
        S.append(r)
        Sb.append(b)
    return np.concatenate(sig), np.concatenate(S), np.concatenate(Sb)


def points_from(cells, sigma, S, S_bulk):
    """(inputs [N,5], stress [N], label [N]) from cell results."""
    ny = cells[0].ny
    nominal = np.array([2.0 * c.u_wall / ny for c in cells])
    S_floor = 1e-3 * nominal
    x = np.stack([np.log(np.maximum(S, S_floor)), [c.g_aa1 for c in cells], [c.g_aa2 for c in cells],
                  [c.g_ab for c in cells], [c.tau for c in cells]], axis=1)
    label = (S_bulk > 0.1 * nominal).astype(np.float64)
    return x, np.asarray(sigma, dtype=np.float64), label


def flow_curve_dataset(n_couplings: int, speeds, L_side: int = 64, steps: int = 20000, span: float = 0.15,
                       seed: int = 7):
    cells = cells_for(couplings_lhs(n_couplings, span, seed), speeds, L_side)
    sigma, S, Sb = run_cells(cells, steps, seed=seed)
    ok = np.isfinite(sigma) & np.isfinite(S)
    x, y, lab = points_from(cells, sigma, S, Sb)
    return x[ok], y[ok], lab[ok], [c for c, o in zip(cells, ok) if o]


# ---------------------------------------------------------------- training --
def train(x: np.ndarray, sigma: np.ndarray, label: np.ndarray, epochs: int = 200, batch: int = 512,
          lr: float = 2e-3, seed: int = 0, sigma_scale: Optional[float] = None, logit_margin: float = 1.0):
    """Trains a fresh surrogate on the points; returns (surrogate, loss history)."""
    import torch
    box = Box.around(x)
    scale = sigma_scale or float(np.max(np.abs(sigma))) or 1.0
    sg = Surrogate(box, scale, max_batch=max(batch, 4096), lr=lr, logit_margin=logit_margin)
    sg.set_params(init_params(seed))
    dev = torch.device("cuda")
    X = torch.tensor(x, dtype=torch.float32, device=dev)
    T = torch.tensor(sigma, dtype=torch.float32, device=dev)
    Y = torch.tensor(label, dtype=torch.float32, device=dev)
    n = X.shape[0]
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    hist = []
    order_seed = seed
    for ep in range(epochs):
        perm = np.argsort(I.uniform01(order_seed + ep, n))
        idx = torch.tensor(perm, device=dev)
        Xs, Ts, Ys = X[idx], T[idx], Y[idx]
        tot, cnt = 0.0, 0
        for k in range(0, n - batch + 1 if n >= batch else 1, batch):
            b = min(batch, n - k)
            sg.train_step(Xs[k:k + b].contiguous(), Ts[k:k + b].contiguous(), Ys[k:k + b].contiguous(), loss)
            if ep == epochs - 1 or ep % 10 == 0:
                tot += float(loss.item()) * b
                cnt += b
        if cnt:
            hist.append(tot / cnt)
    return sg, hist


def serve_with_fallback(sg: Surrogate, x: np.ndarray, L_side: int = 64, steps: int = 20000, seed: int = 99):
    """Answers queries (log S, G_AA1, G_AA2, G_AB, tau): the surrogate where it
    is confident and inside its training box; an LB Couette run at the nominal
    wall speed U = S ny / 2 elsewhere.  Returns dict with stress, logit,
    fallback mask and timings."""
    import torch
    X = torch.tensor(x, dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    stress, logit, fb = sg.serve(X)
    torch.cuda.synchronize()
    t_net = time.perf_counter() - t0
    stress = stress.cpu().numpy().astype(np.float64)
    logit = logit.cpu().numpy().astype(np.float64)
    fb = fb.cpu().numpy().astype(bool)
    t_lb = 0.0
    if fb.any():
        q = x[fb]
        cells = []
        for row in q:
            S = math.exp(row[0])
            cells.append(I.CellParams(nx=L_side, ny=L_side, tau=float(row[4]), rho0=0.83, g_aa1=float(row[1]),
                                      g_aa2=float(row[2]), g_bb1=float(row[1]) + 1.0, g_bb2=float(row[2]) - 1.0,
                                      g_ab=float(row[3]), u_wall=S * L_side / 2.0, bc=1))
        t1 = time.perf_counter()
        s_lb, S_lb, Sb_lb = run_cells(cells, steps, seed=seed)
        t_lb = time.perf_counter() - t1
        stress[fb] = s_lb
        nominal = np.array([2.0 * c.u_wall / L_side for c in cells])
        logit[fb] = np.where(Sb_lb > 0.1 * nominal, 10.0, -10.0)
    return dict(stress=stress, logit=logit, fallback=fb, t_network=t_net, t_lb=t_lb)
