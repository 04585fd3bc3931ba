"""Learned covariance surrogate: data from the DG solver, training, serving.

The network (include/dgsurrogate.h) maps the 128 x 128 occupancy raster of a
periodic cell and (D, Delta) to Sigma / (2 D Delta).  Its training data are
Sigma values of the DG solver (the Sigma scheme of Sec. 4.1 on batched
geometries); the DG solve remains the fallback outside the training envelope
and the reference for the network's error on held-out geometries.  Everything
numeric runs in the library's kernels; this module moves batches around.
"""
from __future__ import annotations

import math
import time

import numpy as np

import dginputs

from . import DG_FP32, DGSolver, Surrogate, rasterize_disks

RES = 128


def conditioning(D: float, delta: float) -> np.ndarray:
    """Network conditioning c = (log(D Delta / um^2), D)."""
    return np.array([math.log(D * delta), D], dtype=np.float32)


def dg_sigma(workloads, device: int = 0, chunk: int = 256, r_factor: float = 8.0):
    """Sigma of every workload at each of its diffusion times, from batched
    FP32 DG solves on the growing window of radius factor r_factor (all
    workloads share the element order p, cell and window).  Returns
    (sigma [n, n_delta, 3], seconds)."""
    out = np.zeros((len(workloads), len(workloads[0].deltas), 3))
    t0 = time.perf_counter()
    for c0 in range(0, len(workloads), chunk):
        ws = workloads[c0:c0 + chunk]
        w0 = ws[0]
        with DGSolver(p=w0.p, precision=DG_FP32, D=w0.D, sigma0=w0.sigma0, device=device) as s:
            s.set_geometry_batch([(w.disks.cx, w.disks.cy, w.disks.r) for w in ws],
                                 [w.L for w in ws], [w.n_cell for w in ws], [w.tiles for w in ws])
            s.set_growing_window(r_factor)
            s.set_sources(np.stack([w.sources for w in ws]))
            for k, d in enumerate(w0.deltas):
                s.propagate_to(d)
                out[c0:c0 + len(ws), k] = s.covariance_batch()[0]
    return out, time.perf_counter() - t0


def build_samples(workloads, sigma):
    """(occ [N, 128, 128] uint8, cond [N, 2], target [N, 3]) for every
    (workload, Delta): target = Sigma / (2 D Delta)."""
    occ, cond, tgt = [], [], []
    for w, sg in zip(workloads, sigma):
        r = rasterize_disks(w.disks.cx, w.disks.cy, w.disks.r, w.L, RES)
        for k, d in enumerate(w.deltas):
            occ.append(r)
            cond.append(conditioning(w.D, d))
            tgt.append(sg[k] / (2.0 * w.D * d))
    return (np.stack(occ).astype(np.uint8), np.stack(cond).astype(np.float32),
            np.stack(tgt).astype(np.float32))


def augment(occ, tgt, k: int, dy: int, dx: int):
    """Exact symmetries of a periodic cell applied to a batch: a periodic
    shift (Sigma unchanged), then for bit 0 of k a flip in x and for bit 1 a
    flip in y (each negates Sxy), for bit 2 a transposition (swaps Sxx and
    Syy).  occ [B, y, x], tgt [B, 3] = (Sxx, Sxy, Syy)."""
    import torch
    o = torch.roll(occ, shifts=(dy, dx), dims=(1, 2))
    t = tgt.clone()
    if k & 1:
        o = torch.flip(o, dims=[2])
        t[:, 1] = -t[:, 1]
    if k & 2:
        o = torch.flip(o, dims=[1])
        t[:, 1] = -t[:, 1]
    if k & 4:
        o = o.transpose(1, 2)
        t = t[:, [2, 1, 0]]
    return o.contiguous(), t.contiguous()


def train(net: Surrogate, occ, cond, tgt, epochs: int = 100, batch: int = 128,
          lr: float = 2e-3, seed: int = 0, augmented: bool = True):
    """Adam on the mean squared error, each batch under a random symmetry of
    the periodic cell; returns the loss history per epoch.  occ/cond/tgt are
    CUDA tensors."""
    import torch
    n = occ.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    for ep in range(epochs):
        rate = lr if ep < int(0.7 * epochs) else lr * 0.2
        perm = torch.randperm(n, generator=g).to(occ.device)
        tot, cnt = 0.0, 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            o, t = occ[idx], tgt[idx]
            if augmented:
                k, dy, dx = (int(v) for v in torch.randint(0, RES, (3,), generator=g))
                o, t = augment(o, t, k % 8, dy, dx)
            loss = net.train_step(o.contiguous(), cond[idx].contiguous(), t.contiguous(), rate)
            tot += loss
            cnt += 1
        hist.append(tot / max(cnt, 1))
    return hist


def packing_features(workloads):
    """(1, phi, phi^2, tau, phi tau, tau^2) per (workload, Delta): phi the
    packing fraction, tau = log(D Delta)."""
    rows = []
    for w in workloads:
        for d in w.deltas:
            ph, lt = w.disks.packing, math.log(w.D * d)
            rows.append([1.0, ph, ph * ph, lt, ph * lt, lt * lt])
    return np.array(rows)


def packing_fit(ws_train, tgt_train, ws_eval):
    """What a user has without the network: least squares of the targets on
    the packing fraction and log(D Delta), evaluated on ws_eval."""
    coef, *_ = np.linalg.lstsq(packing_features(ws_train), np.asarray(tgt_train, np.float64),
                               rcond=None)
    return packing_features(ws_eval) @ coef


class SigmaService:
    """Sigma for a periodic cell: the network inside its training envelope
    (packing and D Delta of the training set), the DG solve outside it."""

    def __init__(self, net: Surrogate, packing_range, tau_range, device: int = 0):
        self.net = net
        self.packing_range = packing_range
        self.tau_range = tau_range
        self.device = device

    def inside(self, w, delta) -> bool:
        tau = w.D * delta
        return (self.packing_range[0] <= w.disks.packing <= self.packing_range[1]
                and self.tau_range[0] <= tau <= self.tau_range[1])

    def sigma(self, w, delta):
        """(sigma3, source) with source 'network' or 'dg'."""
        import torch
        if self.inside(w, delta):
            occ = torch.from_numpy(rasterize_disks(w.disks.cx, w.disks.cy, w.disks.r, w.L, RES)[None]).cuda(self.device)
            cond = torch.from_numpy(conditioning(w.D, delta)[None]).cuda(self.device)
            out = torch.zeros((1, 3), dtype=torch.float32, device=f"cuda:{self.device}")
            self.net.predict(occ, cond, out)
            return out[0].cpu().numpy().astype(np.float64) * 2.0 * w.D * delta, "network"
        ww = dginputs.Workload(w.name, w.p, w.L, w.n_cell, w.tiles, w.D, w.sigma0, [delta], w.disks,
                               w.sources, w.meta)
        sg, _ = dg_sigma([ww], self.device)
        return sg[0, 0], "dg"
