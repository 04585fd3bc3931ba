"""Seeded synthetic inputs for the DG diffusion / covariance path.

This module is shared by the CPU oracle tests and the CUDA path.  It draws
the random substrate (disks with Gamma-distributed radii, placed without
overlap in a periodic square cell) and the random start points of the
Sigma scheme.  It holds none of the method's arithmetic: no element mask,
no DG operator, no moments.  Everything it returns is plain input data
(disk centres and radii in micrometres, start points in micrometres, sizes).

Paper context (Cervantes et al., arXiv 1907.06191):
  * Sec. 1 and Sec. 2.2: the axons are non-overlapping disks whose diameters
    follow a Gamma distribution; the paper's instance has 1901 disks in a
    50 um square, which is not available, so seeded synthetic cells stand in.
  * Sec. 4.1: start points are drawn uniformly at random in the
    extracellular region.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Disks", "gamma_disks", "sample_sources", "window_tiles", "source_box",
    "Workload", "workload_small", "workload_cell40", "workload_batch_member",
    "workload_p5", "free_diffusion_paper", "workload_surrogate_member",
]


@dataclass
class Disks:
    """Disks in a periodic square cell [0, L)^2 (micrometres)."""
    cx: np.ndarray
    cy: np.ndarray
    r: np.ndarray
    L: float
    target_packing: float
    packing: float  # achieved area fraction, sum(pi r^2) / L^2

    @property
    def n(self) -> int:
        return int(self.r.size)


def _min_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.round(d / L)


def gamma_disks(seed: int, L: float, shape: float, scale: float, *,
                n: int | None = None, packing: float | None = None,
                min_gap: float = 0.0, r_min: float = 0.0,
                batch: int = 4096, max_tries: int = 100_000) -> Disks:
    """Non-overlapping disks with Gamma(shape, scale) radii in a periodic cell.

    Either ``n`` (number of radii to draw) or ``packing`` (draw radii until
    their total area reaches ``packing * L^2``) selects how many disks are
    attempted.  Placement is random sequential addition, largest disk first:
    candidate centres are uniform in the cell and accepted when the periodic
    minimum-image distance to every placed disk is at least the sum of radii
    plus ``min_gap``.  A disk that finds no place within ``max_tries``
    candidates is dropped; the achieved packing is returned.
    """
    if (n is None) == (packing is None):
        raise ValueError("give exactly one of n or packing")
    rng = np.random.default_rng(seed)
    if n is not None:
        radii = rng.gamma(shape, scale, size=int(n))
    else:
        radii_l, area = [], 0.0
        goal = float(packing) * L * L
        while area < goal:
            rr = float(rng.gamma(shape, scale))
            radii_l.append(rr)
            area += math.pi * rr * rr
        radii = np.asarray(radii_l)
    radii = np.maximum(radii, r_min)
    # a disk wider than the cell minus the gap cannot be placed periodically
    radii = radii[2.0 * radii + min_gap < L]
    radii = np.sort(radii)[::-1]
    cx = np.empty(radii.size)
    cy = np.empty(radii.size)
    rr_out = np.empty(radii.size)
    # cell lists: two disks can only conflict when their centres are closer
    # than 2 r_max + gap, so a candidate is checked against the disks of its
    # own and the 8 neighbouring cells (periodic); the accepted candidate is
    # the same as with an all-pairs check
    r_max = float(radii[0]) if radii.size else 0.0
    ncell = int(L // (2.0 * r_max + min_gap)) if radii.size else 0
    use_cells = ncell >= 3
    cap = 8
    members = np.zeros((max(ncell, 1) ** 2, cap), dtype=np.int64)
    count = np.zeros(max(ncell, 1) ** 2, dtype=np.int64)
    k = 0
    for r in radii:
        placed = False
        tries = 0
        while tries < max_tries and not placed:
            nb = min(batch, max_tries - tries)
            cand = rng.uniform(0.0, L, size=(nb, 2))
            tries += nb
            if k == 0:
                ok = np.ones(nb, dtype=bool)
            elif not use_cells:
                dx = _min_image(cand[:, 0:1] - cx[None, :k], L)
                dy = _min_image(cand[:, 1:2] - cy[None, :k], L)
                need = (rr_out[None, :k] + r + min_gap) ** 2
                ok = np.all(dx * dx + dy * dy >= need, axis=1)
            else:
                ci = np.minimum((cand[:, 0] * ncell / L).astype(np.int64), ncell - 1)
                cj = np.minimum((cand[:, 1] * ncell / L).astype(np.int64), ncell - 1)
                ok = np.ones(nb, dtype=bool)
                for di in (-1, 0, 1):
                    for dj in (-1, 0, 1):
                        cid = ((cj + dj) % ncell) * ncell + (ci + di) % ncell
                        w = int(count[cid].max())
                        if w == 0:
                            continue
                        idx = members[cid, :w]
                        msk = np.arange(w)[None, :] < count[cid][:, None]
                        dx = _min_image(cand[:, 0:1] - cx[idx], L)
                        dy = _min_image(cand[:, 1:2] - cy[idx], L)
                        need = (rr_out[idx] + r + min_gap) ** 2
                        ok &= np.all((dx * dx + dy * dy >= need) | ~msk, axis=1)
            idx = np.flatnonzero(ok)
            if idx.size:
                cx[k], cy[k] = cand[idx[0]]
                rr_out[k] = r
                if use_cells:
                    c0 = min(int(cy[k] * ncell / L), ncell - 1) * ncell + \
                        min(int(cx[k] * ncell / L), ncell - 1)
                    if count[c0] == cap:
                        members = np.concatenate([members, np.zeros_like(members)], axis=1)
                        cap *= 2
                    members[c0, count[c0]] = k
                    count[c0] += 1
                k += 1
                placed = True
    cx, cy, rr_out = cx[:k].copy(), cy[:k].copy(), rr_out[:k].copy()
    target = float(packing) if packing is not None else float(
        np.sum(math.pi * radii ** 2) / (L * L))
    return Disks(cx, cy, rr_out, float(L), target,
                 float(np.sum(math.pi * rr_out ** 2) / (L * L)))


class NoRoomForSources(RuntimeError):
    """No admissible start point found in the box (the disks, grown by the
    margin, cover it)."""


def sample_sources(seed: int, disks: Disks, m: int, box_lo: float,
                   box_hi: float, margin: float, max_batches: int = 2000) -> np.ndarray:
    """``m`` start points uniform in the box [box_lo, box_hi)^2 (Sec. 4.1).

    A candidate is rejected when it lies within ``r + margin`` of any disk
    (periodic minimum image).  With ``margin`` at least one element side the
    element that contains the point has its centre outside every disk, so the
    point lies in the meshed extracellular region.  Returns an (m, 2) array;
    raises NoRoomForSources after ``max_batches`` batches of 4096 candidates
    without the m points.
    """
    rng = np.random.default_rng(seed)
    out = np.empty((m, 2))
    k = 0
    tries = 0
    while k < m:
        tries += 1
        if tries > max_batches:
            raise NoRoomForSources(f"{k} of {m} start points after {max_batches * 4096} candidates")
        cand = rng.uniform(box_lo, box_hi, size=(4096, 2))
        if disks.n:
            dx = _min_image(cand[:, 0:1] - disks.cx[None, :], disks.L)
            dy = _min_image(cand[:, 1:2] - disks.cy[None, :], disks.L)
            ok = np.all(dx * dx + dy * dy >= (disks.r[None, :] + margin) ** 2,
                        axis=1)
            cand = cand[ok]
        take = min(m - k, cand.shape[0])
        out[k:k + take] = cand[:take]
        k += take
    return out


def window_tiles(L: float, sigma0: float, D: float, delta_max: float,
                 r_factor: float = 6.0) -> int:
    """Number of periodic cells per side of the absorbing solve window.

    Sigma needs unwrapped displacements, so the periodic cell is tiled into a
    finite window with the absorbing edge of Eq. (4).  The diffusion radius is
    R = r_factor * sqrt(sigma0^2 + 2 D delta_max); one cell suffices when
    L >= 3R (start points then stay R away from the edge), otherwise the
    window has 2*ceil(R/L)+1 cells per side and start points lie in the
    central cell.
    """
    R = r_factor * math.sqrt(sigma0 ** 2 + 2.0 * D * delta_max)
    if L >= 3.0 * R:
        return 1
    return 2 * int(math.ceil(R / L)) + 1


def source_box(L: float, tiles: int, sigma0: float, D: float,
               delta_max: float, r_factor: float = 6.0) -> tuple[float, float]:
    """Box (in central-cell coordinates) that start points are drawn from."""
    if tiles == 1:
        R = r_factor * math.sqrt(sigma0 ** 2 + 2.0 * D * delta_max)
        return (R, L - R)
    return (0.0, L)


@dataclass
class Workload:
    """One seeded geometry plus its start points and physical parameters."""
    name: str
    p: int
    L: float               # cell side (um)
    n_cell: int            # elements per cell side
    tiles: int             # cells per window side
    D: float               # diffusivity k0 (um^2/ms)
    sigma0: float          # width of the Gaussian start density (um)
    deltas: list           # diffusion times (ms)
    disks: Disks
    sources: np.ndarray    # (m, 2) start points, central-cell coordinates
    meta: dict = field(default_factory=dict)

    @property
    def h(self) -> float:
        return self.L / self.n_cell

    @property
    def n_window(self) -> int:
        return self.n_cell * self.tiles

    @property
    def origin(self) -> float:
        return -(self.tiles // 2) * self.L


def _workload(name, seed, p, L, n_cell, D, sigma0, deltas, shape, scale, m,
              *, n=None, packing=None, min_gap=0.0, r_factor=6.0, tiles=None):
    disks = gamma_disks(seed, L, shape, scale, n=n, packing=packing,
                        min_gap=min_gap)
    dmax = max(deltas)
    if tiles is None:
        tiles = window_tiles(L, sigma0, D, dmax, r_factor)
    lo, hi = source_box(L, tiles, sigma0, D, dmax, r_factor)
    h = L / n_cell
    src = sample_sources(seed + 7919, disks, m, lo, hi, margin=h)
    return Workload(name, p, L, n_cell, tiles, D, sigma0, list(deltas), disks,
                    src, {"seed": seed, "shape": shape, "scale": scale,
                          "min_gap": min_gap, "r_factor": r_factor})


def workload_small(seed: int = 0, r_factor: float = 6.0) -> Workload:
    """10x10 um periodic cell, 32x32 elements, p=2, 12 Gamma(2, 0.4) disks
    with 0.1 um gaps, D=2 um^2/ms, one sigma0=0.2 um source, Delta=5 ms."""
    return _workload("cell10_p2_32x32", seed, 2, 10.0, 32, 2.0, 0.2, [5.0],
                     2.0, 0.4, 1, n=12, min_gap=0.1, r_factor=r_factor)


def workload_cell40(seed: int = 0, m: int = 64, r_factor: float = 6.0) -> Workload:
    """40x40 um periodic cell, 256x256 elements, p=3, Gamma(2, 0.5) disks at a
    packing drawn uniformly in [0.5, 0.7], 64 start points, D=2 um^2/ms,
    Delta in {5, 10, 20, 50} ms."""
    rng = np.random.default_rng(seed + 104729)
    packing = float(rng.uniform(0.5, 0.7))
    return _workload("cell40_p3_256x256", seed, 3, 40.0, 256, 2.0, 0.2,
                     [5.0, 10.0, 20.0, 50.0], 2.0, 0.5, m, packing=packing,
                     min_gap=0.0, r_factor=r_factor)


def workload_batch_member(seed: int, m: int = 16, delta: float = 20.0) -> Workload:
    """One geometry of the uneven batch: h=0.15625 um, 64..256 elements per
    cell side, p in {2,3,4}, packing 0.40-0.75, Gamma shape 1.5-3.0 with
    scale 0.5 um, 16 start points, Delta = 20 ms (the window is sized for
    ``delta``; the geometry itself does not depend on it)."""
    rng = np.random.default_rng(seed + 15485863)
    n_cell = int(rng.integers(64, 257))
    p = int(rng.choice([2, 3, 4]))
    packing = float(rng.uniform(0.40, 0.75))
    shape = float(rng.uniform(1.5, 3.0))
    h = 40.0 / 256
    return _workload(f"batch{seed}", seed, p, n_cell * h, n_cell, 2.0, 0.2,
                     [float(delta)], shape, 0.5, m, packing=packing)


def workload_surrogate_member(seed: int, m: int = 16) -> Workload:
    """One geometry of the surrogate's training set: 10 um periodic cell of
    32 x 32 elements (h = 0.3125 um), p = 2, Gamma(shape, 0.4 um) disks with
    shape uniform in [1.5, 3.0] at a packing uniform in [0.40, 0.75], 16
    start points, Delta in {1, 2, 3, 4, 5} ms, D = 2 um^2/ms.  A draw whose
    disks leave no room for start points (the last disk can overshoot the
    packing target) is replaced by the draw of seed + 10^7 k, k = 1, 2, ...,
    keeping the name and seed of the slot."""
    for k in range(64):
        sd = seed + 10_000_000 * k
        rng = np.random.default_rng(sd + 32452843)
        packing = float(rng.uniform(0.40, 0.75))
        shape = float(rng.uniform(1.5, 3.0))
        try:
            w = _workload(f"surrogate{seed}", sd, 2, 10.0, 32, 2.0, 0.2,
                          [1.0, 2.0, 3.0, 4.0, 5.0], shape, 0.4, m, packing=packing,
                          min_gap=0.05)
        except NoRoomForSources:
            continue
        w.meta["seed"] = seed
        w.meta["draw_seed"] = sd
        return w
    raise NoRoomForSources(f"no admissible draw for surrogate cell {seed}")


def workload_p5(seed: int = 0, m: int = 32) -> Workload:
    """~153 um cell of 1024x1024 elements, p=5, ~3000 Gamma(2, 0.5) disks,
    32 start points in the central box, Delta=20 ms, one cell."""
    return _workload("cell153_p5_1024x1024", seed, 5, 153.0, 1024, 2.0, 0.2,
                     [20.0], 2.0, 0.5, m, n=3000, tiles=1)


def free_diffusion_paper(n_elem: int = 400, p: int = 2,
                         side: float = 50.0) -> dict:
    """The paper's free-diffusion experiment (Sec. 4.2): a 50 um square with no
    axons, k0 = 450 um^2/s = 0.45 um^2/ms, T = 36 ms, start point at the
    centre.  Analytic covariance 2 T k0 I = 32.4 um^2 I."""
    return {"side": side, "n": n_elem, "p": p, "D": 0.45, "T": 36.0,
            "source": (side / 2.0, side / 2.0)}
