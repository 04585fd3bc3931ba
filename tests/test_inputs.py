"""The seeded input generators (``dginputs``): the synthetic substrates and
start points that stand in for the paper's axon packing (Sec. 2.2, Sec. 4.1).

Each property is checked by brute force, independently of how the generator
computes it: disks never overlap (all pairs, periodic minimum image, gap
included), radii follow the Gamma law they are drawn from, start points lie
in their box and clear of every disk, the absorbing window is wide enough
for the diffusion radius, and the named workloads carry their sizes."""
import math

import numpy as np
import pytest

import dginputs


def _pair_clearance(d):
    """Smallest centre distance minus the sum of radii over all pairs
    (periodic minimum image); +inf for fewer than two disks."""
    if d.n < 2:
        return math.inf
    dx = d.cx[:, None] - d.cx[None, :]
    dy = d.cy[:, None] - d.cy[None, :]
    dx -= d.L * np.round(dx / d.L)
    dy -= d.L * np.round(dy / d.L)
    dist = np.sqrt(dx * dx + dy * dy)
    gap = dist - (d.r[:, None] + d.r[None, :])
    gap[np.arange(d.n), np.arange(d.n)] = math.inf
    return float(gap.min())


@pytest.mark.parametrize("seed,L,shape,scale,kw", [
    (7, 6.0, 2.0, 0.6, dict(n=10, min_gap=0.1)),           # under 3 cells: all-pairs checks
    (0, 10.0, 2.0, 0.4, dict(n=12, min_gap=0.1)),          # the 10 um cell workload
    (1, 40.0, 2.0, 0.5, dict(packing=0.55)),                # cell lists, no gap
    (2, 30.0, 1.5, 0.5, dict(packing=0.45, min_gap=0.05)),  # cell lists with a gap
])
def test_disks_never_overlap(seed, L, shape, scale, kw):
    d = dginputs.gamma_disks(seed, L, shape, scale, **kw)
    assert d.n > 0
    assert _pair_clearance(d) >= kw.get("min_gap", 0.0) - 1e-12
    assert np.all((d.cx >= 0) & (d.cx < L) & (d.cy >= 0) & (d.cy < L))
    # largest first, and the reported packing is the placed disks' area
    assert np.all(np.diff(d.r) <= 0)
    assert d.packing == pytest.approx(np.sum(np.pi * d.r ** 2) / L ** 2, rel=1e-12)
    # radii are drawn until their area reaches the target, so the placed area
    # exceeds it by at most the last drawn disk, no larger than the largest
    assert d.packing <= d.target_packing + np.pi * d.r[0] ** 2 / L ** 2 + 1e-12


def test_same_seed_same_substrate_and_start_points():
    a = dginputs.workload_small(3)
    b = dginputs.workload_small(3)
    c = dginputs.workload_small(4)
    for f in ("cx", "cy", "r"):
        assert np.array_equal(getattr(a.disks, f), getattr(b.disks, f))
    assert np.array_equal(a.sources, b.sources)
    assert not np.array_equal(a.disks.r, c.disks.r)


def test_radii_follow_the_gamma_law():
    """A sparse cell places every drawn radius, so the placed radii are the
    Gamma(shape, scale) sample itself: mean shape*scale and variance
    shape*scale^2 within a few standard errors."""
    shape, scale, n = 2.0, 0.4, 4000
    d = dginputs.gamma_disks(5, 400.0, shape, scale, n=n, batch=16)
    assert d.n == n
    mean, var = shape * scale, shape * scale ** 2
    assert abs(d.r.mean() - mean) < 4 * math.sqrt(var / n)
    # variance of the sample variance of a Gamma law: (mu4 - var^2) / n with
    # mu4 = 3 shape (shape + 2) scale^4
    mu4 = 3 * shape * (shape + 2) * scale ** 4
    assert abs(d.r.var() - var) < 4 * math.sqrt((mu4 - var ** 2) / n)


def test_packing_target_is_reached_when_it_fits():
    d = dginputs.gamma_disks(7, 40.0, 2.0, 0.5, packing=0.5)
    assert d.packing == pytest.approx(d.target_packing, abs=0.02)


def test_start_points_in_the_box_and_clear_of_disks():
    d = dginputs.gamma_disks(11, 20.0, 2.0, 0.5, packing=0.5, min_gap=0.05)
    margin = 20.0 / 128
    src = dginputs.sample_sources(12, d, 300, 2.0, 18.0, margin)
    assert src.shape == (300, 2)
    assert np.all((src >= 2.0) & (src < 18.0))
    dx = src[:, 0:1] - d.cx[None, :]
    dy = src[:, 1:2] - d.cy[None, :]
    dx -= d.L * np.round(dx / d.L)
    dy -= d.L * np.round(dy / d.L)
    assert np.all(np.sqrt(dx * dx + dy * dy) >= d.r[None, :] + margin - 1e-12)
    # the element that holds a start point has its centre outside every disk
    h = margin
    ecx = (np.floor(src[:, 0] / h) + 0.5) * h
    ecy = (np.floor(src[:, 1] / h) + 0.5) * h
    ex = ecx[:, None] - d.cx[None, :]
    ey = ecy[:, None] - d.cy[None, :]
    ex -= d.L * np.round(ex / d.L)
    ey -= d.L * np.round(ey / d.L)
    assert np.all(ex * ex + ey * ey >= d.r[None, :] ** 2)


@pytest.mark.parametrize("L,dmax,expect", [
    (10.0, 5.0, 7),    # R = 26.9 um: 2 ceil(R / L) + 1
    (40.0, 50.0, 7),   # R = 84.9 um
    (40.0, 5.0, 3),    # R = 26.9 um, L < 3R: 2 ceil(R / L) + 1 = 3
    (200.0, 5.0, 1),   # L >= 3R: one cell
])
def test_window_covers_the_diffusion_radius(L, dmax, expect):
    sigma0, D = 0.2, 2.0
    R = 6.0 * math.sqrt(sigma0 ** 2 + 2 * D * dmax)
    t = dginputs.window_tiles(L, sigma0, D, dmax)
    assert t == expect and t % 2 == 1
    lo, hi = dginputs.source_box(L, t, sigma0, D, dmax)
    # every start point is at least R from the absorbing edge of the window,
    # which spans [-half, L + half) in central-cell coordinates
    half = (t // 2) * L
    assert lo + half >= R - 1e-9 and (L + half) - hi >= R - 1e-9


def test_named_workloads_carry_their_sizes():
    w = dginputs.workload_small(0)
    assert (w.p, w.L, w.n_cell, w.tiles, w.D, w.sigma0, w.deltas) == \
        (2, 10.0, 32, 7, 2.0, 0.2, [5.0])
    assert w.sources.shape == (1, 2) and w.disks.n <= 12
    assert _pair_clearance(w.disks) >= 0.1 - 1e-12
    w = dginputs.workload_cell40(0, m=8)
    assert (w.p, w.L, w.n_cell, w.tiles) == (3, 40.0, 256, 7)
    assert w.deltas == [5.0, 10.0, 20.0, 50.0] and w.sources.shape == (8, 2)
    assert 0.5 <= w.disks.target_packing <= 0.7
    assert w.n_window == 1792 and w.h == pytest.approx(0.15625)
    # start points in the central cell of the window
    assert np.all((w.sources >= 0) & (w.sources < w.L))
    fd = dginputs.free_diffusion_paper()
    assert 2 * fd["T"] * fd["D"] == pytest.approx(32.4)


def test_start_points_without_room_raise_instead_of_looping():
    """A box covered by disks (grown by the margin) has no admissible start
    point: the rejection sampler gives up after a bounded number of
    candidates.  The surrogate's cell 2268 is such a draw (its last disk
    overshoots the packing target); its slot is filled by a redraw."""
    import time
    full = dginputs.Disks(np.array([0.5]), np.array([0.5]), np.array([2.0]), 1.0, 0.9, 0.9)
    t0 = time.perf_counter()
    with pytest.raises(dginputs.NoRoomForSources):
        dginputs.sample_sources(1, full, 4, 0.0, 1.0, margin=0.1, max_batches=50)
    assert time.perf_counter() - t0 < 30
    w = dginputs.workload_surrogate_member(2268)
    assert w.meta["seed"] == 2268 and w.meta["draw_seed"] != 2268
    assert w.sources.shape == (16, 2)
