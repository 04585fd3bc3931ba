"""Plain FP64 CPU oracle of the DG diffusion path and the covariance Sigma.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg may use this package; the product path never does.  It
shares no code with the CUDA library and does not import it.

Paper: Cervantes et al., "A GPU implementation of the Discontinuous Galerkin
method for simulation of diffusion in brain tissue", arXiv 1907.06191.

  * ``dgoracle.c`` holds the element loops (Eqs. 6-8, fluxes of Sec. 3.2,
    SSP-RK3, nodal-quadrature moments of Sec. 4.1, the disk mask);
  * this module binds it and adds the Sigma scheme of Sec. 4.1
    (normalise each density, mix with equal weights, moment-matched
    Gaussian) in numpy;
  * ``weakform.py`` assembles the same operator a second, independent way
    (dense matrices of the weak form of Eq. 7) for tiny meshes.

Parity status: every function here is pinned by the CPU tests (closed
forms, invariants, brute force) except the disk-geometry Sigma values, whose
parity is pinned only through those invariants (there is no closed form for
a disordered substrate).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libdgoracle.so")
_SRC = os.path.join(_HERE, "dgoracle.c")
_lib = None

RK3_REAL_LIMIT = None  # filled lazily by rk3_real_limit()


def build(force: bool = False) -> str:
    """Compile dgoracle.c into a shared library (gcc, OpenMP, no FP
    contraction so that mask decisions round like plain C)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp",
           "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_gll.argtypes = [ctypes.c_int, dp, dp, dp]
        lib.orc_apply_L.argtypes = [ctypes.c_void_p, dp, dp]
        lib.orc_rk3.argtypes = [ctypes.c_void_p, dp, ctypes.c_int, ctypes.c_double]
        lib.orc_rk3_adv.argtypes = [ctypes.c_void_p, dp, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_void_p]
        lib.orc_init_gaussian.argtypes = [ctypes.c_void_p, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, dp]
        lib.orc_moments.argtypes = [ctypes.c_void_p, dp, ctypes.c_double,
                                    ctypes.c_double, dp]
        lib.orc_mask_disks.argtypes = [ctypes.c_double, ctypes.c_int, dp, dp, dp,
                                       ctypes.c_int, ctypes.c_void_p]
        lib.orc_mask_disks.restype = None
        lib.orc_power_rho.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64]
        lib.orc_power_rho.restype = ctypes.c_double
        lib.orc_threads.argtypes = []
        lib.orc_threads.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = None
        _lib = lib
    return _lib


class _CMesh(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("h", ctypes.c_double), ("x0", ctypes.c_double),
                ("y0", ctypes.c_double), ("k0", ctypes.c_double),
                ("eta", ctypes.c_double), ("wall_mode", ctypes.c_int),
                ("periodic", ctypes.c_int), ("active", ctypes.c_void_p)]


@dataclass
class Mesh:
    """Uniform grid of nx*ny square elements of side h, lower-left corner
    (x0, y0); ``active[ey, ex]`` marks extracellular elements."""
    p: int
    active: np.ndarray  # uint8 [ny, nx]
    h: float
    x0: float = 0.0
    y0: float = 0.0
    k0: float = 1.0
    eta: float = 0.0
    wall_mode: int = 0   # 0: axon elements removed, 1: kept with k = 0
    periodic: bool = False

    def __post_init__(self):
        self.active = np.ascontiguousarray(self.active, dtype=np.uint8)

    @property
    def n(self) -> int:
        return self.p + 1

    @property
    def ny(self) -> int:
        return int(self.active.shape[0])

    @property
    def nx(self) -> int:
        return int(self.active.shape[1])

    @property
    def field_shape(self):
        return (self.ny, self.nx, self.n, self.n)  # [ey, ex, j, i]

    def c(self) -> _CMesh:
        self._keep = self.active
        return _CMesh(self.p, self.nx, self.ny, self.h, self.x0, self.y0,
                      self.k0, self.eta, self.wall_mode, int(self.periodic),
                      self.active.ctypes.data)

    def zeros(self):
        return np.zeros(self.field_shape)


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def threads() -> int:
    """Threads of the OpenMP team the oracle's element loops run on."""
    return int(_load().orc_threads())


def set_threads(n: int) -> None:
    """Run the oracle's element loops on n threads from now on."""
    _load().orc_set_threads(int(n))


def gll(p: int):
    """GLL nodes, weights and differentiation matrix D[i, m] = l_m'(xi_i)."""
    n = p + 1
    xi, w, D = np.zeros(n), np.zeros(n), np.zeros((n, n))
    if _load().orc_gll(p, _dp(xi), _dp(w), _dp(D)) != 0:
        raise ValueError("p out of range")
    return xi, w, D


def apply_L(mesh: Mesh, u: np.ndarray) -> np.ndarray:
    """L u (Eq. 7 with the Sec. 3.2 fluxes) for one density."""
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(mesh.field_shape)
    out = np.empty_like(u)
    cm = mesh.c()
    if _load().orc_apply_L(ctypes.byref(cm), _dp(u), _dp(out)) != 0:
        raise RuntimeError("orc_apply_L failed")
    return out


def rk3(mesh: Mesh, u: np.ndarray, nsteps: int, dt: float, advance=None) -> np.ndarray:
    """nsteps SSP-RK3 steps of size dt; returns a new array.  advance: None
    (every element) or a [ny, nx] mask of the elements that advance; the
    others keep their values."""
    v = np.array(u, dtype=np.float64, order="C").reshape(mesh.field_shape)
    cm = mesh.c()
    if advance is None:
        rc = _load().orc_rk3(ctypes.byref(cm), _dp(v), int(nsteps), float(dt))
    else:
        adv = np.ascontiguousarray(advance, dtype=np.uint8)
        assert adv.shape == (mesh.ny, mesh.nx)
        rc = _load().orc_rk3_adv(ctypes.byref(cm), _dp(v), int(nsteps), float(dt),
                                 adv.ctypes.data)
    if rc != 0:
        raise RuntimeError("orc_rk3 failed")
    return v


def window_d2(mesh: Mesh, box) -> np.ndarray:
    """Squared distance [ny, nx] from each element centre to the box
    (x_lo, x_hi, y_lo, y_hi) spanned by the start points, in FP64 with the
    operations in this order (the library's growing window takes the same
    decisions from the same values)."""
    x = mesh.x0 + (np.arange(mesh.nx) + 0.5) * mesh.h
    y = mesh.y0 + (np.arange(mesh.ny) + 0.5) * mesh.h
    dx = np.maximum(np.maximum(box[0] - x, x - box[1]), 0.0)
    dy = np.maximum(np.maximum(box[2] - y, y - box[3]), 0.0)
    return (dx * dx)[None, :] + (dy * dy)[:, None]


def rk3_growing(mesh: Mesh, u: np.ndarray, nsteps: int, dt: float, box, r_factor: float,
                sigma0: float, t0: float = 0.0, group: int = 64) -> np.ndarray:
    """RK3 on a window that grows with the density (Sec. 4.1 window of
    radius R = r_factor sqrt(sigma0^2 + 2 k0 t) around the start-point box).
    Steps go in groups of ``group``; in each group an element advances when
    its centre lies within R of the box at the group's end time, the rest
    keep their values."""
    d2 = window_d2(mesh, box)
    v = np.array(u, dtype=np.float64)
    done = 0
    while done < nsteps:
        k = min(group, nsteps - done)
        t_end = t0 + (done + k) * dt
        r2 = r_factor * r_factor * (sigma0 * sigma0 + 2.0 * mesh.k0 * t_end)
        adv = (mesh.active != 0) & (d2 <= r2)
        v = rk3(mesh, v, k, dt, advance=adv)
        done += k
    return v


def init_gaussian(mesh: Mesh, xs: float, ys: float, sigma0: float) -> np.ndarray:
    u = mesh.zeros()
    cm = mesh.c()
    if _load().orc_init_gaussian(ctypes.byref(cm), xs, ys, sigma0, _dp(u)) != 0:
        raise RuntimeError("orc_init_gaussian failed")
    return u


def moments(mesh: Mesh, u: np.ndarray, xs: float, ys: float) -> np.ndarray:
    """{M0, Mx, My, Mxx, Mxy, Myy} about (xs, ys) by GLL nodal quadrature."""
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(mesh.field_shape)
    out = np.zeros(6)
    cm = mesh.c()
    if _load().orc_moments(ctypes.byref(cm), _dp(u), xs, ys, _dp(out)) != 0:
        raise RuntimeError("orc_moments failed")
    return out


def mask_disks(L: float, n_cell: int, cx, cy, r) -> np.ndarray:
    """Element mask [n_cell, n_cell] of the periodic cell: 1 where the element
    centre lies outside every disk (squared distance >= r^2)."""
    cx = np.ascontiguousarray(cx, dtype=np.float64)
    cy = np.ascontiguousarray(cy, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    out = np.zeros((n_cell, n_cell), dtype=np.uint8)
    _load().orc_mask_disks(float(L), int(n_cell), _dp(cx), _dp(cy), _dp(r),
                           int(r.size), out.ctypes.data)
    return out


def window_mask(cell: np.ndarray, tiles: int) -> np.ndarray:
    """Tile the periodic cell mask into a tiles x tiles window."""
    return np.ascontiguousarray(np.tile(cell, (tiles, tiles)))


def power_rho(mesh: Mesh, iters: int = 200, seed: int = 12345) -> float:
    cm = mesh.c()
    r = _load().orc_power_rho(ctypes.byref(cm), int(iters), int(seed))
    if r < 0:
        raise RuntimeError("orc_power_rho failed")
    return float(r)


def rk3_real_limit() -> float:
    """Largest x with |1 - x + x^2/2 - x^3/6| <= 1 on [0, x]: the step bound
    dt * rho(L) of SSP-RK3 for a symmetric negative semidefinite L.  It is
    the real root of 1 + z + z^2/2 + z^3/6 = -1."""
    global RK3_REAL_LIMIT
    if RK3_REAL_LIMIT is None:
        roots = np.roots([1.0 / 6.0, 0.5, 1.0, 2.0])
        real = [float(z.real) for z in roots if abs(z.imag) < 1e-12]
        RK3_REAL_LIMIT = -min(real)
    return RK3_REAL_LIMIT


def step_plan(rho: float, delta: float, cfl_safety: float = 0.9):
    """Equal steps to reach delta: N = ceil(delta / dt_max), dt = delta / N,
    dt_max = cfl_safety * (RK3 real-axis limit) / rho."""
    dt_max = cfl_safety * rk3_real_limit() / rho
    nsteps = max(1, int(math.ceil(delta / dt_max - 1e-12)))
    return nsteps, delta / nsteps


def aggregate(mom: np.ndarray, mom0: np.ndarray | None = None):
    """The Sigma scheme of Sec. 4.1 on raw moments [m, 6] about each start
    point.  Each density is normalised by its mass (centred at its start
    point), the normalised densities are mixed with weights 1/m, and the
    moment-matched Gaussian of the mixture gives
        mu = mean_s (Mx, My)/M0,
        Sigma_mix = mean_s (Mxx, Mxy, Myy)/M0 - mu mu^T.
    With ``mom0`` (moments of the start densities) the start width is
    removed: Sigma = Sigma_mix(t) - Sigma_mix(0).  Returns
    (sigma3 = [Sxx, Sxy, Syy], mu2, mass[m])."""
    def mix(mm):
        mm = np.asarray(mm, dtype=np.float64).reshape(-1, 6)
        m0 = mm[:, 0]
        mu = np.array([np.mean(mm[:, 1] / m0), np.mean(mm[:, 2] / m0)])
        s = np.array([np.mean(mm[:, 3] / m0), np.mean(mm[:, 4] / m0),
                      np.mean(mm[:, 5] / m0)])
        s = s - np.array([mu[0] * mu[0], mu[0] * mu[1], mu[1] * mu[1]])
        return s, mu, m0.copy()
    s, mu, m0 = mix(mom)
    if mom0 is not None:
        s0, _, _ = mix(mom0)
        s = s - s0
    return s, mu, m0


def mixture_fit(mom: np.ndarray):
    """Moment-matched Gaussian of the mixture (Sec. 4.1) without removing the
    start width: (mu [2], Sigma_mix [2, 2])."""
    mm = np.asarray(mom, dtype=np.float64).reshape(-1, 6)
    m0 = mm[:, 0]
    mu = np.array([np.mean(mm[:, 1] / m0), np.mean(mm[:, 2] / m0)])
    S = np.array([[np.mean(mm[:, 3] / m0), np.mean(mm[:, 4] / m0)],
                  [np.mean(mm[:, 4] / m0), np.mean(mm[:, 5] / m0)]])
    return mu, S - np.outer(mu, mu)


def ls_residual(mesh: Mesh, fields, sources, mom) -> float:
    """Least-squares residual of the Gaussian fit (Sec. 4.2): the sum over
    nodes of [f(x; Sigma) - u_ij]^2, f the fitted bivariate Gaussian density.
    For a mixture of densities centred at their own start points, each
    normalised density u_s / M0_s is compared at its own nodes with
    f(x - x_s - mu; Sigma_mix), and the sums are averaged over densities."""
    mu, S = mixture_fit(mom)
    Si = np.linalg.inv(S)
    norm = 1.0 / (2.0 * math.pi * math.sqrt(np.linalg.det(S)))
    X, Y = node_coords(mesh)
    act = np.repeat(np.repeat(mesh.active[:, :, None, None], mesh.n, 2), mesh.n, 3).astype(bool)
    total = 0.0
    mm = np.asarray(mom).reshape(-1, 6)
    for f, (xs, ys), q in zip(fields, np.asarray(sources).reshape(-1, 2), mm):
        dx = X - xs - mu[0]
        dy = Y - ys - mu[1]
        quad = Si[0, 0] * dx * dx + 2 * Si[0, 1] * dx * dy + Si[1, 1] * dy * dy
        g = norm * np.exp(-0.5 * quad)
        r = (g - np.asarray(f).reshape(mesh.field_shape) / q[0])[act]
        total += float(np.sum(r * r))
    return total / len(mm)


def dense_operator(mesh: Mesh) -> np.ndarray:
    """Matrix of L in the dense node ordering, from unit vectors (tiny meshes)."""
    N = int(np.prod(mesh.field_shape))
    A = np.zeros((N, N))
    e = np.zeros(N)
    for k in range(N):
        e[k] = 1.0
        A[:, k] = apply_L(mesh, e).ravel()
        e[k] = 0.0
    return A


def node_weights(mesh: Mesh) -> np.ndarray:
    """GLL quadrature weight J^2 w_i w_j of every node, dense ordering."""
    _, w, _ = gll(mesh.p)
    J = 0.5 * mesh.h
    wt = (J * J) * np.outer(w, w)  # [j, i]
    return np.broadcast_to(wt, mesh.field_shape).copy()


def node_coords(mesh: Mesh):
    """Physical x and y of every node, dense ordering [ey, ex, j, i]."""
    xi, _, _ = gll(mesh.p)
    ex = np.arange(mesh.nx)
    ey = np.arange(mesh.ny)
    x = mesh.x0 + (ex[None, :, None, None] + 0.5) * mesh.h + 0.5 * mesh.h * xi[None, None, None, :]
    y = mesh.y0 + (ey[:, None, None, None] + 0.5) * mesh.h + 0.5 * mesh.h * xi[None, None, :, None]
    return (np.broadcast_to(x, mesh.field_shape).copy(),
            np.broadcast_to(y, mesh.field_shape).copy())


def solve(mesh: Mesh, sources: np.ndarray, sigma0: float, deltas,
          *, nsteps=None, dt=None, rho=None, cfl_safety: float = 0.9):
    """Full Sigma solve: one density per start point, propagated through the
    diffusion times in ``deltas`` (ascending) with equal steps per interval.
    Either give (nsteps, dt) lists per interval, or let the power iteration
    pick them.  Returns dict with per-delta raw moments, Sigma, mu, mass."""
    sources = np.asarray(sources, dtype=np.float64).reshape(-1, 2)
    deltas = list(deltas)
    if nsteps is None:
        if rho is None:
            rho = power_rho(mesh)
        plans, t = [], 0.0
        for d in deltas:
            plans.append(step_plan(rho, d - t, cfl_safety))
            t = d
    else:
        plans = list(zip(nsteps, dt))
    fields = [init_gaussian(mesh, xs, ys, sigma0) for xs, ys in sources]
    mom0 = np.array([moments(mesh, f, xs, ys) for f, (xs, ys) in zip(fields, sources)])
    out = {"mom0": mom0, "plans": plans, "moments": [], "sigma": [], "mu": [],
           "mass": []}
    for (ns, dts) in plans:
        fields = [rk3(mesh, f, ns, dts) for f in fields]
        mom = np.array([moments(mesh, f, xs, ys) for f, (xs, ys) in zip(fields, sources)])
        s, mu, m0 = aggregate(mom, mom0)
        out["moments"].append(mom)
        out["sigma"].append(s)
        out["mu"].append(mu)
        out["mass"].append(m0)
    out["fields"] = fields
    return out
