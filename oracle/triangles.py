"""FP64 oracle of the paper's own element: every square pixel split by its
diagonal into two triangles (Sec. 3.3) with a Lagrange basis of order p on
each triangle (Eq. 8, "as in the Finite Element Method with lagrangian
interpolation"), the weak form of Eq. 7 integrated exactly, and the fluxes of
Sec. 3.2 (central h_u, harmonic-mean h_q).

TEST INFRASTRUCTURE ONLY: only the test suite, the smoke check and the
benchmark's CPU baseline use it.  It shares nothing with the CUDA path.

Readings (the paper is silent on them):
  - the diagonal runs from the pixel's lower-left to its upper-right corner:
    triangle A (lower right) has vertices (x0, y0), (x1, y0), (x1, y1),
    triangle B (upper left) (x0, y0), (x1, y1), (x0, y1);
  - Lagrange nodes equispaced on the triangle (the finite-element P_p nodes),
    p = 1..3 ("p <= 3 suffices", Sec. 3.1 remark);
  - all integrals of Eq. 7 exact: mass, derivative and face matrices of the
    polynomials, so the mass matrix is full, not diagonal;
  - walls, outer edge and the paper's kept-axon mode as for the square
    elements: removed axon pixels give u_hat = u^- and h_q = 0; mode 1 keeps
    them at u = 0 with k = 0 (u_hat = u^-/2, h_q = 0); the outer edge is
    Eq. 4 (u_hat = 0, h_q = k q^- . n); no penalty term.

Layout: u[ey, ex, tri, node], tri 0 = A, 1 = B; node k of a triangle is the
reference point (i/p, j/p), k running over j = 0..p, then i = 0..p - j.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from functools import lru_cache

import numpy as np

# reference triangle (r, s): vertices (0, 0), (1, 0), (0, 1); edges
# e0: (0,0)->(1,0), e1: (1,0)->(0,1), e2: (0,1)->(0,0)


def n_nodes(p: int) -> int:
    return (p + 1) * (p + 2) // 2


def ref_nodes(p: int) -> np.ndarray:
    """Equispaced Lagrange nodes [(r, s)] in the layout order."""
    return np.array([(i / p, j / p) for j in range(p + 1) for i in range(p + 1 - j)])


def _exps(p: int):
    return [(a, b) for a in range(p + 1) for b in range(p + 1 - a)]


def _mono_int(a: int, b: int) -> float:
    """Exact integral of r^a s^b over the reference triangle."""
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


def edge_nodes(p: int):
    """Node indices along each reference edge, in the edge's direction."""
    idx = {(round(r * p), round(s * p)): k for k, (r, s) in enumerate(ref_nodes(p))}
    e0 = [idx[(i, 0)] for i in range(p + 1)]
    e1 = [idx[(p - j, j)] for j in range(p + 1)]
    e2 = [idx[(0, p - j)] for j in range(p + 1)]
    return [e0, e1, e2]


@lru_cache(maxsize=None)
def ref_matrices(p: int):
    """Lagrange basis on the reference triangle and its exact integrals.

    Returns dict with
      C   [monomial, node]: N_k = sum_m C[m, k] r^a_m s^b_m
      M   [i, j] = int N_i N_j
      Sr  [i, j] = int N_i dN_j/dr,  Ss likewise
      E1  [t, u] = int_0^1 l_t l_u  (1D mass of the edge nodes, unit length)
      mono_w[(a, b)] [j] = int r^a s^b N_j   for a + b <= 2 + p (moments)
    """
    ex = _exps(p)
    X = ref_nodes(p)
    V = np.array([[r ** a * s ** b for (a, b) in ex] for (r, s) in X])
    C = np.linalg.inv(V)                 # columns: basis functions
    nm = len(ex)
    I = np.array([[_mono_int(a1 + a2, b1 + b2) for (a2, b2) in ex] for (a1, b1) in ex])
    M = C.T @ I @ C
    # d/dr of monomial m = a r^(a-1) s^b
    Dr = np.zeros((nm, nm))
    Ds = np.zeros((nm, nm))
    pos = {e: k for k, e in enumerate(ex)}
    for k, (a, b) in enumerate(ex):
        if a > 0:
            Dr[pos[(a - 1, b)], k] = a
        if b > 0:
            Ds[pos[(a, b - 1)], k] = b
    Sr = C.T @ I @ (Dr @ C)
    Ss = C.T @ I @ (Ds @ C)
    # 1D Lagrange on equispaced points of [0, 1]
    t = np.linspace(0.0, 1.0, p + 1)
    V1 = np.vander(t, p + 1, increasing=True)
    C1 = np.linalg.inv(V1)
    I1 = np.array([[1.0 / (a + b + 1) for b in range(p + 1)] for a in range(p + 1)])
    E1 = C1.T @ I1 @ C1
    mono_w = {}
    for a in range(3):
        for b in range(3 - a):
            mono_w[(a, b)] = np.array([sum(C[m, j] * _mono_int(a + am, b + bm)
                                           for m, (am, bm) in enumerate(ex)) for j in range(nm)])
    return dict(C=C, M=M, Sr=Sr, Ss=Ss, E1=E1, mono_w=mono_w, ex=ex)


# ---- the two triangles of a pixel of side h --------------------------------
# A: x = x0 + h (r + s), y = y0 + h s       (vertices (x0,y0), (x1,y0), (x1,y1))
# B: x = x0 + h r,       y = y0 + h (r + s) (vertices (x0,y0), (x1,y1), (x0,y1))
# inverse Jacobians (dr/dx, dr/dy, ds/dx, ds/dy) times h:
_INVJ = {0: (1.0, -1.0, 0.0, 1.0), 1: (1.0, 0.0, -1.0, 1.0)}
# outward unit normals and lengths (in units of h) of edges e0, e1, e2
_S2 = math.sqrt(0.5)
_EDGE = {0: [((0.0, -1.0), 1.0), ((1.0, 0.0), 1.0), ((-_S2, _S2), math.sqrt(2.0))],
         1: [((_S2, -_S2), math.sqrt(2.0)), ((0.0, 1.0), 1.0), ((-1.0, 0.0), 1.0)]}
# edge -> (neighbour pixel offset (dx, dy), neighbour triangle, neighbour edge)
_NEIGH = {0: [((0, -1), 1, 1), ((1, 0), 1, 2), ((0, 0), 1, 0)],
          1: [((0, 0), 0, 2), ((0, 1), 0, 0), ((-1, 0), 0, 1)]}


def node_xy(p: int, h: float, x0: float, y0: float, nx: int, ny: int):
    """Physical node coordinates X, Y [ny, nx, 2, Np]."""
    R = ref_nodes(p)
    ex = np.arange(nx)[None, :, None]
    ey = np.arange(ny)[:, None, None]
    X = np.empty((ny, nx, 2, len(R)))
    Y = np.empty_like(X)
    r, s = R[:, 0][None, None, :], R[:, 1][None, None, :]
    X[:, :, 0, :] = x0 + (ex + r + s) * h
    Y[:, :, 0, :] = y0 + (ey + s) * h
    X[:, :, 1, :] = x0 + (ex + r) * h
    Y[:, :, 1, :] = y0 + (ey + r + s) * h
    return X, Y


@dataclass
class TriMesh:
    p: int
    active: np.ndarray          # [ny, nx] pixels in the extracellular region
    h: float
    x0: float = 0.0
    y0: float = 0.0
    k0: float = 1.0
    wall_mode: int = 0           # 0: axon pixels removed, 1: kept with k = 0
    periodic: bool = False

    def __post_init__(self):
        self.active = np.asarray(self.active, dtype=np.uint8)

    @property
    def ny(self):
        return self.active.shape[0]

    @property
    def nx(self):
        return self.active.shape[1]

    @property
    def np_(self):
        return n_nodes(self.p)

    @property
    def shape(self):
        return (self.ny, self.nx, 2, self.np_)

    def zeros(self):
        return np.zeros(self.shape)


def _neighbour(mesh: TriMesh, arr, d):
    """arr[ey + dy, ex + dx] for every pixel, with a validity mask ([ny, nx])
    and an 'outside the domain' mask."""
    dx, dy = d
    ny, nx = mesh.ny, mesh.nx
    ey = np.arange(ny)[:, None] + dy
    ex = np.arange(nx)[None, :] + dx
    out = (ey < 0) | (ey >= ny) | (ex < 0) | (ex >= nx)
    if mesh.periodic:
        ey, ex = ey % ny, ex % nx
        out = np.zeros((ny, nx), bool)
    eyc = np.clip(ey, 0, ny - 1) * np.ones((1, nx), int)
    exc = np.clip(ex, 0, nx - 1) * np.ones((ny, 1), int)
    return arr[eyc, exc], np.broadcast_to(out, (ny, nx))


def apply_L(mesh: TriMesh, u: np.ndarray) -> np.ndarray:
    """du/dt = L u of Eq. 7 (two passes: q = grad u with h_u, then the
    divergence of k q with h_q), for one density u[ny, nx, 2, Np]."""
    p, h, k0 = mesh.p, mesh.h, mesh.k0
    R = ref_matrices(p)
    Minv = np.linalg.inv(R["M"])
    E1 = R["E1"]
    EN = edge_nodes(p)
    u = np.asarray(u, dtype=np.float64).reshape(mesh.shape)
    act = mesh.active != 0
    in_mesh = np.ones_like(act) if mesh.wall_mode == 1 else act
    kpix = np.where(act, k0, 0.0)
    u = np.where(in_mesh[:, :, None, None], u, 0.0)

    def traces(field, tri, e):            # field [ny, nx, 2, Np] -> [ny, nx, p+1]
        return field[:, :, tri, EN[e]]

    def face_info(tri, e):
        d, nt, ne = _NEIGH[tri][e]
        kn, outside = _neighbour(mesh, kpix, d)
        inn, _ = _neighbour(mesh, in_mesh, d)
        return d, nt, ne, kn, outside, inn

    # pass 1: q = grad u, Eq. 7 first line
    q = np.zeros((2,) + mesh.shape)      # q[0] = q_x, q[1] = q_y
    for tri in (0, 1):
        rx, ry, sx, sy = (v / h for v in _INVJ[tri])
        uk = u[:, :, tri, :]
        # - int u dN_i/dx = -(rx Sr^T + sx Ss^T) u  (h^2 of dx cancels M_K = h^2 M)
        vol_x = -(uk @ (rx * R["Sr"] + sx * R["Ss"]))
        vol_y = -(uk @ (ry * R["Sr"] + sy * R["Ss"]))
        fx = np.zeros_like(uk)
        fy = np.zeros_like(uk)
        for e in range(3):
            (nxv, nyv), ln = _EDGE[tri][e]
            d, nt, ne, kn, outside, inn = face_info(tri, e)
            um = traces(u, tri, e)
            up_all, _ = _neighbour(mesh, u, d)
            up = up_all[:, :, nt, :][:, :, EN[ne]][:, :, ::-1]
            kme = kpix
            interior = (~outside) & (kn > 0)
            wall = (~outside) & (kn == 0)
            uhat = np.where(interior[:, :, None], 0.5 * (um + up), 0.0)
            if mesh.wall_mode == 1:
                uhat = np.where(wall[:, :, None], 0.5 * um, uhat)
            else:
                uhat = np.where(wall[:, :, None], um, uhat)
            uhat = np.where(outside[:, :, None], 0.0, uhat)
            uhat = np.where((kme > 0)[:, :, None], uhat, 0.0)
            g = (uhat @ E1.T) * (ln * h)            # int_e N_t uhat, edge nodes
            fx[:, :, EN[e]] += nxv * g
            fy[:, :, EN[e]] += nyv * g
        q[0, :, :, tri, :] = (vol_x + fx / (h * h)) @ Minv.T
        q[1, :, :, tri, :] = (vol_y + fy / (h * h)) @ Minv.T
    # pass 2: du/dt = div(k q), Eq. 7 second line
    out = np.zeros(mesh.shape)
    for tri in (0, 1):
        rx, ry, sx, sy = (v / h for v in _INVJ[tri])
        kk = kpix[:, :, None]
        qx, qy = q[0, :, :, tri, :], q[1, :, :, tri, :]
        vol = -kk * (qx @ (rx * R["Sr"] + sx * R["Ss"]) + qy @ (ry * R["Sr"] + sy * R["Ss"]))
        fs = np.zeros_like(qx)
        for e in range(3):
            (nxv, nyv), ln = _EDGE[tri][e]
            d, nt, ne, kn, outside, inn = face_info(tri, e)
            qn_m = traces(q[0], tri, e) * nxv + traces(q[1], tri, e) * nyv
            qx_all, _ = _neighbour(mesh, q[0], d)
            qy_all, _ = _neighbour(mesh, q[1], d)
            qn_p = (qx_all[:, :, nt, :][:, :, EN[ne]][:, :, ::-1] * nxv
                    + qy_all[:, :, nt, :][:, :, EN[ne]][:, :, ::-1] * nyv)
            km = kpix
            kh = np.where((km + kn) > 0, 2 * km * kn / np.where((km + kn) > 0, km + kn, 1), 0.0)
            flux = kh[:, :, None] * 0.5 * (qn_m + qn_p)
            flux = np.where(outside[:, :, None], km[:, :, None] * qn_m, flux)
            g = (flux @ E1.T) * (ln * h)
            fs[:, :, EN[e]] += g
        out[:, :, tri, :] = (vol + fs / (h * h)) @ Minv.T
    return np.where(in_mesh[:, :, None, None] & (kpix > 0)[:, :, None, None], out, 0.0)


def rk3(mesh: TriMesh, u: np.ndarray, nsteps: int, dt: float) -> np.ndarray:
    """SSP-RK3 (Shu-Osher form), as for the square elements."""
    u = np.array(u, dtype=np.float64).reshape(mesh.shape)
    for _ in range(nsteps):
        u1 = u + dt * apply_L(mesh, u)
        u2 = 0.75 * u + 0.25 * (u1 + dt * apply_L(mesh, u1))
        u = u / 3.0 + 2.0 * (u2 + dt * apply_L(mesh, u2)) / 3.0
    return u


def init_gaussian(mesh: TriMesh, xs: float, ys: float, sigma0: float) -> np.ndarray:
    """Normalised Gaussian interpolated at the nodes of mesh pixels (Sec. 4.1)."""
    X, Y = node_xy(mesh.p, mesh.h, mesh.x0, mesh.y0, mesh.nx, mesh.ny)
    g = np.exp(-((X - xs) ** 2 + (Y - ys) ** 2) / (2 * sigma0 ** 2)) / (2 * math.pi * sigma0 ** 2)
    return np.where((mesh.active != 0)[:, :, None, None], g, 0.0)


def moments(mesh: TriMesh, u: np.ndarray, xs: float, ys: float) -> np.ndarray:
    """M0, Mx, My, Mxx, Mxy, Myy of the density about (xs, ys), integrating
    the polynomial exactly on every triangle."""
    p, h = mesh.p, mesh.h
    W = ref_matrices(p)["mono_w"]
    u = np.asarray(u, dtype=np.float64).reshape(mesh.shape)
    ex = np.arange(mesh.nx)[None, :]
    ey = np.arange(mesh.ny)[:, None]
    cx = mesh.x0 + ex * h - xs           # pixel corner relative to the start point
    cy = mesh.y0 + ey * h - ys
    out = np.zeros(6)
    for tri in (0, 1):
        uk = u[:, :, tri, :]
        # local coordinates (x - x0, y - y0) = h (r + s, s) for A, h (r, r + s) for B
        def I(a, b):     # int (r)^a (s)^b u_h  over the reference, per pixel
            return uk @ W[(a, b)]
        i00 = I(0, 0)
        if tri == 0:
            lx = [I(1, 0) + I(0, 1)]                        # r + s
            ly = [I(0, 1)]                                  # s
            lxx = I(2, 0) + 2 * I(1, 1) + I(0, 2)
            lxy = I(1, 1) + I(0, 2)
            lyy = I(0, 2)
        else:
            lx = [I(1, 0)]
            ly = [I(1, 0) + I(0, 1)]
            lxx = I(2, 0)
            lxy = I(2, 0) + I(1, 1)
            lyy = I(2, 0) + 2 * I(1, 1) + I(0, 2)
        J = h * h
        m0 = J * i00
        mx_loc = J * h * lx[0]
        my_loc = J * h * ly[0]
        out[0] += m0.sum()
        out[1] += (cx * m0 + mx_loc).sum()
        out[2] += (cy * m0 + my_loc).sum()
        out[3] += (cx * cx * m0 + 2 * cx * mx_loc + J * h * h * lxx).sum()
        out[4] += (cx * cy * m0 + cx * my_loc + cy * mx_loc + J * h * h * lxy).sum()
        out[5] += (cy * cy * m0 + 2 * cy * my_loc + J * h * h * lyy).sum()
    return out


def dense_operator(mesh: TriMesh) -> np.ndarray:
    """L as a dense matrix over all nodes (columns = L applied to unit vectors)."""
    n = int(np.prod(mesh.shape))
    L = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        L[:, j] = apply_L(mesh, e).ravel()
    return L


def mass_matrix(mesh: TriMesh) -> np.ndarray:
    """Global (block-diagonal) mass matrix of the same node ordering."""
    M = ref_matrices(mesh.p)["M"] * mesh.h * mesh.h
    nblk = mesh.ny * mesh.nx * 2
    return np.kron(np.eye(nblk), M)


def power_rho(mesh: TriMesh, iters: int = 300, seed: int = 1) -> float:
    """Spectral radius of L by power iteration in the mass inner product."""
    rng = np.random.default_rng(seed)
    M = ref_matrices(mesh.p)["M"] * mesh.h * mesh.h
    v = rng.standard_normal(mesh.shape) * (mesh.active != 0)[:, :, None, None]
    def nrm(x):
        return math.sqrt(float(np.einsum('yxti,ij,yxtj->', x, M, x)))
    v /= nrm(v)
    lam = 0.0
    for _ in range(iters):
        w = apply_L(mesh, v)
        lam = nrm(w)
        v = w / lam
    return lam
