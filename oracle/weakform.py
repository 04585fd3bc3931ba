"""Independent dense assembly of the DG operator from the weak form of Eq. 7.

TEST INFRASTRUCTURE ONLY (tiny meshes).  This is a second construction of
the operator that ``dgoracle.c`` evaluates in strong form.  It shares no
code with it: the GLL nodes come from numpy's Legendre roots, the Lagrange
basis is built from a Vandermonde solve, and every integral of the weak form
is evaluated by GLL quadrature with the basis functions evaluated at the
quadrature points (nothing assumes the Kronecker-delta property), the
surface integrals with the fluxes of Sec. 3.2 substituted for u n and
k q . n.

For an element K (side h, J = h/2) and test functions v (vector) and w:
    (q, v)_K   = <h_u, v>_dK - (u, div v)_K                   (Eq. 7, line 1)
    (u_t, w)_K = <h_q, w>_dK - (k q, grad w)_K                (Eq. 7, line 2)
h_u = (u^- + u^+)/2 n^-, h_q = k_h (q^- + q^+)/2 . n^- - tau (u^- - u^+),
k_h = 2 k^- k^+ / (k^- + k^+), tau = eta k_h (p+1)^2 / h.  Walls of removed
axon elements: h_u = u^- n, h_q = 0.  Domain edge (Eq. 4): h_u = 0,
h_q = k q^- . n - eta k (p+1)^2/h u^-.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly

__all__ = ["gll_numpy", "assemble"]


def gll_numpy(p: int):
    """GLL nodes (endpoints and roots of P_p') and weights 2/(p(p+1)P_p^2)."""
    cp = np.zeros(p + 1)
    cp[p] = 1.0
    inner = np.sort(np.real(npleg.legroots(npleg.legder(cp)))) if p > 1 else np.array([])
    x = np.concatenate([[-1.0], inner, [1.0]])
    Pp = npleg.legval(x, cp)
    w = 2.0 / (p * (p + 1) * Pp ** 2)
    return x, w


def _lagrange(nodes):
    """Monomial coefficients of the Lagrange basis on ``nodes`` and of their
    derivatives."""
    n = nodes.size
    V = np.vander(nodes, n, increasing=True)        # V[i, k] = x_i^k
    C = np.linalg.solve(V, np.eye(n))                # column m: l_m coefficients
    coeffs = [C[:, m] for m in range(n)]
    dcoeffs = [nppoly.polyder(c) for c in coeffs]
    return coeffs, dcoeffs


def assemble(mesh) -> np.ndarray:
    """Dense matrix of u -> u_t, node ordering [ey, ex, j, i] (as the oracle).

    ``mesh`` is an ``oracle.Mesh`` (only its plain fields are read)."""
    p, n = mesh.p, mesh.p + 1
    nx, ny, h = mesh.nx, mesh.ny, mesh.h
    J = 0.5 * h
    act = np.asarray(mesh.active, dtype=bool)
    mode_a = mesh.wall_mode == 1
    in_mesh = np.ones_like(act) if mode_a else act
    kval = np.where(act, mesh.k0, 0.0)
    xq, wq = gll_numpy(p)
    coeffs, dcoeffs = _lagrange(xq)

    def ell(x):  # basis values at x: [n]
        return np.array([nppoly.polyval(x, c) for c in coeffs])

    def dell(x):
        return np.array([nppoly.polyval(x, c) for c in dcoeffs])

    Np = n * n
    Ne = nx * ny
    N = Ne * Np

    def gidx(e, a, b):  # node (a along x, b along y) of element e
        return e * Np + b * n + a

    def phi(xr, yr):  # tensor basis at reference point, ordered b*n + a
        lx, ly = ell(xr), ell(yr)
        return np.outer(ly, lx).ravel()

    def dphi(xr, yr):  # reference gradients of the basis functions
        lx, ly, dlx, dly = ell(xr), ell(yr), dell(xr), dell(yr)
        return np.outer(ly, dlx).ravel(), np.outer(dly, lx).ravel()

    # local mass (quadrature at the GLL points) and volume integrals
    Mloc = np.zeros((Np, Np))
    Kx = np.zeros((Np, Np))   # (u, d/dx v): rows test, cols trial
    Ky = np.zeros((Np, Np))
    for qi in range(n):
        for qj in range(n):
            wt = J * J * wq[qi] * wq[qj]
            ph = phi(xq[qi], xq[qj])
            gx, gy = dphi(xq[qi], xq[qj])
            Mloc += wt * np.outer(ph, ph)
            Kx += wt * np.outer(gx / J, ph)
            Ky += wt * np.outer(gy / J, ph)
    Minv_loc = np.linalg.inv(Mloc)

    # face geometry: reference point of face node t in the element, outward
    # normal, and the direction of the neighbour
    def face_pts(d, t):
        s = xq[t]
        return {0: (1.0, s), 1: (-1.0, s), 2: (s, 1.0), 3: (s, -1.0)}[d]
    normals = {0: (1.0, 0.0), 1: (-1.0, 0.0), 2: (0.0, 1.0), 3: (0.0, -1.0)}
    opp = {0: 1, 1: 0, 2: 3, 3: 2}
    step = {0: (1, 0), 1: (-1, 0), 2: (0, 1), 3: (0, -1)}

    def neighbour(ex, ey, d):
        qx, qy = ex + step[d][0], ey + step[d][1]
        if not (0 <= qx < nx and 0 <= qy < ny):
            if not mesh.periodic:
                return "edge", -1
            qx %= nx
            qy %= ny
        e2 = qy * nx + qx
        if not in_mesh.ravel()[e2]:
            return "wall", e2
        return "interior", e2

    # gradient: M q_c = G_c u (c = x, y)
    Gx = np.zeros((N, N))
    Gy = np.zeros((N, N))
    # divergence: M u_t = Bx qx + By qy + Bu u
    Bx = np.zeros((N, N))
    By = np.zeros((N, N))
    Bu = np.zeros((N, N))
    pen = mesh.eta * n * n / h

    for ey in range(ny):
        for ex in range(nx):
            e = ey * nx + ex
            if not in_mesh.ravel()[e]:
                continue
            k = kval.ravel()[e]
            rows = np.arange(e * Np, (e + 1) * Np)
            Gx[np.ix_(rows, rows)] -= Kx
            Gy[np.ix_(rows, rows)] -= Ky
            Bx[np.ix_(rows, rows)] -= k * Kx
            By[np.ix_(rows, rows)] -= k * Ky
            for d in range(4):
                kind, e2 = neighbour(ex, ey, d)
                nxv, nyv = normals[d]
                for t in range(n):
                    wf = J * wq[t]
                    xr, yr = face_pts(d, t)
                    test = phi(xr, yr)           # test functions at the point
                    tr_m = phi(xr, yr)           # trace of own trial functions
                    # coefficient vectors over global DoFs
                    um = np.zeros(N)
                    um[rows] = tr_m
                    up = np.zeros(N)
                    if kind == "interior":
                        xr2, yr2 = face_pts(opp[d], t)
                        up[e2 * Np:(e2 + 1) * Np] = phi(xr2, yr2)
                        uhat = 0.5 * (um + up)
                    elif kind == "wall":
                        uhat = um
                    else:
                        uhat = np.zeros(N)
                    Gx[rows, :] += wf * nxv * np.outer(test, uhat)
                    Gy[rows, :] += wf * nyv * np.outer(test, uhat)
                    # q-flux: h_q = kh (q^- + q^+)/2 . n - tau (u^- - u^+)
                    if kind == "interior":
                        k2 = kval.ravel()[e2]
                        kh = 2.0 * k * k2 / (k + k2) if (k + k2) > 0 else 0.0
                        qavg = 0.5 * (um + up)  # same trace map for q components
                        Bx[rows, :] += wf * kh * nxv * np.outer(test, qavg)
                        By[rows, :] += wf * kh * nyv * np.outer(test, qavg)
                        Bu[rows, :] += -wf * pen * kh * np.outer(test, um - up)
                    elif kind == "edge":
                        Bx[rows, :] += wf * k * nxv * np.outer(test, um)
                        By[rows, :] += wf * k * nyv * np.outer(test, um)
                        Bu[rows, :] += -wf * pen * k * np.outer(test, um)
                    # walls: h_q = 0, nothing to add

    Minv = np.zeros((N, N))
    for e in range(Ne):
        sl = slice(e * Np, (e + 1) * Np)
        if in_mesh.ravel()[e]:
            Minv[sl, sl] = Minv_loc
    Qx = Minv @ Gx
    Qy = Minv @ Gy
    return Minv @ (Bx @ Qx + By @ Qy + Bu)
