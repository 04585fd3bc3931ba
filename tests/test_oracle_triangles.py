"""Pins of the triangle oracle (oracle/triangles.py, the paper's Sec. 3.3
pixel triangles) against what the mathematics fixes: exact integration
identities of the reference matrices, symmetry and semidefiniteness of the
discrete operator, exactness on polynomials, free diffusion 2Tk = 32.4
(Sec. 4.2), mass conservation per connected component, the order of
convergence on a heat solution, and the x <-> y symmetry of the diagonal."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import triangles as T

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("p", [1, 2, 3])
def test_reference_matrices(p):
    R = T.ref_matrices(p)
    n = T.n_nodes(p)
    assert abs(R["M"].sum() - 0.5) < 1e-14                 # area of the reference triangle
    assert np.abs(R["Sr"].sum(axis=1)).max() < 1e-14       # derivative of a constant
    # integration by parts: Sr + Sr^T = boundary integral of N_i N_j n_r
    EN, E1 = T.edge_nodes(p), R["E1"]
    Br, Bs = np.zeros((n, n)), np.zeros((n, n))
    for e, (nr, ns, ln) in enumerate([(0.0, -1.0, 1.0), (math.sqrt(0.5), math.sqrt(0.5), math.sqrt(2.0)),
                                      (-1.0, 0.0, 1.0)]):
        Br[np.ix_(EN[e], EN[e])] += nr * ln * E1
        Bs[np.ix_(EN[e], EN[e])] += ns * ln * E1
    assert np.abs(R["Sr"] + R["Sr"].T - Br).max() < 1e-13
    assert np.abs(R["Ss"] + R["Ss"].T - Bs).max() < 1e-13
    # the basis interpolates: N_k(node j) = delta_kj
    X = T.ref_nodes(p)
    V = np.array([[r ** a * s ** b for (a, b) in R["ex"]] for (r, s) in X])
    assert np.abs(V @ R["C"] - np.eye(n)).max() < 1e-12
    # moments of a constant: int r^a s^b = a! b! / (a + b + 2)!
    for (a, b), w in R["mono_w"].items():
        assert abs(w.sum() - math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)) < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3])
def test_operator_symmetric_semidefinite_and_nullspace(p):
    act = np.ones((4, 5), np.uint8)
    act[1, 1:4] = 0
    act[2:4, 2] = 0                    # walls that split off a pocket
    act[3, 1] = 0
    m = T.TriMesh(p=p, active=act, h=0.5, k0=1.3, periodic=True)
    L = T.dense_operator(m)
    Mg = T.mass_matrix(m)
    keep = np.repeat(act.ravel() != 0, 2 * T.n_nodes(p))
    A = (Mg @ L)[np.ix_(keep, keep)]
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.max() < 1e-10 * np.abs(ev).max()
    # components of the active pixel graph (4-neighbour, periodic)
    from scipy.ndimage import label
    lab, ncomp = label(np.tile(act, (3, 3)))
    comps = len(np.unique(lab[4:8, 5:10][act != 0]))
    nz = np.sum(np.abs(ev) < 1e-9 * np.abs(ev).max())
    assert nz == comps


@pytest.mark.parametrize("p", [1, 2, 3])
def test_paper_wall_mode_is_stable(p):
    act = np.ones((3, 4), np.uint8)
    act[1, 2] = 0
    m = T.TriMesh(p=p, active=act, h=0.5, k0=1.0, periodic=True, wall_mode=1)
    ev = np.linalg.eigvals(T.dense_operator(m))
    assert ev.real.max() < 1e-10 * np.abs(ev).max()


@pytest.mark.parametrize("p", [2, 3])
def test_operator_exact_on_quadratics(p):
    """q = grad u and div(k q) are exact for u in P_p: L x = L y = L xy = 0 and
    L x^2 = L y^2 = 2k at every node of pixels away from the absorbing edge."""
    k, h = 0.7, 0.4
    m = T.TriMesh(p=p, active=np.ones((6, 7), np.uint8), h=h, x0=-1.0, y0=0.3, k0=k)
    X, Y = T.node_xy(p, h, m.x0, m.y0, m.nx, m.ny)
    inner = (slice(1, -1), slice(1, -1))
    for f, want in ((X, 0.0), (Y, 0.0), (X * Y, 0.0), (X * X, 2 * k), (Y * Y, 2 * k),
                    (X * X - 3 * X * Y + Y, 2 * k)):
        Lu = T.apply_L(m, f)
        assert np.abs(Lu[inner] - want).max() < 1e-10 * max(1.0, np.abs(f).max())


@pytest.mark.parametrize("p", [2, 3])
def test_free_diffusion_paper_value(p):
    """Sec. 4.2: free diffusion for T = 36 ms at k = 0.45 gives Sigma = 2Tk I
    = 32.4 I.  x^2 lies in the DG space for p >= 2 and L is symmetric in the
    mass inner product, so d/dt M_xx = 2k M0 holds exactly and RK3
    integrates it exactly: Sigma is exact until the density's tail reaches
    the absorbing edge.  The central fluxes give a heavier than Gaussian far
    tail (at 10 sigma the density is 1e-11, not 1e-22), whose loss at the
    edge, weighted by x^2 ~ 1e4, moves Sigma(36 ms) by 1e-8."""
    g = json.load(open(os.path.join(GOLD, "paper_free_diffusion.json")))
    k, Tt = g["k0_um2_per_ms"], g["T_ms"]
    nel, side, s0 = 50, 200.0, 8.0
    h = side / nel
    m = T.TriMesh(p=p, active=np.ones((nel, nel), np.uint8), h=h, x0=-side / 2, y0=-side / 2, k0=k)
    n, dt = O.step_plan(T.power_rho(m, iters=150), Tt)
    xs, ys = 0.3 * h, -0.2 * h
    u0 = T.init_gaussian(m, xs, ys, s0)
    m0 = T.moments(m, u0, xs, ys)
    # the rate identity on the start density
    rate = T.moments(m, T.apply_L(m, u0), xs, ys)
    assert abs(rate[3] / (2 * k * m0[0]) - 1) < 1e-12 and abs(rate[0]) < 1e-15 * m0[0]
    # a quarter of the way: exact
    q = n // 4
    u = T.rk3(m, u0, q, dt)
    s = O.aggregate(np.array([T.moments(m, u, xs, ys)]), np.array([m0]))[0]
    assert abs(s[0] / (2 * k * q * dt) - 1) < 1e-10 and abs(s[2] / (2 * k * q * dt) - 1) < 1e-10
    # the paper's T
    u = T.rk3(m, u, n - q, dt)
    m1 = T.moments(m, u, xs, ys)
    s = O.aggregate(np.array([m1]), np.array([m0]))[0]
    assert abs(s[0] - g["sigma_analytic_diag"]) < 1e-8 * 32.4
    assert abs(s[2] - g["sigma_analytic_diag"]) < 1e-8 * 32.4
    assert abs(s[1]) < 1e-8 * 32.4
    assert abs(m1[0] / m0[0] - 1) < 1e-9


def test_mass_conservation_per_component():
    act = np.ones((8, 8), np.uint8)
    act[2:6, 2] = act[2:6, 5] = 0
    act[2, 2:6] = act[5, 2:6] = 0          # a closed ring of wall pixels
    m = T.TriMesh(p=2, active=act, h=0.5, k0=2.0, periodic=True)
    u0 = T.init_gaussian(m, 1.3, 1.1, 0.4)  # straddles the ring
    n, dt = O.step_plan(T.power_rho(m, iters=150), 0.3)
    u = T.rk3(m, u0, n, dt)
    inside = np.zeros(act.shape, bool)
    inside[3:5, 3:5] = True
    for region in (inside, ~inside):
        a, b = u0.copy(), u.copy()
        a[~region] = 0
        b[~region] = 0
        ma, mb = T.moments(m, a, 0, 0)[0], T.moments(m, b, 0, 0)[0]
        assert ma > 1e-4
        assert abs(mb / ma - 1) < 1e-12


@pytest.mark.parametrize("p,order", [(1, 1.7), (2, 2.7), (3, 3.7)])
def test_manufactured_heat_convergence(p, order):
    """u = 1 + exp(-2 D a^2 t) sin(a x) sin(a y) on a periodic square."""
    D, Lside, tend = 1.0, 2.0, 0.05
    a = 2 * math.pi / Lside
    errs = []
    for nel in (6, 12):
        h = Lside / nel
        m = T.TriMesh(p=p, active=np.ones((nel, nel), np.uint8), h=h, k0=D, periodic=True)
        X, Y = T.node_xy(p, h, 0.0, 0.0, nel, nel)
        u0 = 1 + np.sin(a * X) * np.sin(a * Y)
        rho = T.power_rho(m, iters=100)
        n = int(math.ceil(tend / (0.1 * O.rk3_real_limit() / rho)))
        u = T.rk3(m, u0, n, tend / n)
        exact = 1 + math.exp(-2 * D * a * a * tend) * np.sin(a * X) * np.sin(a * Y)
        err = u - exact
        M = T.ref_matrices(p)["M"] * h * h
        errs.append(math.sqrt(float(np.einsum("yxti,ij,yxtj->", err, M, err))))
    assert math.log2(errs[0] / errs[1]) > order


def test_diagonal_symmetry():
    """Swapping x and y maps the pixel triangulation onto itself (A <-> B): a
    transposed geometry and start point swap Sigma_xx and Sigma_yy."""
    rng = np.random.default_rng(5)
    act = (rng.random((10, 10)) > 0.2).astype(np.uint8)
    act[4:6, 4:6] = 1
    h, s0 = 0.5, 0.6
    out = []
    for A, (xs, ys) in ((act, (2.3, 2.6)), (act.T.copy(), (2.6, 2.3))):
        m = T.TriMesh(p=2, active=A, h=h, k0=1.0, periodic=True)
        u0 = T.init_gaussian(m, xs, ys, s0)
        u = T.rk3(m, u0, 40, 2e-3)
        out.append(O.aggregate(np.array([T.moments(m, u, xs, ys)]),
                               np.array([T.moments(m, u0, xs, ys)]))[0])
    assert abs(out[0][0] - out[1][2]) < 1e-12 and abs(out[0][2] - out[1][0]) < 1e-12
    assert abs(out[0][1] - out[1][1]) < 1e-12
