"""The nodal tables the kernels use (dg_basis_tables, host only, no device).

FP64: nodes and weights equal the textbook GLL closed forms and D the
oracle's independently computed differentiation matrix.  FP32: the values
the FP32 kernels hold must keep what conservation of mass rests on.  The
derivative of a constant is zero, so every row of D and of D D sums to
exactly zero in exact arithmetic on the stored FP32 values.  The left-right
mirror symmetry of the basis must also hold exactly.  Each entry must stay
within a few FP32 ulps of the FP64 value.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def dg():
    from paper_1907_06191_gb300 import _build
    _build.build()
    O.build()
    import paper_1907_06191_gb300 as m
    return m


def _exact_row_sums(M):
    return [sum((Fraction(float(v)) for v in row), Fraction(0)) for row in M]


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_fp64_tables(dg, p):
    xi, w, D, D2 = dg.basis_tables(p, dg.DG_FP64)
    gold = json.load(open(os.path.join(HERE, "golden", "gll_closed_forms.json")))
    if f"p{p}" in gold:
        assert np.abs(xi - gold[f"p{p}"]["nodes"]).max() < 1e-15
        assert np.abs(w - gold[f"p{p}"]["weights"]).max() < 1e-15
    xo, wo, Do = O.gll(p)
    assert np.abs(xi - xo).max() < 1e-15 and np.abs(w - wo).max() < 1e-15
    assert np.abs(D - Do).max() < 1e-13 * np.abs(Do).max()
    assert np.abs(D2 - Do @ Do).max() <= 1e-13 * max(np.abs(Do @ Do).max(), 1.0)
    assert np.array_equal(xi, -xi[::-1])       # mirrored nodes, 0 in the middle
    # summation by parts, W D + D^T W = diag(-1, 0, ..., 0, 1)
    B = np.diag(w) @ D + D.T @ np.diag(w)
    E = np.zeros_like(B)
    E[0, 0], E[p, p] = -1.0, 1.0
    assert np.abs(B - E).max() < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_fp32_tables_conserve(dg, p):
    _, w, D, D2 = dg.basis_tables(p, dg.DG_FP64)
    _, _, Df, D2f = dg.basis_tables(p, dg.DG_FP32)
    for M in (Df, D2f):
        assert np.array_equal(M.astype(np.float32).astype(np.float64), M)  # FP32 values
        assert all(s == 0 for s in _exact_row_sums(M))
    assert np.array_equal(Df, -Df[::-1, ::-1])
    assert np.array_equal(D2f, D2f[::-1, ::-1])
    for M, R in ((Df, D), (D2f, D2)):
        nz = R != 0
        ulp = np.spacing(np.abs(R[nz]).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(M[nz] - R[nz]) <= 3 * ulp)
        assert np.all(M[~nz] == 0)
    # consequence: the weighted volume term of a constant adds exactly no mass
    assert sum((Fraction(float(wa)) * s for wa, s in zip(w, _exact_row_sums(D2f))), Fraction(0)) == 0


def test_plain_rounding_would_break_row_sums(dg):
    """The correction is needed: rounding D D to FP32 entry by entry leaves
    nonzero row sums at p = 3 (a source of mass proportional to u)."""
    _, _, _, D2 = dg.basis_tables(3, dg.DG_FP64)
    rounded = D2.astype(np.float32).astype(np.float64)
    assert any(s != 0 for s in _exact_row_sums(rounded))


def test_bad_arguments(dg):
    L = dg.lib()
    assert L.dg_basis_tables(0, dg.DG_FP64, None, None, None, None) == dg.DG_EINVAL
    assert L.dg_basis_tables(6, dg.DG_FP64, None, None, None, None) == dg.DG_EINVAL
    assert L.dg_basis_tables(3, 7, None, None, None, None) == dg.DG_EINVAL
    assert L.dg_basis_tables(3, dg.DG_FP32, None, None, None, None) == dg.DG_OK


@pytest.mark.parametrize("p", [1, 2, 3])
def test_triangle_tables_match_the_oracle(dg, p):
    """The library builds its triangle tables on its own (Gauss-Jordan on the
    monomial Vandermonde matrix, exact monomial integrals); they must equal
    the oracle's independently assembled matrices."""
    from oracle import triangles as T
    r, s, G, Lf, mono = dg.triangle_tables(p)
    R = T.ref_matrices(p)
    Minv = np.linalg.inv(R["M"])
    X = T.ref_nodes(p)
    assert np.abs(r - X[:, 0]).max() < 1e-15 and np.abs(s - X[:, 1]).max() < 1e-15
    EN = T.edge_nodes(p)
    for t in (0, 1):
        rx, ry, sx, sy = T._INVJ[t]
        assert np.abs(G[t, 0] + Minv @ (rx * R["Sr"].T + sx * R["Ss"].T)).max() < 1e-10
        assert np.abs(G[t, 1] + Minv @ (ry * R["Sr"].T + sy * R["Ss"].T)).max() < 1e-10
        for e in range(3):
            ln = T._EDGE[t][e][1]
            assert np.abs(Lf[t, e] - ln * Minv[:, EN[e]] @ R["E1"]).max() < 1e-10
    for q, ab in enumerate([(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]):
        assert np.abs(mono[q] - R["mono_w"][ab]).max() < 1e-14
    # exactness the kernels rely on: with u_hat = u on every edge, the weak
    # gradient G u + sum_e n_e Lf_e u_e is the gradient of u in P_p (h = 1)
    for t, (x, y) in enumerate(((r + s, s), (r, r + s))):
        for u, gx, gy in ((x, 1.0, 0.0), (y, 0.0, 1.0), (x * y if p > 1 else x, None, None)):
            qx, qy = G[t, 0] @ u, G[t, 1] @ u
            for e in range(3):
                (nx_, ny_), _ = T._EDGE[t][e]
                lift = Lf[t, e] @ u[EN[e]]
                qx, qy = qx + nx_ * lift, qy + ny_ * lift
            if gx is None:
                gx, gy = (y, x) if p > 1 else (1.0, 0.0)
            assert np.abs(qx - gx).max() < 1e-10 and np.abs(qy - gy).max() < 1e-10
