"""The FP64 reference of the surrogate network, pinned by finite
differences (BF16 emulation off, so the loss is smooth)."""
import numpy as np
import pytest

from oracle import surrogate as S


def test_reference_gradient_matches_finite_differences(monkeypatch):
    monkeypatch.setattr(S, "ROUND_BF16", False)
    rng = np.random.default_rng(4)
    n = sum(int(np.prod(shp)) for _, shp in S.layout())
    params = rng.normal(size=n) * 0.15
    # the network is fully convolutional up to the global average: a 32 x 32
    # raster exercises every layer at a fraction of the cost
    occ = (rng.random((2, 32, 32)) > 0.6).astype(np.float64)
    cond = rng.normal(size=(2, 2))
    tgt = rng.normal(size=(2, 3)) * 0.3
    loss, grad, _ = S.loss_and_grad(params, occ, cond, tgt)
    # a few coordinates in every block
    off = 0
    for name, shp in S.layout():
        size = int(np.prod(shp))
        for k in rng.choice(size, size=min(2, size), replace=False):
            i = off + int(k)
            eps = 1e-5
            pp, pm = params.copy(), params.copy()
            pp[i] += eps
            pm[i] -= eps
            fd = (S.loss_and_grad(pp, occ, cond, tgt)[0] - S.loss_and_grad(pm, occ, cond, tgt)[0]) / (2 * eps)
            assert abs(fd - grad[i]) <= 1e-6 + 1e-4 * abs(fd), (name, k, fd, grad[i])
        off += size


def test_bf16_rounding_is_round_to_nearest_even():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -9, -2.5, 3.14159])
    r = S.bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0 + 2 ** -7 or r[1] == 1.0  # halfway: ties to even
    assert r[3] == 1.0                              # below halfway
    assert r[2] == 1.0 + 2 ** -7                    # above halfway
    assert r[4] == -2.5
    assert abs(r[5] - 3.140625) < 1e-12
