"""FP64 numpy reference of the covariance surrogate network.

TEST INFRASTRUCTURE ONLY: checks the CUDA forward, backward and training
kernels of the surrogate (include/dgsurrogate.h).  The paper has no learned
part; the network maps an occupancy raster and (D, Delta) to Sigma/(2 D Delta)
and is trained on Sigma values of the DG solver.

Same architecture and parameter order as the library.  The library keeps
weights and activations in BF16 and accumulates in FP32; this reference
rounds weights and activations to BF16 at the same points (round to nearest
even) and accumulates in FP64, so the two agree to FP32 accumulation error
except where a BF16 rounding of an intermediate value falls the other way.
The gradient of each convolution's output is rounded to BF16 before it
enters the weight, bias and input gradients (the library's tensor cores take
BF16 operands).
"""
from __future__ import annotations

import numpy as np

CH = (1, 48, 96, 192, 384)
RES = 128
COND, HIDDEN, OUT = 2, 256, 3
FEAT = CH[-1] + COND


ROUND_BF16 = True  # False turns the BF16 emulation off (smooth loss for finite differences)


def bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    if not ROUND_BF16:
        return np.asarray(x, dtype=np.float64)
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def layout():
    """(name, shape) of every parameter block in order."""
    out = []
    for l in range(4):
        out.append((f"conv{l}_w", (CH[l + 1], CH[l], 3, 3)))
        out.append((f"conv{l}_b", (CH[l + 1],)))
    out += [("f1_w", (HIDDEN, FEAT)), ("f1_b", (HIDDEN,)), ("f2_w", (OUT, HIDDEN)), ("f2_b", (OUT,))]
    return out


def unpack(vec):
    vec = np.asarray(vec, dtype=np.float64)
    p, off = {}, 0
    for name, shp in layout():
        n = int(np.prod(shp))
        p[name] = vec[off:off + n].reshape(shp)
        off += n
    assert off == vec.size
    return p


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in layout()])


def _conv(x, w):
    """3x3 convolution with zero padding, x [B, Ci, H, W], w [Co, Ci, 3, 3]."""
    B, Ci, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    z = np.zeros((B, w.shape[0], H, W))
    for ky in range(3):
        for kx in range(3):
            z += np.einsum("oc,bchw->bohw", w[:, :, ky, kx], xp[:, :, ky:ky + H, kx:kx + W])
    return z


def _conv_t(dz, w):
    """Gradient of _conv with respect to its input."""
    B, Co, H, W = dz.shape
    dxp = np.zeros((B, w.shape[1], H + 2, W + 2))
    for ky in range(3):
        for kx in range(3):
            dxp[:, :, ky:ky + H, kx:kx + W] += np.einsum("oc,bohw->bchw", w[:, :, ky, kx], dz)
    return dxp[:, :, 1:H + 1, 1:W + 1]


def _conv_w(dz, x):
    """Gradient of _conv with respect to its weights."""
    B, Ci, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    g = np.zeros((dz.shape[1], Ci, 3, 3))
    for ky in range(3):
        for kx in range(3):
            g[:, :, ky, kx] = np.einsum("bohw,bchw->oc", dz, xp[:, :, ky:ky + H, kx:kx + W])
    return g


def forward(params, occ, cond):
    """Returns (y [B, 3], cache).  occ [B, 128, 128] in {0, 1}, cond [B, 2]."""
    p = unpack(params)
    x = np.asarray(occ, dtype=np.float64)[:, None, :, :]
    cache = {"x": [x], "a": []}
    for l in range(4):
        z = _conv(x, bf16(p[f"conv{l}_w"])) + p[f"conv{l}_b"][None, :, None, None]
        a = bf16(np.maximum(z, 0.0))
        B, C, H, W = a.shape
        x = bf16(0.25 * a.reshape(B, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5)))
        cache["a"].append(a)
        cache["x"].append(x)
    g = x.mean(axis=(2, 3))
    g32 = np.float32(g).astype(np.float64) if ROUND_BF16 else g
    feat = np.concatenate([g32, np.asarray(cond, dtype=np.float64)], axis=1)
    fb = bf16(feat)
    hid = np.maximum(fb @ bf16(p["f1_w"]).T + p["f1_b"], 0.0)
    hb = bf16(hid)
    y = hb @ bf16(p["f2_w"]).T + p["f2_b"]
    cache.update(feat=feat, fb=fb, hid=hid, hb=hb, p=p)
    return y, cache


def loss_and_grad(params, occ, cond, target):
    """Mean squared error over the batch and outputs, and its gradient."""
    y, c = forward(params, occ, cond)
    p = c["p"]
    B = y.shape[0]
    t = np.asarray(target, dtype=np.float64)
    loss = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / (B * OUT)
    g = {}
    g["f2_w"] = dy.T @ c["hb"]
    g["f2_b"] = dy.sum(0)
    dh = (dy @ bf16(p["f2_w"])) * (c["hid"] > 0)
    g["f1_w"] = dh.T @ c["fb"]
    g["f1_b"] = dh.sum(0)
    df = dh @ bf16(p["f1_w"])
    x4 = c["x"][4]
    HW = x4.shape[2] * x4.shape[3]
    dx = np.broadcast_to(df[:, :CH[-1], None, None] / HW, x4.shape).copy()
    for l in range(3, -1, -1):
        a = c["a"][l]
        dz = bf16(0.25 * np.repeat(np.repeat(dx, 2, axis=2), 2, axis=3) * (a > 0))
        g[f"conv{l}_w"] = _conv_w(dz, c["x"][l])
        g[f"conv{l}_b"] = dz.sum(axis=(0, 2, 3))
        if l > 0:
            dx = _conv_t(dz, bf16(p[f"conv{l}_w"]))
    return loss, pack(g), y
