"""Surrogate kernels (forward, backward, Adam) against the FP64 numpy
reference with the same BF16 rounding points; the raster against the
oracle's mask."""
import numpy as np
import pytest

import dginputs
import oracle as O
from oracle import surrogate as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_06191_gb300 as dg  # noqa: E402


def _batch(n, seed):
    occ, cond = [], []
    for k in range(n):
        w = dginputs.workload_surrogate_member(seed + k)
        occ.append(dg.rasterize_disks(w.disks.cx, w.disks.cy, w.disks.r, w.L, 128))
        cond.append([np.log(w.D * (1.0 + k)), w.D])
    return np.stack(occ), np.array(cond, dtype=np.float32)


def test_raster_is_complement_of_oracle_mask():
    w = dginputs.workload_surrogate_member(3)
    occ = dg.rasterize_disks(w.disks.cx, w.disks.cy, w.disks.r, w.L, 128)
    ref = 1 - O.mask_disks(w.L, 128, w.disks.cx, w.disks.cy, w.disks.r)
    assert np.array_equal(occ, ref)


def test_gradients_and_prediction_match_reference():
    """Every gradient entry against the FP64 reference with the same BF16
    rounding points.  Both sides round the same intermediate values to BF16;
    where an FP32 and an FP64 sum straddle a rounding boundary one BF16 unit
    (2^-8 relative) moves, and a gradient entry sums many such terms, so the
    per-entry bound is a few BF16 units of the entry plus a few units of the
    block's typical entry (for entries that cancel to near zero)."""
    net = dg.Surrogate(max_batch=8, seed=3, device=0)
    occ, cond = _batch(4, 100)
    rng = np.random.default_rng(1)
    tgt = rng.uniform(0.3, 1.0, size=(4, 3)).astype(np.float32)
    to = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dt)
    occ_t, cond_t, tgt_t = to(occ, torch.uint8), to(cond, torch.float32), to(tgt, torch.float32)
    params = net.get_params()
    loss, grad = net.gradients(occ_t, cond_t, tgt_t)
    out = torch.zeros((4, 3), dtype=torch.float32, device="cuda:0")
    net.predict(occ_t, cond_t, out)
    rloss, rgrad, ry = S.loss_and_grad(params.astype(np.float64), occ, cond, tgt)
    assert np.abs(out.cpu().numpy() - ry).max() <= 1e-2 * np.abs(ry).max()
    assert abs(loss / rloss - 1) < 1e-2
    ulp = 2.0 ** -8
    off = 0
    for name, shp in S.layout():
        size = int(np.prod(shp))
        g, r = grad[off:off + size].astype(np.float64), rgrad[off:off + size]
        typ = np.sqrt(np.mean(r * r)) + 1e-30
        err = np.abs(g - r)
        bound = 4 * ulp * np.abs(r) + 4 * ulp * typ
        worst = float((err / bound).max())
        print(f"{name}: max |g - r| / bound = {worst:.3f}, max rel {float((err / (np.abs(r) + typ)).max()):.2e}")
        assert np.all(err <= bound), name
        off += size
    net.close()


def test_training_reduces_loss():
    net = dg.Surrogate(max_batch=64, seed=5, device=0)
    occ, cond = _batch(64, 200)
    frac = occ.reshape(64, -1).mean(1)
    tgt = np.stack([1 - 0.6 * frac, 0.02 * np.sin(cond[:, 0]), 1 - 0.5 * frac], 1).astype(np.float32)
    to = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dt)
    occ_t, cond_t, tgt_t = to(occ, torch.uint8), to(cond, torch.float32), to(tgt, torch.float32)
    first = net.train_step(occ_t, cond_t, tgt_t, 2e-3)
    for _ in range(150):
        last = net.train_step(occ_t, cond_t, tgt_t, 2e-3)
    assert last < first / 10
    p = net.get_params()
    net2 = dg.Surrogate(max_batch=64, seed=9, device=0)
    net2.set_params(p)
    a = torch.zeros((64, 3), device="cuda:0")
    b = torch.zeros((64, 3), device="cuda:0")
    net.predict(occ_t, cond_t, a)
    net2.predict(occ_t, cond_t, b)
    assert torch.equal(a, b)
    net.close()
    net2.close()


def test_augmentation_is_an_exact_symmetry_of_the_dg_sigma():
    """A flipped / transposed / shifted cell solved by DG gives the Sigma that
    augment() predicts from the original (up to the start-point sampling,
    which is carried along by transforming the start points too)."""
    from paper_1907_06191_gb300 import surrogate as sgm
    w = dginputs.workload_surrogate_member(7, m=8)
    w.deltas = [1.0]
    L = w.L
    # transpose: swap x and y of disks and start points
    t = dginputs.Workload(w.name, w.p, L, w.n_cell, w.tiles, w.D, w.sigma0, w.deltas,
                          dginputs.Disks(w.disks.cy.copy(), w.disks.cx.copy(), w.disks.r.copy(), L,
                                         w.disks.target_packing, w.disks.packing),
                          w.sources[:, ::-1].copy(), w.meta)
    s0, _ = sgm.dg_sigma([w])
    s1, _ = sgm.dg_sigma([t])
    occ0 = torch.from_numpy(dg.rasterize_disks(w.disks.cx, w.disks.cy, w.disks.r, L)[None]).cuda()
    occ1 = torch.from_numpy(dg.rasterize_disks(t.disks.cx, t.disks.cy, t.disks.r, L)[None]).cuda()
    tg = torch.from_numpy(s0[:, 0].astype(np.float32)).cuda()
    o, tt = sgm.augment(occ0, tg, 4, 0, 0)
    assert torch.equal(o, occ1)
    assert np.allclose(tt.cpu().numpy(), s1[:, 0], rtol=1e-5, atol=1e-7)


def test_trained_network_beats_the_packing_fit_on_held_out_cells():
    """The gain over the method without the network: trained on DG Sigma of
    seeded cells, the network's error on held-out cells (against their DG
    Sigma) is below that of a least-squares fit on the packing fraction and
    log(D Delta), the summary a user would have without it."""
    from paper_1907_06191_gb300 import surrogate as sgm
    ws_tr = [dginputs.workload_surrogate_member(s, m=16) for s in range(256)]
    ws_te = [dginputs.workload_surrogate_member(50000 + s, m=16) for s in range(48)]
    sig_tr, _ = sgm.dg_sigma(ws_tr)
    sig_te, _ = sgm.dg_sigma(ws_te)
    occ, cond, tgt = sgm.build_samples(ws_tr, sig_tr)
    occ_e, cond_e, tgt_e = sgm.build_samples(ws_te, sig_te)
    to = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dt)
    net = dg.Surrogate(max_batch=256, seed=1, device=0)
    sgm.train(net, to(occ, torch.uint8), to(cond, torch.float32), to(tgt, torch.float32),
              epochs=40, batch=64, lr=1e-3)
    pred = torch.zeros((occ_e.shape[0], 3), device="cuda:0")
    oe, ce = to(occ_e, torch.uint8), to(cond_e, torch.float32)
    for b0 in range(0, oe.shape[0], 256):
        net.predict(oe[b0:b0 + 256], ce[b0:b0 + 256], pred[b0:b0 + 256])
    rel = np.linalg.norm(pred.cpu().numpy() - tgt_e, axis=1) / np.linalg.norm(tgt_e, axis=1)
    base = sgm.packing_fit(ws_tr, tgt, ws_te)
    rel_b = np.linalg.norm(base - tgt_e, axis=1) / np.linalg.norm(tgt_e, axis=1)
    print(f"held-out error: network {rel.mean():.3f}, packing fit {rel_b.mean():.3f}")
    assert rel.mean() < rel_b.mean()
    net.close()
