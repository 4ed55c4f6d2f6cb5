"""Surrogate kernels vs the FP64 oracle on tiny shapes (needs a GPU).

The GPU keeps activations in BF16 and multiplies BF16 weights; the oracle
runs in FP64 on the same BF16-rounded inputs and weights.  Bounds: exact for
data movement (pooling, upsampling), FP32 accumulation error for the weight
gradient of BF16 operands, and relative errors of order the BF16 unit
roundoff (2^-8) per stored layer for everything downstream of a stored
activation: 1e-2 of the tensor's largest magnitude per layer.  Whole-network
gradients are compared with the oracle's layers composed with BF16 rounding
at the GPU's storage points (1e-2 in norm), and by direction (cosine > 0.99)
with the plain FP64 oracle, from which ReLU masks of near-zero
pre-activations can differ."""
import numpy as np
import pytest

from oracle import surrogate_oracle as so

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_01827_gb300 import build
    build.build()


def bf16_round(a):
    """Round-to-nearest-even to BF16, returned as float64."""
    a = np.asarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _t(a, dtype):
    import torch
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


def _conv_case(B=2, H=6, W=10, Cin=16, Cout=24, seed=0):
    r = np.random.default_rng(seed)
    x = bf16_round(r.standard_normal((B, H, W, Cin)))
    w = bf16_round(r.standard_normal((Cout, 3, 3, Cin)) * 0.2)
    b = r.standard_normal(Cout).astype(np.float32).astype(np.float64)
    return x, w, b


@pytest.mark.parametrize("relu", [0, 1])
def test_conv3x3_forward(relu):
    import torch
    from oracle import surrogate_oracle as so
    from paper_2509_01827_gb300.surrogate import _p, sg
    x, w, b = _conv_case(B=3, H=7, W=13, Cin=24, Cout=40)  # ragged pixel and channel tiles
    B, H, W, Cin = x.shape
    Cout = w.shape[0]
    ldy, yoff = Cout + 8, 8  # write into a channel slice
    y = torch.zeros((B * H * W, ldy), dtype=torch.bfloat16, device="cuda")
    xd, wd, bd = _t(x, torch.bfloat16), _t(w, torch.bfloat16), _t(b, torch.float32)
    rc = sg().cem_sg_conv3x3(_p(xd), B, H, W, Cin, Cin, _p(wd), _p(bd), Cout, relu, None, 0, _p(y),
                             ldy, yoff, 0)
    assert rc == 0
    torch.cuda.synchronize()
    yg = y.float().cpu().numpy().reshape(B, H, W, ldy)
    ref = so.conv2d(x, w, b, 1)
    if relu:
        ref = so.relu(ref)
    assert _rel(yg[..., yoff:], ref) < 1e-2
    assert np.all(yg[..., :yoff] == 0)  # other channels untouched


@pytest.mark.parametrize("cin,cout", [(32, 32), (16, 136)])
def test_conv3x3_many_tiles(cin, cout):
    """64,000 pixels: several waves of 128-pixel tiles on the tcgen05 path
    (with a ragged channel tile for 136 outputs).  Against the oracle, with
    bias and ReLU, and as a data gradient with the ReLU mask of a layer
    input."""
    import ctypes
    import torch
    from oracle import surrogate_oracle as so
    from paper_2509_01827_gb300.surrogate import _p, sg
    x, w, b = _conv_case(B=8, H=80, W=100, Cin=cin, Cout=cout, seed=cin + cout)
    B, H, W, _ = x.shape
    P = B * H * W
    L = sg()
    xd, wd, bd = _t(x, torch.bfloat16), _t(w, torch.bfloat16), _t(b, torch.float32)
    y = torch.zeros((P, cout), dtype=torch.bfloat16, device="cuda")
    assert L.cem_sg_conv3x3(_p(xd), B, H, W, cin, cin, _p(wd), _p(bd), cout, 1, None, 0, _p(y),
                            cout, 0, 0) == 0
    mask = _t(bf16_round(np.random.default_rng(5).standard_normal((P, cout))), torch.bfloat16)
    ym = torch.zeros_like(y)
    assert L.cem_sg_conv3x3(_p(xd), B, H, W, cin, cin, _p(wd), None, cout, 0, _p(mask), cout,
                            _p(ym), cout, 0, 0) == 0
    torch.cuda.synchronize()
    ref = so.conv2d(x, w, b, 1)
    assert _rel(y.float().cpu().numpy().reshape(B, H, W, cout), so.relu(ref)) < 1e-2
    ref0 = (ref - b).reshape(P, cout)
    got = ym.float().cpu().numpy()
    keep = mask.float().cpu().numpy() > 0
    assert np.all(got[~keep] == 0)
    assert _rel(np.where(keep, got, 0.0), np.where(keep, ref0, 0.0)) < 1e-2
    n = ctypes.c_int(-1)
    assert L.cem_sg_timeouts(ctypes.byref(n)) == 0 and n.value == 0


def test_conv3x3_weight_gradient_and_data_gradient():
    import torch
    from oracle import surrogate_oracle as so
    from paper_2509_01827_gb300.surrogate import _p, sg
    x, w, b = _conv_case(B=2, H=9, W=11, Cin=16, Cout=24, seed=1)
    B, H, W, Cin = x.shape
    Cout = w.shape[0]
    r = np.random.default_rng(2)
    dy = bf16_round(r.standard_normal((B, H, W, Cout)))
    dx_ref, dw_ref, db_ref = so.conv2d_bwd(x, w, dy, 1)
    L = sg()
    ws_bytes = L.cem_sg_wgrad_workspace(B, H, W, Cin, Cout)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    xd, dyd = _t(x, torch.bfloat16), _t(dy, torch.bfloat16)
    dw = torch.empty((Cout, 3, 3, Cin), dtype=torch.float32, device="cuda")
    db = torch.empty(Cout, dtype=torch.float32, device="cuda")
    assert L.cem_sg_conv3x3_wgrad(_p(xd), Cin, _p(dyd), Cout, B, H, W, Cin, Cout, _p(dw), _p(db),
                                  _p(ws), ws_bytes, 0) == 0
    # data gradient: the forward kernel with the transposed, flipped weights
    wt = np.transpose(w[:, ::-1, ::-1, :], (3, 1, 2, 0)).copy()  # [Cin][3][3][Cout]
    dx = torch.empty((B * H * W, Cin), dtype=torch.bfloat16, device="cuda")
    wtd = _t(wt, torch.bfloat16)
    assert L.cem_sg_conv3x3(_p(dyd), B, H, W, Cout, Cout, _p(wtd), None, Cin, 0, None, 0,
                            _p(dx), Cin, 0, 0) == 0
    # the same with the ReLU mask of the layer's input applied in the epilogue
    dxm = torch.empty_like(dx)
    assert L.cem_sg_conv3x3(_p(dyd), B, H, W, Cout, Cout, _p(wtd), None, Cin, 0, _p(xd), Cin,
                            _p(dxm), Cin, 0, 0) == 0
    torch.cuda.synchronize()
    # BF16 x BF16 products are exact in FP32; only the FP32 sums round
    assert _rel(dw.cpu().numpy(), dw_ref) < 1e-5
    assert _rel(db.cpu().numpy(), db_ref) < 1e-5
    dxg = dx.float().cpu().numpy().reshape(B, H, W, Cin)
    assert _rel(dxg, dx_ref) < 1e-2
    np.testing.assert_array_equal(dxm.float().cpu().numpy().reshape(B, H, W, Cin),
                                  np.where(x > 0, dxg, 0.0))


def test_adam_writes_flipped_copy():
    import torch
    from oracle import surrogate_oracle as so
    from paper_2509_01827_gb300.surrogate import _p, sg
    r = np.random.default_rng(3)
    Cout, Cin = 16, 8
    w = r.standard_normal((Cout, 3, 3, Cin)).astype(np.float32)
    g = r.standard_normal(w.shape).astype(np.float32)
    m = r.standard_normal(w.shape).astype(np.float32) * 0.1
    v = np.abs(r.standard_normal(w.shape)).astype(np.float32) * 0.1
    wd, gd, md, vd = (_t(a, torch.float32) for a in (w, g, m, v))
    wb = torch.empty(w.shape, dtype=torch.bfloat16, device="cuda")
    wt = torch.empty((Cin, 3, 3, Cout), dtype=torch.bfloat16, device="cuda")
    assert sg().cem_sg_adam(_p(wd), _p(gd), _p(md), _p(vd), w.size, 1e-2, 0.9, 0.999, 1e-8, 3,
                            _p(wb), _p(wt), Cout, Cin, 0) == 0
    torch.cuda.synchronize()
    # the kernel's hyperparameters are FP32 numbers: give the oracle the same
    f = lambda v: float(np.float32(v))
    w1, m1, v1 = so.adam(w.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                         v.astype(np.float64), 3, f(1e-2), f(0.9), f(0.999), f(1e-8))
    np.testing.assert_allclose(wd.cpu().numpy(), w1, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(md.cpu().numpy(), m1, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(vd.cpu().numpy(), v1, rtol=1e-5, atol=1e-8)
    wn = wd.cpu().numpy()
    np.testing.assert_array_equal(wb.float().cpu().numpy(), bf16_round(wn))
    np.testing.assert_array_equal(wt.float().cpu().numpy(),
                                  bf16_round(np.transpose(wn[:, ::-1, ::-1, :], (3, 1, 2, 0))))


def test_pool_upsample_exact():
    import torch
    from oracle import surrogate_oracle as so
    from paper_2509_01827_gb300.surrogate import _p, sg
    r = np.random.default_rng(4)
    B, H, W, C = 2, 4, 6, 8  # pooled size
    x = bf16_round(r.standard_normal((B, 2 * H, 2 * W, C)))
    dy = bf16_round(r.standard_normal((B, H, W, C)))
    skip = bf16_round(r.standard_normal((B, 2 * H, 2 * W, C)))
    L = sg()
    xd, dyd, skd = _t(x, torch.bfloat16), _t(dy, torch.bfloat16), _t(skip, torch.bfloat16)
    y = torch.empty((B * H * W, C), dtype=torch.bfloat16, device="cuda")
    dx = torch.empty((B * 4 * H * W, C), dtype=torch.bfloat16, device="cuda")
    assert L.cem_sg_maxpool2(_p(xd), C, B, H, W, C, _p(y), 0) == 0
    assert L.cem_sg_maxpool2_bwd(_p(xd), C, _p(dyd), _p(skd), C, 0, B, H, W, C, 0, _p(dx), 0) == 0
    dxr = torch.empty_like(dx)  # with the ReLU mask of x
    assert L.cem_sg_maxpool2_bwd(_p(xd), C, _p(dyd), _p(skd), C, 0, B, H, W, C, 1, _p(dxr), 0) == 0
    up = torch.zeros((B * 4 * H * W, C + 8), dtype=torch.bfloat16, device="cuda")
    assert L.cem_sg_upsample2(_p(dyd), B, H, W, C, _p(up), C + 8, 8, 0) == 0
    dup = torch.empty((B * H * W, C), dtype=torch.bfloat16, device="cuda")
    assert L.cem_sg_upsample2_bwd(_p(up, 8), C + 8, B, H, W, C, None, 0, _p(dup), 0) == 0
    mk = bf16_round(r.standard_normal((B, H, W, C)))
    dupm = torch.empty_like(dup)
    assert L.cem_sg_upsample2_bwd(_p(up, 8), C + 8, B, H, W, C, _p(_t(mk, torch.bfloat16)), C,
                                  _p(dupm), 0) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(y.float().cpu().numpy().reshape(B, H, W, C), so.maxpool2(x))
    ref_dx = bf16_round(so.maxpool2_bwd(x, dy) + skip)
    np.testing.assert_array_equal(dx.float().cpu().numpy().reshape(x.shape), ref_dx)
    np.testing.assert_array_equal(dxr.float().cpu().numpy().reshape(x.shape),
                                  np.where(x > 0, ref_dx, 0.0))
    np.testing.assert_array_equal(up.float().cpu().numpy().reshape(B, 2 * H, 2 * W, C + 8)[..., 8:],
                                  so.upsample2(dy))
    ref_up = bf16_round(so.upsample2_bwd(so.upsample2(dy)))
    np.testing.assert_array_equal(dup.float().cpu().numpy().reshape(B, H, W, C), ref_up)
    np.testing.assert_array_equal(dupm.float().cpu().numpy().reshape(B, H, W, C),
                                  np.where(mk > 0, ref_up, 0.0))


def test_bce_and_head():
    import torch
    from oracle import surrogate_oracle as so
    from paper_2509_01827_gb300.surrogate import _p, sg
    r = np.random.default_rng(5)
    P, C = 3000, 24
    x = bf16_round(r.standard_normal((P, C)))
    w = r.standard_normal(C).astype(np.float32).astype(np.float64)
    b = np.array([0.3])
    t = (r.random(P) < 0.1).astype(np.uint8)
    L = sg()
    xd, wd, bd = _t(x, torch.bfloat16), _t(w, torch.float32), _t(b, torch.float32)
    z = torch.empty(P, dtype=torch.float32, device="cuda")
    assert L.cem_sg_head_fwd(_p(xd), P, C, _p(wd), _p(bd), _p(z), 0) == 0
    dz = torch.empty_like(z)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    wsb = int(max(L.cem_sg_bce_workspace(P), L.cem_sg_head_workspace(P, C)))
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    td = _t(t, torch.uint8)
    assert L.cem_sg_bce(_p(z), _p(td), P, 7.0, _p(dz), _p(loss), _p(ws), wsb, 0) == 0
    dx = torch.empty((P, C), dtype=torch.bfloat16, device="cuda")
    dw = torch.empty(C, dtype=torch.float32, device="cuda")
    db = torch.empty(1, dtype=torch.float32, device="cuda")
    assert L.cem_sg_head_bwd(_p(xd), P, C, _p(wd), _p(dz), _p(dx), _p(dw), _p(db), _p(ws), wsb,
                             0) == 0
    torch.cuda.synchronize()
    zr = so.conv2d(x.reshape(1, 1, P, C), w.reshape(1, 1, 1, C), b, 0).reshape(P)
    assert _rel(z.cpu().numpy(), zr) < 1e-5
    lr, dzr = so.bce_logits(zr, t, 7.0)
    assert abs(loss.item() - lr) <= 1e-5 * abs(lr)
    assert _rel(dz.cpu().numpy(), dzr) < 1e-4
    dxr, dwr, dbr = so.conv2d_bwd(x.reshape(1, 1, P, C), w.reshape(1, 1, 1, C), dzr.reshape(1, 1, P, 1), 0)
    assert _rel(dw.cpu().numpy(), dwr.reshape(C)) < 1e-4
    assert _rel(db.cpu().numpy(), dbr) < 1e-4
    # the head's input is a ReLU output: no gradient where it is <= 0
    assert _rel(dx.float().cpu().numpy(), np.where(x > 0, dxr.reshape(P, C), 0.0)) < 1e-2


@pytest.mark.parametrize("n_per", [9000, 4096, 1])
def test_soft_dice_against_the_oracle(n_per):
    """cem_sg_dice on 3 images (9000 elements: two whole 4096-element chunks
    and a ragged one; exactly one chunk; one element): the loss and the
    gradient it adds to an existing dz against the oracle's soft Dice, to
    FP32 summation accuracy."""
    import torch
    from paper_2509_01827_gb300.surrogate import _p, sg
    r = np.random.default_rng(11)
    B = 3
    z = (r.standard_normal((B, n_per)) * 3).astype(np.float32).astype(np.float64)
    t = (r.random((B, n_per)) < 0.2).astype(np.uint8)
    dz0 = r.standard_normal((B, n_per)).astype(np.float32).astype(np.float64) * 1e-3
    L = sg()
    wsb = int(L.cem_sg_dice_workspace(B, n_per))
    assert wsb > 0
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    zd, td, dzd = _t(z, torch.float32), _t(t, torch.uint8), _t(dz0, torch.float32)
    loss = torch.zeros(2, dtype=torch.float32, device="cuda")
    assert L.cem_sg_dice(_p(zd), _p(td), B, n_per, 0.7, 1.0, _p(dzd), _p(loss, 1), _p(ws), wsb,
                         0) == 0
    torch.cuda.synchronize()
    lr, dzr = so.soft_dice(z, t, eps=1.0)
    assert loss[0].item() == 0.0
    assert abs(loss[1].item() - 0.7 * lr) <= 1e-5 * max(1e-3, abs(lr))
    assert _rel(dzd.cpu().numpy() - dz0, 0.7 * dzr) < 1e-4
    # bad arguments
    assert L.cem_sg_dice(_p(zd), _p(td), B, n_per, 0.7, 0.0, _p(dzd), _p(loss), _p(ws), wsb, 0) != 0
    assert L.cem_sg_dice(_p(zd), _p(td), B, n_per, 0.7, 1.0, _p(dzd), _p(loss), _p(ws), wsb - 4,
                         0) != 0


def _unet_bf16_reference(p, x, t, chans, pw):
    """The oracle's layers composed with BF16 rounding wherever the GPU
    stores a tensor in BF16 (conv outputs, data gradients, pooled and
    upsampled gradients); logits, loss gradient and weight gradients stay
    unrounded.  Returns the loss and the parameter gradients."""
    R = bf16_round
    L = len(chans)
    ea, eb, pools, cats, da, db = {}, {}, {}, {}, {}, {}
    h = x
    for l in range(L):
        ea[l] = R(so.relu(so.conv2d(h, p[f"e{l}a.w"], p[f"e{l}a.b"], 1)))
        eb[l] = R(so.relu(so.conv2d(ea[l], p[f"e{l}b.w"], p[f"e{l}b.b"], 1)))
        if l < L - 1:
            pools[l] = so.maxpool2(eb[l])
            h = pools[l]
    ins = {0: x}
    for l in range(1, L):
        ins[l] = pools[l - 1]
    h = eb[L - 1]
    for l in range(L - 2, -1, -1):
        cats[l] = np.concatenate([so.upsample2(h), eb[l]], axis=3)
        da[l] = R(so.relu(so.conv2d(cats[l], p[f"d{l}a.w"], p[f"d{l}a.b"], 1)))
        db[l] = R(so.relu(so.conv2d(da[l], p[f"d{l}b.w"], p[f"d{l}b.b"], 1)))
        h = db[l]
    z = so.conv2d(h, p["out.w"], p["out.b"], 0)
    loss, dz = so.bce_logits(z[..., 0], t, pw)
    g = {}
    dh, g["out.w"], g["out.b"] = so.conv2d_bwd(h, p["out.w"], dz[..., None], 0)
    dh = R(dh)
    dskip = {}
    for l in range(L - 1):
        dh = so.relu_bwd(db[l], dh)
        dx, g[f"d{l}b.w"], g[f"d{l}b.b"] = so.conv2d_bwd(da[l], p[f"d{l}b.w"], dh, 1)
        dh = so.relu_bwd(da[l], R(dx))
        dx, g[f"d{l}a.w"], g[f"d{l}a.b"] = so.conv2d_bwd(cats[l], p[f"d{l}a.w"], dh, 1)
        dx = R(dx)
        cu = dx.shape[3] - chans[l]
        dskip[l] = dx[..., cu:]
        dh = R(so.upsample2_bwd(dx[..., :cu]))
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            dh = R(so.maxpool2_bwd(eb[l], dh) + dskip[l])
        dh = so.relu_bwd(eb[l], dh)
        dx, g[f"e{l}b.w"], g[f"e{l}b.b"] = so.conv2d_bwd(ea[l], p[f"e{l}b.w"], dh, 1)
        dh = so.relu_bwd(ea[l], R(dx))
        dx, g[f"e{l}a.w"], g[f"e{l}a.b"] = so.conv2d_bwd(ins[l], p[f"e{l}a.w"], dh, 1)
        dh = R(dx)
    return loss, g


def test_unet_loss_gradients_vs_oracle():
    """Whole network: logits, loss and every parameter gradient, against the
    oracle's layers with the GPU's BF16 storage points (tight), and against
    the plain FP64 oracle (direction of every gradient)."""
    import torch
    from oracle import surrogate_oracle as so
    from paper_2509_01827_gb300.surrogate import UNet
    chans = [8, 16, 24]
    B, H, W = 2, 8, 12
    net = UNet(B, H, W, chans=chans, seed=3, pos_weight=4.0)
    r = np.random.default_rng(6)
    # non-zero biases so that every path is exercised
    for p in net.convs.values():
        p["b"].copy_(torch.tensor(r.standard_normal(p["cout"]) * 0.1, dtype=torch.float32))
    net._refresh_copies()
    x3 = bf16_round(r.standard_normal((B, H, W, 3)))
    x8 = np.zeros((B, H, W, 8))
    x8[..., :3] = x3
    net.set_input(torch.tensor(x8.reshape(-1, 8), dtype=torch.float32, device="cuda"))
    t = (r.random((B, H, W)) < 0.2).astype(np.uint8)
    td = torch.tensor(t.reshape(-1), dtype=torch.uint8, device="cuda")
    net.forward()
    loss = net.loss_and_grad(td)
    net.backward()
    torch.cuda.synchronize()
    p = net.params_numpy()
    pr = {k: (bf16_round(v) if k.endswith(".w") and k != "out.w" else v) for k, v in p.items()}
    z_ref, _ = so.unet_forward(pr, x3, chans)
    assert _rel(net.z.cpu().numpy().reshape(B, H, W), z_ref[..., 0]) < 3e-2
    loss_ref, g_ref = so.unet_loss_and_grads(pr, x3, t, chans, 4.0)
    assert abs(loss[0].item() - loss_ref) <= 1e-2 * abs(loss_ref)
    g = net.grads_numpy()
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
    loss_e, g_e = _unet_bf16_reference(pr, x3, t, chans, 4.0)
    assert abs(loss[0].item() - loss_e) <= 1e-4 * abs(loss_e)
    errs = {k: rel(g[k], g_e[k]) for k in g_e}
    print("relative gradient errors vs the BF16-storage reference:",
          {k: round(v, 5) for k, v in errs.items()})
    assert max(errs.values()) < 1e-2, errs
    cos = {k: float(np.sum(g[k] * g_ref[k]) / (np.linalg.norm(g[k]) * np.linalg.norm(g_ref[k])))
           for k in g_ref}
    print("cosine vs the FP64 oracle:", {k: round(v, 4) for k, v in cos.items()})
    assert min(cos.values()) > 0.99, cos


def test_training_reduces_loss():
    import torch
    from paper_2509_01827_gb300.surrogate import UNet
    B, H, W = 4, 16, 16
    net = UNet(B, H, W, chans=[8, 16], seed=0, pos_weight=2.0, lr=3e-3)
    r = np.random.default_rng(7)
    x = r.standard_normal((B, H, W, 8)).astype(np.float32)
    x[..., 3:] = 0
    t = (x[..., 0] > 0.5).astype(np.uint8)  # a learnable map
    net.set_input(torch.tensor(x.reshape(-1, 8), device="cuda"))
    td = torch.tensor(t.reshape(-1), device="cuda")
    losses = [float(net.train_step(td)[0].item()) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0], losses[::10]


@pytest.mark.parametrize("cin,cout", [(8, 32), (24, 40), (32, 64), (64, 128), (96, 32), (128, 256), (40, 96),
                                      (16, 18), (256, 512), (256, 768)])
def test_tcgen05_and_mma_paths_agree(cin, cout):
    """The tcgen05 (TMEM) and mma.sync paths of the 3x3 convolution against the
    oracle, ragged pixel counts, every N tile width; no bounded wait gives up."""
    import ctypes
    import torch
    from paper_2509_01827_gb300.surrogate import _p, sg
    x, w, b = _conv_case(B=2, H=9, W=23, Cin=cin, Cout=cout, seed=cin + cout)
    B, H, W, _ = x.shape
    L = sg()
    xd, wd, bd = _t(x, torch.bfloat16), _t(w, torch.bfloat16), _t(b, torch.float32)
    mk = _t(bf16_round(np.random.default_rng(9).standard_normal((B, H, W, cout))), torch.bfloat16)
    ref = so.relu(so.conv2d(x, w, b, 1))
    mref = np.where(mk.float().cpu().numpy().reshape(B, H, W, cout) > 0, ref, 0.0)
    out = {}
    try:
        for path in (1, 0):
            assert L.cem_sg_set_gemm_path(path) == 0
            y = torch.zeros((B * H * W, cout), dtype=torch.bfloat16, device="cuda")
            assert L.cem_sg_conv3x3(_p(xd), B, H, W, cin, cin, _p(wd), _p(bd), cout, 1, _p(mk),
                                    cout, _p(y), cout, 0, 0) == 0
            torch.cuda.synchronize()
            out[path] = y.float().cpu().numpy().reshape(B, H, W, cout)
    finally:
        L.cem_sg_set_gemm_path(1)
    n = ctypes.c_int(-1)
    assert L.cem_sg_timeouts(ctypes.byref(n)) == 0 and n.value == 0
    for path in (1, 0):
        assert _rel(out[path], mref) < 1e-2, path


@pytest.mark.parametrize("cin,cout", [(16, 24), (8, 32), (32, 64), (64, 128), (40, 96), (128, 256),
                                      (768, 256), (256, 512)])
def test_weight_gradient_paths_agree(cin, cout):
    """Weight and bias gradients on the tcgen05 path and on the mma.sync path
    against the oracle (BF16 products are exact in FP32)."""
    import ctypes
    import torch
    from paper_2509_01827_gb300.surrogate import _p, sg
    x, w, b = _conv_case(B=2, H=9, W=23, Cin=cin, Cout=cout, seed=3 * cin + cout)
    B, H, W, _ = x.shape
    dy = bf16_round(np.random.default_rng(cout).standard_normal((B, H, W, cout)))
    _, dw_ref, db_ref = so.conv2d_bwd(x, w, dy, 1)
    L = sg()
    ws_bytes = L.cem_sg_wgrad_workspace(B, H, W, cin, cout)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    xd, dyd = _t(x, torch.bfloat16), _t(dy, torch.bfloat16)
    try:
        for path in (1, 0):
            assert L.cem_sg_set_gemm_path(path) == 0
            dw = torch.full((cout, 3, 3, cin), float("nan"), dtype=torch.float32, device="cuda")
            db = torch.full((cout,), float("nan"), dtype=torch.float32, device="cuda")
            assert L.cem_sg_conv3x3_wgrad(_p(xd), cin, _p(dyd), cout, B, H, W, cin, cout, _p(dw),
                                          _p(db), _p(ws), ws_bytes, 0) == 0
            torch.cuda.synchronize()
            assert _rel(dw.cpu().numpy(), dw_ref) < 1e-5, path
            assert _rel(db.cpu().numpy(), db_ref) < 1e-5, path
    finally:
        L.cem_sg_set_gemm_path(1)
    n = ctypes.c_int(-1)
    assert L.cem_sg_timeouts(ctypes.byref(n)) == 0 and n.value == 0
