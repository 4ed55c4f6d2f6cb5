"""Pins of the surrogate's FP64 oracle (CPU only).

Each layer is checked against something other than itself: brute-force
loops on tiny inputs, scipy's 2-D correlation (a textbook special case),
adjoint identities, closed forms, and central finite differences of the
hand-derived gradients on random coordinates."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import surrogate_oracle as so


def _rng(s=0):
    return np.random.default_rng(s)


def test_conv2d_brute_force():
    r = _rng(1)
    x = r.standard_normal((2, 5, 6, 3))
    w = r.standard_normal((4, 3, 3, 3))
    b = r.standard_normal(4)
    y = so.conv2d(x, w, b, 1)
    for n in range(2):
        for h in range(5):
            for q in range(6):
                for o in range(4):
                    acc = b[o]
                    for ky in range(3):
                        for kx in range(3):
                            hh, ww = h + ky - 1, q + kx - 1
                            if 0 <= hh < 5 and 0 <= ww < 6:
                                for c in range(3):
                                    acc += x[n, hh, ww, c] * w[o, ky, kx, c]
                    assert abs(y[n, h, q, o] - acc) < 1e-12


def test_conv2d_is_a_sum_of_2d_correlations():
    r = _rng(2)
    x = r.standard_normal((1, 7, 9, 2))
    w = r.standard_normal((3, 3, 3, 2))
    y = so.conv2d(x, w, np.zeros(3), 1)
    for o in range(3):
        ref = sum(correlate2d(x[0, :, :, c], w[o, :, :, c], mode="same") for c in range(2))
        np.testing.assert_allclose(y[0, :, :, o], ref, rtol=0, atol=1e-12)


def test_conv2d_identity_kernel():
    x = _rng(3).standard_normal((2, 4, 4, 3))
    w = np.zeros((3, 3, 3, 3))
    for c in range(3):
        w[c, 1, 1, c] = 1.0
    np.testing.assert_array_equal(so.conv2d(x, w, np.zeros(3), 1), x)


def _fd_check(f, arr, grad, coords, h=1e-6, rtol=1e-6):
    for idx in coords:
        old = arr[idx]
        arr[idx] = old + h
        fp = f()
        arr[idx] = old - h
        fm = f()
        arr[idx] = old
        num = (fp - fm) / (2 * h)
        assert abs(num - grad[idx]) <= rtol * max(1.0, abs(num)), (idx, num, grad[idx])


def _coords(shape, k, r):
    return [tuple(int(r.integers(0, s)) for s in shape) for _ in range(k)]


@pytest.mark.parametrize("pad", [1, 0])
def test_conv2d_gradients_by_finite_differences(pad):
    r = _rng(4)
    K = 2 * pad + 1
    x = r.standard_normal((2, 5, 4, 3))
    w = r.standard_normal((4, K, K, 3))
    b = r.standard_normal(4)
    dy = r.standard_normal((2, 5, 4, 4))
    dx, dw, db = so.conv2d_bwd(x, w, dy, pad)
    f = lambda: float(np.sum(dy * so.conv2d(x, w, b, pad)))
    _fd_check(f, x, dx, _coords(x.shape, 16, r))
    _fd_check(f, w, dw, _coords(w.shape, 16, r))
    _fd_check(f, b, db, [(o,) for o in range(4)])


def test_pool_and_upsample_adjoint_and_gradient():
    r = _rng(5)
    x = r.standard_normal((2, 4, 6, 3))
    y = r.standard_normal((2, 8, 12, 3))
    # <up(x), y> = <x, up^T(y)>
    assert abs(np.sum(so.upsample2(x) * y) - np.sum(x * so.upsample2_bwd(y))) < 1e-12
    # max pooling: gradient by finite differences (no ties in random data)
    xm = r.standard_normal((2, 4, 6, 3))
    dy = r.standard_normal((2, 2, 3, 3))
    dx = so.maxpool2_bwd(xm, dy)
    f = lambda: float(np.sum(dy * so.maxpool2(xm)))
    _fd_check(f, xm, dx, _coords(xm.shape, 16, r))
    # ties go to the first element of the window
    xt = np.ones((1, 2, 2, 1))
    g = so.maxpool2_bwd(xt, np.ones((1, 1, 1, 1)))
    assert g[0, 0, 0, 0] == 1.0 and g.sum() == 1.0


def test_bce_closed_form_and_gradient():
    z = np.zeros((3, 4))
    t = np.zeros((3, 4))
    t[0, 0] = 1
    loss, dz = so.bce_logits(z, t, 5.0)
    # at z = 0 every term is log 2, weighted 5 on the one positive element
    assert abs(loss - np.log(2.0) * (11 + 5) / 12) < 1e-15
    r = _rng(6)
    z = r.standard_normal((3, 4))
    t = (r.random((3, 4)) < 0.3).astype(float)
    loss, dz = so.bce_logits(z, t, 3.0)
    _fd_check(lambda: so.bce_logits(z, t, 3.0)[0], z, dz, _coords(z.shape, 12, r), rtol=1e-7)


def test_soft_dice_closed_forms_and_gradient():
    # z = 0: p = 1/2 on all m elements of a sample with k cracked ones, so
    # D = (k + eps) / (m/2 + k + eps)
    z = np.zeros((2, 5, 4))
    t = np.zeros((2, 5, 4))
    t[0, 1, :3] = 1
    t[1, 4, 0] = 1
    loss, _ = so.soft_dice(z, t, eps=1.0)
    d = [(3 + 1.0) / (10 + 3 + 1.0), (1 + 1.0) / (10 + 1 + 1.0)]
    assert abs(loss - (1.0 - np.mean(d))) < 1e-15
    # saturated logits: p is the 0/1 map, and with eps = 0 the Dice index of
    # two sets is 2 J / (1 + J), J their Jaccard index
    r = _rng(7)
    for _ in range(4):
        a = r.random((1, 6, 7)) < 0.4
        b = r.random((1, 6, 7)) < 0.4
        zz = np.where(a, 60.0, -60.0)
        j = so.jaccard(a, b)
        loss, _ = so.soft_dice(zz, b.astype(float), eps=0.0)
        assert abs((1.0 - loss) - 2 * j / (1 + j)) < 1e-12
    # samples are independent: the loss of a batch is the mean of its samples'
    z = r.standard_normal((3, 4, 5))
    t = (r.random((3, 4, 5)) < 0.3).astype(float)
    per = [so.soft_dice(z[i:i + 1], t[i:i + 1])[0] for i in range(3)]
    loss, dz = so.soft_dice(z, t)
    assert abs(loss - np.mean(per)) < 1e-15
    _fd_check(lambda: so.soft_dice(z, t)[0], z, dz, _coords(z.shape, 16, r), rtol=1e-7)


def test_adam_first_step_moves_by_lr():
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    w1, m, v = so.adam(w, g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(w1, w - 0.01 * np.sign(g), rtol=0, atol=1e-15)


def test_unet_gradients_by_finite_differences():
    r = _rng(7)
    chans = [4, 6, 8]
    p = so.unet_init(3, chans, seed=1)
    for k in p:
        if k.endswith(".b"):
            p[k] = r.standard_normal(p[k].shape) * 0.1
    x = r.standard_normal((2, 8, 8, 3))
    t = (r.random((2, 8, 8)) < 0.2).astype(float)
    loss, g = so.unet_loss_and_grads(p, x, t, chans, 4.0)
    f = lambda: so.unet_loss_and_grads(p, x, t, chans, 4.0)[0]
    for k in ("e0a.w", "e1b.w", "e2a.w", "d1a.w", "d0b.w", "out.w", "d0a.b", "e2b.b"):
        _fd_check(f, p[k], g[k], _coords(p[k].shape, 2, r), rtol=1e-5)


def test_unet_shapes_param_count():
    # the 4-level, 32-base network of the surrogate: about 1.9 M parameters
    s = so.unet_shapes(3, [32, 64, 128, 256])
    n = sum(int(np.prod(v)) + v[0] for v in s.values())
    assert 1.8e6 < n < 2.1e6


def test_jaccard_definition():
    a = np.array([1, 1, 0, 0], bool)
    b = np.array([1, 0, 1, 0], bool)
    assert so.jaccard(a, b) == 1 / 3
    assert so.jaccard(np.zeros(3), np.zeros(3)) == 1.0
