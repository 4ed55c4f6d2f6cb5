"""FP64 CPU oracle of the crack-map surrogate -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the CUDA library never does.

The surrogate maps a 3-channel image of a notched-plate run (traction,
notch, critical energy release rate field) to the probability that each
element is cracked at the end of the run (the cracked-element map the
explicit solver produces, Secs. 3-4).  The network is a U-Net: per level two
3x3 convolutions with ReLU, 2x2 max pooling down, nearest-neighbour 2x
upsampling up, skip connections by channel concatenation, a final 1x1
convolution to one logit, and a class-weighted binary cross-entropy.  Every
function below is the plain definition in FP64 with numpy; the layer
gradients are derived by hand (no automatic differentiation) and pinned by
finite differences in the tests.

Layout: tensors are NHWC, x[b, h, w, c]; 3x3 weights are w[co, ky, kx, ci].
"""
import numpy as np


# ------------------------------------------------------------------ layers
def conv2d(x, w, b, pad):
    """y[n,h,w,o] = b[o] + sum_{ky,kx,c} x[n, h+ky-pad, w+kx-pad, c] w[o,ky,kx,c]
    (zero outside the image); stride 1, 'same' size for K = 2 pad + 1."""
    n, H, W, C = x.shape
    O, K, K2, C2 = w.shape
    assert K == K2 and C == C2 and K == 2 * pad + 1
    xp = np.zeros((n, H + 2 * pad, W + 2 * pad, C))
    xp[:, pad:pad + H, pad:pad + W, :] = x
    y = np.broadcast_to(b.astype(np.float64), (n, H, W, O)).copy()
    for ky in range(K):
        for kx in range(K):
            y += np.einsum("nhwc,oc->nhwo", xp[:, ky:ky + H, kx:kx + W, :], w[:, ky, kx, :])
    return y


def conv2d_bwd(x, w, dy, pad):
    """Gradients of sum(dy * conv2d(x, w, b, pad)) with respect to x, w, b."""
    n, H, W, C = x.shape
    O, K, _, _ = w.shape
    xp = np.zeros((n, H + 2 * pad, W + 2 * pad, C))
    xp[:, pad:pad + H, pad:pad + W, :] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros(w.shape)
    for ky in range(K):
        for kx in range(K):
            dw[:, ky, kx, :] = np.einsum("nhwo,nhwc->oc", dy, xp[:, ky:ky + H, kx:kx + W, :])
            dxp[:, ky:ky + H, kx:kx + W, :] += np.einsum("nhwo,oc->nhwc", dy, w[:, ky, kx, :])
    dx = dxp[:, pad:pad + H, pad:pad + W, :]
    db = dy.sum(axis=(0, 1, 2))
    return dx, dw, db


def relu(x):
    return np.maximum(x, 0.0)


def relu_bwd(y, dy):
    """Gradient through y = relu(x), given the output y (x > 0 iff y > 0)."""
    return np.where(y > 0.0, dy, 0.0)


def maxpool2(x):
    """2x2 max pooling, stride 2 (H and W even)."""
    n, H, W, C = x.shape
    v = x.reshape(n, H // 2, 2, W // 2, 2, C)
    return v.max(axis=(2, 4))


def maxpool2_bwd(x, dy):
    """The gradient goes to the maximum of each window; among equal maxima to
    the first in the order (0,0), (0,1), (1,0), (1,1)."""
    n, H, W, C = x.shape
    dx = np.zeros_like(x, dtype=np.float64)
    taken = np.zeros((n, H // 2, W // 2, C), bool)
    y = maxpool2(x)
    for dyy in range(2):
        for dxx in range(2):
            xs = x[:, dyy::2, dxx::2, :]
            hit = (xs == y) & ~taken
            dx[:, dyy::2, dxx::2, :] = np.where(hit, dy, 0.0)
            taken |= hit
    return dx


def upsample2(x):
    """Nearest-neighbour 2x upsampling."""
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_bwd(dy):
    n, H, W, C = dy.shape
    return dy.reshape(n, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def bce_logits(z, t, pos_weight):
    """Mean over elements of  pw t log(1+e^-z) + (1-t) log(1+e^z)  (class
    weight pw on cracked elements) and its gradient with respect to z."""
    z = z.astype(np.float64)
    t = t.astype(np.float64)
    sp_neg = np.logaddexp(0.0, -z)  # log(1 + e^-z)
    sp_pos = np.logaddexp(0.0, z)   # log(1 + e^z)
    loss = pos_weight * t * sp_neg + (1.0 - t) * sp_pos
    sig = 1.0 / (1.0 + np.exp(-z))
    dz = (pos_weight * t * (sig - 1.0) + (1.0 - t) * sig) / z.size
    return loss.mean(), dz


def soft_dice(z, t, eps=1.0):
    """Soft Dice loss of each sample's probability map against its target,
    averaged over the samples (z, t [n, ...]; p = sigmoid(z)):
        D_b = (2 sum p t + eps) / (sum p + sum t + eps),  loss = 1 - mean_b D_b,
    and its gradient with respect to z,
        d loss / d z_i = -(1/n) (2 t_i (S_b + eps) - (2 I_b + eps)) / (S_b + eps)^2
                         * p_i (1 - p_i),
    I_b = sum p t and S_b = sum p + sum t of the sample b that holds i."""
    z = z.astype(np.float64)
    t = t.astype(np.float64)
    n = z.shape[0]
    p = 1.0 / (1.0 + np.exp(-z))
    ax = tuple(range(1, z.ndim))
    inter = (p * t).sum(axis=ax)
    s = p.sum(axis=ax) + t.sum(axis=ax)
    d = (2.0 * inter + eps) / (s + eps)
    shape = (n,) + (1,) * (z.ndim - 1)
    S, I = (s + eps).reshape(shape), inter.reshape(shape)
    dd_dp = (2.0 * t * S - (2.0 * I + eps)) / (S * S)
    dz = -dd_dp * p * (1.0 - p) / n
    return 1.0 - d.mean(), dz


def adam(w, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba) with bias correction; step counts from 1."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------------ U-Net
def unet_shapes(cin, chans):
    """Parameter shapes: encoder level l has convs e{l}a, e{l}b; decoder level
    l < L-1 has convs d{l}a (input: upsampled level l+1 output concatenated
    with the level-l skip), d{l}b; 'out' is the 1x1 head."""
    shapes = {}
    c = cin
    for l, ch in enumerate(chans):
        shapes[f"e{l}a"] = (ch, 3, 3, c)
        shapes[f"e{l}b"] = (ch, 3, 3, ch)
        c = ch
    for l in range(len(chans) - 2, -1, -1):
        ch = chans[l]
        shapes[f"d{l}a"] = (ch, 3, 3, c + ch)
        shapes[f"d{l}b"] = (ch, 3, 3, ch)
        c = ch
    shapes["out"] = (1, 1, 1, c)
    return shapes


def unet_init(cin, chans, seed=0):
    """He-normal weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for k, s in unet_shapes(cin, chans).items():
        fan_in = s[1] * s[2] * s[3]
        p[k + ".w"] = rng.standard_normal(s) * np.sqrt(2.0 / fan_in)
        p[k + ".b"] = np.zeros(s[0])
    return p


def unet_forward(p, x, chans):
    """Logits [n, H, W, 1] and the cache the backward pass needs."""
    cache = {}
    h = x
    skips = []
    L = len(chans)
    for l in range(L):
        cache[f"e{l}a.in"] = h
        h = relu(conv2d(h, p[f"e{l}a.w"], p[f"e{l}a.b"], 1))
        cache[f"e{l}a.out"] = h
        cache[f"e{l}b.in"] = h
        h = relu(conv2d(h, p[f"e{l}b.w"], p[f"e{l}b.b"], 1))
        cache[f"e{l}b.out"] = h
        if l < L - 1:
            skips.append(h)
            cache[f"pool{l}.in"] = h
            h = maxpool2(h)
    for l in range(L - 2, -1, -1):
        u = upsample2(h)
        h = np.concatenate([u, skips[l]], axis=3)
        cache[f"d{l}a.in"] = h
        h = relu(conv2d(h, p[f"d{l}a.w"], p[f"d{l}a.b"], 1))
        cache[f"d{l}a.out"] = h
        cache[f"d{l}b.in"] = h
        h = relu(conv2d(h, p[f"d{l}b.w"], p[f"d{l}b.b"], 1))
        cache[f"d{l}b.out"] = h
    cache["out.in"] = h
    z = conv2d(h, p["out.w"], p["out.b"], 0)
    return z, cache


def unet_backward(p, cache, dz, chans):
    """Gradients of sum(dz * logits) with respect to every parameter."""
    g = {}
    L = len(chans)
    dh, g["out.w"], g["out.b"] = conv2d_bwd(cache["out.in"], p["out.w"], dz, 0)
    dskip = [None] * (L - 1)
    for l in range(0, L - 1):
        dh = relu_bwd(cache[f"d{l}b.out"], dh)
        dh, g[f"d{l}b.w"], g[f"d{l}b.b"] = conv2d_bwd(cache[f"d{l}b.in"], p[f"d{l}b.w"], dh, 1)
        dh = relu_bwd(cache[f"d{l}a.out"], dh)
        dh, g[f"d{l}a.w"], g[f"d{l}a.b"] = conv2d_bwd(cache[f"d{l}a.in"], p[f"d{l}a.w"], dh, 1)
        cu = dh.shape[3] - chans[l]
        dskip[l] = dh[..., cu:]
        dh = upsample2_bwd(dh[..., :cu])
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            dh = maxpool2_bwd(cache[f"pool{l}.in"], dh) + dskip[l]
        dh = relu_bwd(cache[f"e{l}b.out"], dh)
        dh, g[f"e{l}b.w"], g[f"e{l}b.b"] = conv2d_bwd(cache[f"e{l}b.in"], p[f"e{l}b.w"], dh, 1)
        dh = relu_bwd(cache[f"e{l}a.out"], dh)
        dh, g[f"e{l}a.w"], g[f"e{l}a.b"] = conv2d_bwd(cache[f"e{l}a.in"], p[f"e{l}a.w"], dh, 1)
    return g


def unet_loss_and_grads(p, x, t, chans, pos_weight):
    z, cache = unet_forward(p, x, chans)
    loss, dz = bce_logits(z[..., 0], t, pos_weight)
    g = unet_backward(p, cache, dz[..., None], chans)
    return loss, g


def jaccard(a, b):
    """|A n B| / |A u B| of two boolean maps (1 when both are empty)."""
    a = np.asarray(a, bool)
    b = np.asarray(b, bool)
    u = np.logical_or(a, b).sum()
    return 1.0 if u == 0 else float(np.logical_and(a, b).sum()) / float(u)
