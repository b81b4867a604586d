"""FP64 CPU oracle of the learned warm-start network.

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the bench's
CPU-baseline leg, never by the product path.  It shares no code with the
CUDA kernels.

The paper has no learned component.  What it does have is the hook: in the
non-linear extension of the Galerkin solver (section 2.1.1) the strain of the
previous load step is the initial iterate of the next solve.  Here a small
network proposes that initial iterate instead, from the phase map phi and
the macro strain E_bar; the solver then starts from it (after projecting it
onto compatible fields) and the FP64 true residual decides when to stop.

Network (fixed architecture, channel widths configurable for tests):
  * periodic 3x3x3 convolutions (cross-correlation, wrap-around padding),
    taps t = 9 (dz+1) + 3 (dy+1) + (dx+1), weights W[t, c_out, c_in], bias;
  * ReLU after every convolution except the head;
  * encoder: two convolutions per level, 2x2x2 average pooling between
    levels; decoder: nearest-neighbour upsampling of the coarser level,
    concatenated after the skip tensor of the same level ([skip, up]), two
    convolutions;
  * head: one convolution to 36 channels M[6 c + J]; the prediction is
    x0_c = sum_J M[6 c + J] E_J, i.e. linear in E_bar by construction (the
    elastic cell problem is linear in the macro strain).  Components are
    Mandel (shears times sqrt 2) for E_bar and x0.
Tensors are channels-last: [batch, n1, n2, n3, channels].
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


# ----------------------------------------------------------------- primitives
def shift(x, dz, dy, dx):
    """y[z, y, x] = x[(z+dz) % n1, (y+dy) % n2, (x+dx) % n3] on [B, n1, n2, n3, C]."""
    return np.roll(x, (-dz, -dy, -dx), axis=(1, 2, 3))


def conv3d(x, W, b):
    """Periodic 3x3x3 cross-correlation: y = sum_t shift_t(x) W[t]^T + b."""
    y = np.zeros(x.shape[:4] + (W.shape[1],))
    for t, (dz, dy, dx) in enumerate(OFFSETS):
        y += shift(x, dz, dy, dx) @ W[t].T
    return y + b


def conv3d_dgrad(g, W):
    """Gradient w.r.t. the input of conv3d: dx = sum_t shift_{-t}(g) W[t]."""
    dx = np.zeros(g.shape[:4] + (W.shape[2],))
    for t, (dz, dy, dx_) in enumerate(OFFSETS):
        dx += shift(g, -dz, -dy, -dx_) @ W[t]
    return dx


def conv3d_wgrad(g, x):
    """Gradients w.r.t. W and b: dW[t] = sum_v g[v] outer shift_t(x)[v]."""
    cout, cin = g.shape[-1], x.shape[-1]
    dW = np.zeros((27, cout, cin))
    g2 = g.reshape(-1, cout)
    for t, (dz, dy, dx) in enumerate(OFFSETS):
        dW[t] = g2.T @ shift(x, dz, dy, dx).reshape(-1, cin)
    return dW, g2.sum(axis=0)


def avgpool2(x):
    B, n1, n2, n3, C = x.shape
    return x.reshape(B, n1 // 2, 2, n2 // 2, 2, n3 // 2, 2, C).mean(axis=(2, 4, 6))


def avgpool2_grad(g):
    """Adjoint of avgpool2 (each fine voxel gets 1/8 of its coarse gradient)."""
    return upsample2(g) / 8.0


def upsample2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


def upsample2_grad(g):
    """Adjoint of nearest upsampling: sum of the 8 fine gradients."""
    return avgpool2(g) * 8.0


def relu(x):
    return np.maximum(x, 0.0)


def bf16(x):
    """Round to bfloat16 (round to nearest, ties to even), returned as float64;
    used to mirror where a BF16 implementation stores tensors."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# -------------------------------------------------------------- architecture
def layer_specs(channels=(16, 32, 48, 64), cin=1, cout=36):
    """Convolution layers in forward order: (name, c_in, c_out, relu)."""
    c1, c2, c3, c4 = channels
    return [
        ("e1a", cin, c1, True), ("e1b", c1, c1, True),
        ("e2a", c1, c2, True), ("e2b", c2, c2, True),
        ("e3a", c2, c3, True), ("e3b", c3, c3, True),
        ("bna", c3, c4, True), ("bnb", c4, c4, True),
        ("d3a", c3 + c4, c3, True), ("d3b", c3, c3, True),
        ("d2a", c2 + c3, c2, True), ("d2b", c2, c2, True),
        ("d1a", c1 + c2, c1, True), ("d1b", c1, c1, True),
        ("head", c1, cout, False),
    ]


def init_params(specs, rng):
    """He-normal weights (fan-in 27 c_in), zero biases; the head is scaled
    down by 10 so the first predictions are small."""
    P = {}
    for name, ci, co, act in specs:
        std = np.sqrt(2.0 / (27 * ci)) * (1.0 if act else 0.1)
        P[name + ".W"] = rng.standard_normal((27, co, ci)) * std
        P[name + ".b"] = np.zeros(co)
    return P


def forward(P, phi, Ebar, specs=None, store=None):
    """phi [B, n1, n2, n3], Ebar [B, 6] (Mandel) -> x0 [B, n1, n2, n3, 6] and
    the cache of intermediates for backward.  store(x) is applied to every
    stored activation (identity, or bf16 to mirror a BF16 implementation)."""
    specs = specs or layer_specs()
    st = store or (lambda a: a)
    cache = {}

    def conv(name, x):
        y = conv3d(x, P[name + ".W"], P[name + ".b"])
        act = dict((s[0], s[3]) for s in specs)[name]
        cache[name + ".in"] = x
        if act:
            y = st(relu(y))
        cache[name + ".out"] = y
        return y

    x = st(phi[..., None].astype(np.float64))
    s1 = conv("e1b", conv("e1a", x))
    s2 = conv("e2b", conv("e2a", st(avgpool2(s1))))
    s3 = conv("e3b", conv("e3a", st(avgpool2(s2))))
    bn = conv("bnb", conv("bna", st(avgpool2(s3))))
    d3 = conv("d3b", conv("d3a", np.concatenate([s3, upsample2(bn)], axis=-1)))
    d2 = conv("d2b", conv("d2a", np.concatenate([s2, upsample2(d3)], axis=-1)))
    d1 = conv("d1b", conv("d1a", np.concatenate([s1, upsample2(d2)], axis=-1)))
    M = conv("head", d1)                                  # [B, ..., 36]
    B = phi.shape[0]
    Mr = M.reshape(M.shape[:4] + (6, 6))                  # [..., c, J]
    x0 = np.einsum("bzyxcj,bj->bzyxc", Mr, Ebar)
    cache.update(M=M, Ebar=np.asarray(Ebar, dtype=np.float64), B=B,
                 widths={"s1": s1.shape[-1], "s2": s2.shape[-1], "s3": s3.shape[-1]})
    return x0, cache


def loss_and_grad_out(x0, target, weight=None):
    """Mean squared error over all components and voxels (each voxel's terms
    times weight[b, z, y, x] if given), and d loss / d x0."""
    d = x0 - target
    w = np.ones(x0.shape[:4]) if weight is None else weight
    wd = w[..., None] * d
    return float(np.sum(wd * d) / d.size), 2.0 * wd / d.size


def backward(P, cache, gx0, specs=None, store=None):
    """Gradients of the loss w.r.t. every parameter, given d loss / d x0.
    store(g) is applied where a BF16 implementation stores a gradient tensor
    that feeds a convolution (the masked output gradients)."""
    specs = specs or layer_specs()
    st = store or (lambda a: a)
    acts = dict((s[0], s[3]) for s in specs)
    G = {}
    Ebar = cache["Ebar"]
    gM = np.einsum("bzyxc,bj->bzyxcj", gx0, Ebar).reshape(cache["M"].shape)

    def conv_back(name, gy, need_dx=True):
        if acts[name]:
            gy = gy * (cache[name + ".out"] > 0)
        gy = st(gy)
        dW, db = conv3d_wgrad(gy, cache[name + ".in"])
        G[name + ".W"] = dW
        G[name + ".b"] = db
        return st(conv3d_dgrad(gy, P[name + ".W"])) if need_dx else None

    w = cache["widths"]
    gd1 = conv_back("head", gM)
    gcat1 = conv_back("d1a", conv_back("d1b", gd1))
    gs1 = gcat1[..., :w["s1"]]
    gd2 = upsample2_grad(gcat1[..., w["s1"]:])
    gcat2 = conv_back("d2a", conv_back("d2b", gd2))
    gs2 = gcat2[..., :w["s2"]]
    gd3 = upsample2_grad(gcat2[..., w["s2"]:])
    gcat3 = conv_back("d3a", conv_back("d3b", gd3))
    gs3 = gcat3[..., :w["s3"]]
    gbn = upsample2_grad(gcat3[..., w["s3"]:])
    gs3 = gs3 + avgpool2_grad(conv_back("bna", conv_back("bnb", gbn)))
    gs2 = gs2 + avgpool2_grad(conv_back("e3a", conv_back("e3b", gs3)))
    gs1 = gs1 + avgpool2_grad(conv_back("e2a", conv_back("e2b", gs2)))
    conv_back("e1a", conv_back("e1b", gs1), need_dx=False)
    return G


def adam_step(P, G, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam (Kingma and Ba, 2015) with bias correction; updates in place."""
    for k in P:
        m[k] = beta1 * m[k] + (1 - beta1) * G[k]
        v[k] = beta2 * v[k] + (1 - beta2) * G[k] ** 2
        mh = m[k] / (1 - beta1 ** step)
        vh = v[k] / (1 - beta2 ** step)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)


def upsample_trilinear(x, s):
    """Periodic trilinear interpolation of voxel-centred values by an integer
    factor s along each axis: [B, m1, m2, m3, C] -> [B, s m1, s m2, s m3, C]."""
    out = x
    for ax in (1, 2, 3):
        m = out.shape[ax]
        pos = (np.arange(m * s) + 0.5) / s - 0.5          # fine centres in coarse index units
        i0 = np.floor(pos).astype(int)
        t = pos - i0
        a = np.take(out, i0 % m, axis=ax)
        b = np.take(out, (i0 + 1) % m, axis=ax)
        shape = [1] * out.ndim
        shape[ax] = m * s
        t = t.reshape(shape)
        out = a * (1 - t) + b * t
    return out
