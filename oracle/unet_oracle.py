"""FP64 numpy oracle for the learned gradient preconditioner (a U-Net) and its training step.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` may import this module.  It shares no code with the CUDA library.

The paper names learned regularisation only as motivation (Sec. 1); the network is this
library's own design, written here as plain definitions:

* layout: activations [n, H, W, C] (channels last); a 3x3 convolution's weight is
  [Co, 3, 3, Ci] (cross-correlation with one cell of zero padding on each side, stride 1),
  a 1x1 convolution's weight is [Co, Ci]; every convolution has a bias [Co];
* ``levels`` encoder levels with c_l = base * 2**l channels; level l has two 3x3
  convolution + ReLU layers; between levels a 2x2 max pool (stride 2);
* decoder levels l = levels-2 .. 0: nearest-neighbour 2x upsampling of the level below,
  concatenated as [upsampled, skip] along channels, then two 3x3 convolution + ReLU layers
  down to c_l channels;
* output: a 1x1 convolution to ``cout`` channels, no activation;
* loss: L = 1/(2 n H W cout) sum mask[n,h,w] (y - t)^2 with a 0/1 mask;
* Adam (Kingma & Ba 2015, Algorithm 1) with bias correction.

The flat parameter vector lists, for each convolution in the order enc0a, enc0b, enc1a, ...,
enc(L-1)b, dec(L-2)a, dec(L-2)b, ..., dec0a, dec0b, out: the weight, then the bias.
Backward passes below are derived by hand from those definitions; the tests pin them to
central differences of the forward pass.

Optional storage rounding (``quantize``): a function applied where a BF16 implementation
stores operands of its products -- the network input, every weight (not the biases), every
convolution's activated output, and the output gradient of each convolution before its
weight- and input-gradient products (the bias gradient uses the unrounded one).  With
``quantize=bf16`` the ReLU masks and max-pool choices are taken on the same stored values a
BF16 implementation sees, so such an implementation can be compared tightly; the products
themselves stay FP64.  :func:`bf16` rounds to the nearest BF16 value, ties to even (the
format keeps the top 16 bits of an IEEE binary32 pattern: sign, 8 exponent bits, 7 fraction
bits).
"""
from __future__ import annotations

import numpy as np


def layer_shapes(levels, base, cin, cout):
    """[(name, ksize, Ci, Co)] in parameter order."""
    c = [base * 2 ** l for l in range(levels)]
    out = []
    ci = cin
    for l in range(levels):
        out.append((f"enc{l}a", 3, ci, c[l]))
        out.append((f"enc{l}b", 3, c[l], c[l]))
        ci = c[l]
    for l in range(levels - 2, -1, -1):
        out.append((f"dec{l}a", 3, c[l + 1] + c[l], c[l]))
        out.append((f"dec{l}b", 3, c[l], c[l]))
    out.append(("out", 1, c[0], cout))
    return out


def param_count(levels, base, cin, cout):
    return sum(k * k * ci * co + co for _, k, ci, co in layer_shapes(levels, base, cin, cout))


def unpack(params, levels, base, cin, cout):
    """Flat vector -> {name: (W, b)} views (W [Co,3,3,Ci] or [Co,Ci])."""
    params = np.asarray(params, dtype=np.float64)
    out, off = {}, 0
    for name, k, ci, co in layer_shapes(levels, base, cin, cout):
        nw = k * k * ci * co
        w = params[off:off + nw]
        w = w.reshape(co, 3, 3, ci) if k == 3 else w.reshape(co, ci)
        off += nw
        out[name] = (w, params[off:off + co])
        off += co
    assert off == params.size
    return out


def pack(grads, levels, base, cin, cout):
    parts = []
    for name, _, _, _ in layer_shapes(levels, base, cin, cout):
        gw, gb = grads[name]
        parts += [gw.reshape(-1), gb.reshape(-1)]
    return np.concatenate(parts)


def init_params(rng, levels, base, cin, cout):
    """He-normal weights (std sqrt(2 / fan_in)), small random biases."""
    parts = []
    for _, k, ci, co in layer_shapes(levels, base, cin, cout):
        fan = k * k * ci
        parts.append(rng.standard_normal(k * k * ci * co) * np.sqrt(2.0 / fan))
        parts.append(0.01 * rng.standard_normal(co))
    return np.concatenate(parts)


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _same(a):
    return a


# -- layers (definitions) ------------------------------------------------------------------

def conv3x3(x, w, b):
    """y[n,h,w,o] = b[o] + sum_{dh,dw,i} x[n, h+dh-1, w+dw-1, i] w[o,dh,dw,i] (zero outside)."""
    n, H, W, ci = x.shape
    xp = np.zeros((n, H + 2, W + 2, ci))
    xp[:, 1:-1, 1:-1, :] = x
    y = np.broadcast_to(b, (n, H, W, w.shape[0])).copy()
    for dh in range(3):
        for dw in range(3):
            y += xp[:, dh:dh + H, dw:dw + W, :] @ w[:, dh, dw, :].T
    return y


def conv3x3_backward(x, w, dy):
    """Gradients of sum(dy * conv3x3(x, w, b)) with respect to x, w and b."""
    n, H, W, ci = x.shape
    xp = np.zeros((n, H + 2, W + 2, ci))
    xp[:, 1:-1, 1:-1, :] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for dh in range(3):
        for dwi in range(3):
            win = xp[:, dh:dh + H, dwi:dwi + W, :]
            dw[:, dh, dwi, :] = np.tensordot(dy, win, axes=([0, 1, 2], [0, 1, 2]))
            dxp[:, dh:dh + H, dwi:dwi + W, :] += dy @ w[:, dh, dwi, :]
    return dxp[:, 1:-1, 1:-1, :], dw, dy.sum(axis=(0, 1, 2))


def conv1x1(x, w, b):
    return x @ w.T + b


def conv1x1_backward(x, w, dy):
    return dy @ w, np.tensordot(dy, x, axes=([0, 1, 2], [0, 1, 2])), dy.sum(axis=(0, 1, 2))


def relu(z):
    return np.maximum(z, 0.0)


def maxpool2(x):
    n, H, W, c = x.shape
    return x.reshape(n, H // 2, 2, W // 2, 2, c).max(axis=(2, 4))


def maxpool2_backward(x, dy):
    """The gradient of each 2x2 window goes to its first maximal element, scanning the
    window row by row."""
    n, H, W, c = x.shape
    dx = np.zeros_like(x)
    y = maxpool2(x)
    taken = np.zeros(y.shape, dtype=bool)
    for a in range(2):
        for bb in range(2):
            v = x[:, a::2, bb::2, :]
            hit = (v == y) & ~taken
            dx[:, a::2, bb::2, :] = np.where(hit, dy, 0.0)
            taken |= hit
    return dx


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_backward(dy):
    n, H2, W2, c = dy.shape
    return dy.reshape(n, H2 // 2, 2, W2 // 2, 2, c).sum(axis=(2, 4))


# -- the network ---------------------------------------------------------------------------

def _weights(params, levels, base, cin, cout, q):
    return {k: (q(w), b) for k, (w, b) in unpack(params, levels, base, cin, cout).items()}


def forward(params, x, levels, base, cin, cout, keep=False, quantize=None):
    """y [n,H,W,cout]; with ``keep`` also the intermediate activations for backward."""
    q = quantize or _same
    P = _weights(params, levels, base, cin, cout, q)
    x = np.asarray(x, dtype=np.float64)
    acts = {}
    h = q(x)
    skips = []
    for l in range(levels):
        if l > 0:
            acts[f"pool{l}_in"] = h
            h = maxpool2(h)
        acts[f"enc{l}a_in"] = h
        h = q(relu(conv3x3(h, *P[f"enc{l}a"])))
        acts[f"enc{l}a_out"] = h
        acts[f"enc{l}b_in"] = h
        h = q(relu(conv3x3(h, *P[f"enc{l}b"])))
        acts[f"enc{l}b_out"] = h
        skips.append(h)
    for l in range(levels - 2, -1, -1):
        u = upsample2(h)
        cat = np.concatenate([u, skips[l]], axis=3)
        acts[f"dec{l}a_in"] = cat
        h = q(relu(conv3x3(cat, *P[f"dec{l}a"])))
        acts[f"dec{l}a_out"] = h
        acts[f"dec{l}b_in"] = h
        h = q(relu(conv3x3(h, *P[f"dec{l}b"])))
        acts[f"dec{l}b_out"] = h
    acts["out_in"] = h
    y = conv1x1(h, *P["out"])
    return (y, acts) if keep else y


def loss(y, t, mask=None):
    """L = 1/(2 n H W cout) sum mask (y - t)^2 and dL/dy."""
    n, H, W, c = y.shape
    m = np.ones((n, H, W, 1)) if mask is None else np.asarray(mask, np.float64)[..., None]
    r = m * (y - t)
    inv = 1.0 / (n * H * W * c)
    return 0.5 * inv * float(np.sum(r * r)), inv * m * r


def loss_and_gradient(params, x, t, mask, levels, base, cin, cout, quantize=None):
    """(L, dL/dparams flat, y)."""
    q = quantize or _same
    P = _weights(params, levels, base, cin, cout, q)
    y, A = forward(params, x, levels, base, cin, cout, keep=True, quantize=quantize)
    L, dy = loss(y, t, mask)
    G = {}
    dh, gw, _ = conv1x1_backward(A["out_in"], P["out"][0], q(dy))
    G["out"] = (gw, dy.sum(axis=(0, 1, 2)))
    dskip = [None] * levels
    for l in range(0, levels - 1):
        for part in ("b", "a"):
            name = f"dec{l}{part}"
            out = A[f"{name}_out"]
            dz = dh * (out > 0)
            dx, gw, _ = conv3x3_backward(A[f"{name}_in"], P[name][0], q(dz))
            G[name] = (gw, dz.sum(axis=(0, 1, 2)))
            dh = dx
        c_up = dh.shape[3] - base * 2 ** l
        dskip[l] = dh[..., c_up:]
        dh = upsample2_backward(dh[..., :c_up])
    for l in range(levels - 1, -1, -1):
        if dskip[l] is not None:
            dh = dh + dskip[l]
        for part in ("b", "a"):
            name = f"enc{l}{part}"
            out = A[f"{name}_out"]
            dz = dh * (out > 0)
            dx, gw, _ = conv3x3_backward(A[f"{name}_in"], P[name][0], q(dz))
            G[name] = (gw, dz.sum(axis=(0, 1, 2)))
            dh = dx
        if l > 0:
            dh = maxpool2_backward(A[f"pool{l}_in"], dh)
    return L, pack(G, levels, base, cin, cout), y


def adam_step(w, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1); returns (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def flops_per_sample(levels, base, cin, cout, H, W):
    """Multiply-add count x 2 of one forward pass on an H x W input."""
    f = 0
    c = [base * 2 ** l for l in range(levels)]
    for name, k, ci, co in layer_shapes(levels, base, cin, cout):
        if name == "out":
            l = 0
        else:
            l = int(name[3])
        f += 2 * (H >> l) * (W >> l) * k * k * ci * co
    return f
