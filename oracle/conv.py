"""Oracle for the learned preconditioner correction: a three-layer 3x3
convolution network (2 -> 32 -> 32 -> 2 channels, ReLU between layers,
periodic padding) in plain FP64 numpy, with its backward pass and the Adam
update.  The paper has no learned component; the network corrects the output
of the FFT preconditioner of Sec. III (Eq. PreconFFT_ECS) inside a flexible
CG, and this module is the slow reference its GPU kernels are checked
against.

TEST INFRASTRUCTURE (see ``oracle/__init__``).

Conventions: a field has shape [C][H][W] (or [B][C][H][W]); weights W have
shape [Cout][Cin][3][3], out[o, y, x] = b[o] + sum_{i, dy, dx}
W[o, i, dy+1, dx+1] in[i, y+dy, x+dx] with indices taken mod H and W
(cross-correlation, as in every deep-learning framework)."""
from __future__ import annotations

import numpy as np

TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv3x3(x, W, b):
    """x [B][Cin][H][W] -> [B][Cout][H][W], periodic padding."""
    out = np.zeros((x.shape[0], W.shape[0]) + x.shape[2:], dtype=np.float64)
    for (dy, dx) in TAPS:
        xs = np.roll(x, shift=(-dy, -dx), axis=(2, 3))       # xs[.., y, x] = x[.., y+dy, x+dx]
        out += np.einsum("oi,bihw->bohw", W[:, :, dy + 1, dx + 1], xs)
    return out + b[None, :, None, None]


def conv3x3_backward(x, W, gout):
    """Gradients of conv3x3 w.r.t. its input, weights and bias."""
    gx = np.zeros_like(x, dtype=np.float64)
    gW = np.zeros_like(W, dtype=np.float64)
    for (dy, dx) in TAPS:
        xs = np.roll(x, shift=(-dy, -dx), axis=(2, 3))
        gW[:, :, dy + 1, dx + 1] = np.einsum("bohw,bihw->oi", gout, xs)
        gxs = np.einsum("oi,bohw->bihw", W[:, :, dy + 1, dx + 1], gout)
        gx += np.roll(gxs, shift=(dy, dx), axis=(2, 3))
    gb = gout.sum(axis=(0, 2, 3))
    return gx, gW, gb


def init_params(rng, widths=(2, 32, 32, 2), scale_last=0.1):
    """He-style initial weights; the last layer starts small."""
    params = []
    for li in range(3):
        cin, cout = widths[li], widths[li + 1]
        W = rng.standard_normal((cout, cin, 3, 3)) * np.sqrt(2.0 / (9 * cin))
        if li == 2:
            W *= scale_last
        params.append([W, np.zeros(cout)])
    return params


def forward(params, x):
    """Returns the output and the activations needed by backward."""
    acts = [x]
    h = x
    for li, (W, b) in enumerate(params):
        z = conv3x3(h, W, b)
        h = np.maximum(z, 0.0) if li < 2 else z
        acts.append(h)
    return h, acts


def loss_and_grads(params, x, target):
    """Mean squared error over all elements and its parameter gradients."""
    out, acts = forward(params, x)
    diff = out - target
    n = diff.size
    loss = float(np.sum(diff * diff) / n)
    g = 2.0 * diff / n
    grads = [None] * 3
    for li in (2, 1, 0):
        W, b = params[li]
        if li < 2:
            g = g * (acts[li + 1] > 0)
        gx, gW, gb = conv3x3_backward(acts[li], W, g)
        grads[li] = [gW, gb]
        g = gx
    return loss, grads


def adam_update(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba) on arrays p with gradient g; returns the
    new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
