"""Pins of the conv-net oracle: special cases with known results and finite
differences for every gradient."""
import numpy as np

from oracle import conv as CV


def test_identity_and_shift_kernels():
    """A centre-tap identity kernel returns the input; a single off-centre tap
    is a periodic shift (cross-correlation convention)."""
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 8, 6))
    W = np.zeros((3, 3, 3, 3))
    for c in range(3):
        W[c, c, 1, 1] = 1.0
    assert np.allclose(CV.conv3x3(x, W, np.zeros(3)), x)
    W2 = np.zeros((1, 1, 3, 3))
    W2[0, 0, 0, 2] = 1.0                        # dy = -1, dx = +1
    y = CV.conv3x3(x[:, :1], W2, np.zeros(1))
    assert np.allclose(y[0, 0], np.roll(x[0, 0], shift=(1, -1), axis=(0, 1)))


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 2, 5, 4))
    W = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    y = CV.conv3x3(x, W, b)
    H, Wd = 5, 4
    for o in range(3):
        for yy in range(H):
            for xx in range(Wd):
                s = b[o]
                for i in range(2):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            s += W[o, i, dy + 1, dx + 1] * x[0, i, (yy + dy) % H, (xx + dx) % Wd]
                assert abs(y[0, o, yy, xx] - s) < 1e-12


def test_gradients_by_finite_differences():
    rng = np.random.default_rng(2)
    params = CV.init_params(rng, widths=(2, 4, 4, 2), scale_last=1.0)
    x = rng.standard_normal((2, 2, 6, 5))
    tgt = rng.standard_normal((2, 2, 6, 5))
    loss, grads = CV.loss_and_grads(params, x, tgt)
    h = 1e-6
    for li in range(3):
        for pi in range(2):
            P = params[li][pi]
            G = grads[li][pi]
            for idx in [tuple(rng.integers(0, s) for s in P.shape) for _ in range(4)]:
                old = P[idx]
                P[idx] = old + h
                lp, _ = CV.loss_and_grads(params, x, tgt)
                P[idx] = old - h
                lm, _ = CV.loss_and_grads(params, x, tgt)
                P[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - G[idx]) < 1e-7 * max(1.0, abs(fd)), (li, pi, idx, fd, G[idx])


def test_adam_matches_closed_form_first_step():
    """After one Adam step the update is lr * sign(g) (bias-corrected)."""
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p1, m, v = CV.adam_update(p, g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(p1, p - 0.01 * np.sign(g), atol=1e-6)
