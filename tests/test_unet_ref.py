"""Pins of the FP64 numpy U-Net reference (CPU): convolution against its written-out
definition, and every backpropagated gradient against central finite differences."""
import numpy as np
import pytest

from oracle import unet_ref as U


def test_conv3x3_matches_definition():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 6, 3))
    W = rng.standard_normal((3, 3, 3, 4))
    b = rng.standard_normal(4)
    y = U.conv3x3(x, W, b)
    for n in range(2):
        for h in range(5):
            for w in range(6):
                for co in range(4):
                    s = b[co]
                    for dh in (-1, 0, 1):
                        for dw in (-1, 0, 1):
                            hh, ww = h + dh, w + dw
                            if 0 <= hh < 5 and 0 <= ww < 6:
                                s += x[n, hh, ww] @ W[dh + 1, dw + 1, :, co]
                    assert abs(y[n, h, w, co] - s) < 1e-12


def test_pool_up_are_adjoint():
    """<pool(x), y> = <x, pool_backward(y)> and <up(x), y> = <x, up_backward(y)>."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 8, 6, 3))
    y = rng.standard_normal((1, 4, 3, 3))
    assert abs((U.pool(x) * y).sum() - (x * U.pool_backward(y)).sum()) < 1e-12
    xs = rng.standard_normal((1, 4, 3, 3))
    ys = rng.standard_normal((1, 8, 6, 3))
    assert abs((U.up(xs) * ys).sum() - (xs * U.up_backward(ys)).sum()) < 1e-12
    assert np.allclose(U.pool(np.ones((1, 4, 4, 1))), 1.0)


@pytest.mark.parametrize("name", ["e0a.W", "e1b.W", "b_a.W", "d2a.W", "d0b.W", "head.W", "e2a.b", "d1b.b", "head.b"])
def test_gradients_match_finite_differences(name):
    rng = np.random.default_rng(2)
    cin, cout, ch = 3, 2, (3, 4, 5, 6)
    params = U.init_params(cin, cout, ch, seed=3)
    x = rng.standard_normal((1, 16, 8, cin))
    t = rng.standard_normal((1, 16, 8, cout))
    wch = [1.0, 0.5]
    _, g = U.loss_and_grads(params, x, t, wch)
    flat = params[name].reshape(-1)
    for k in rng.choice(flat.size, size=min(6, flat.size), replace=False):
        old = flat[k]
        eps = 1e-6
        flat[k] = old + eps
        lp = U.loss_and_grads(params, x, t, wch)[0]
        flat[k] = old - eps
        lm = U.loss_and_grads(params, x, t, wch)[0]
        flat[k] = old
        fd = (lp - lm) / (2 * eps)
        an = g[name].reshape(-1)[k]
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, k, fd, an)
