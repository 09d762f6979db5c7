"""Pins of the FP64 reference network (oracle/nn.py): central finite
differences of the loss for every parameter tensor and for the input, and
layer identities against direct loops."""
import numpy as np
import pytest

from oracle import nn


def _loss(p, x, t, levels):
    y, _ = nn.forward(p, x, levels)
    return nn.mse(y, t)


@pytest.mark.parametrize("levels,base", [(2, 3), (3, 2)])
def test_gradients_match_finite_differences(levels, base):
    rng = np.random.default_rng(7)
    x = rng.standard_normal((2, 8, 8, 3))
    t = rng.standard_normal((2, 8, 8, 3))
    p = nn.init_params(1, base=base, levels=levels)
    for k in p:  # non-zero biases so every term is exercised
        if k.endswith(".b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1
    y, cache = nn.forward(p, x, levels)
    g = nn.backward(p, cache, y, t, levels)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = _loss(p, x, t, levels)
            flat[i] = old - h
            lm = _loss(p, x, t, levels)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert g[k].reshape(-1)[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), (k, i)


def test_conv3x3_matches_direct_loops():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1, 5, 6, 2))
    w = rng.standard_normal((3, 3, 2, 4))
    b = rng.standard_normal(4)
    y = nn.conv3x3(x, w, b)
    for i in range(5):
        for j in range(6):
            for o in range(4):
                s = b[o]
                for dy in range(3):
                    for dx in range(3):
                        ii, jj = i + dy - 1, j + dx - 1
                        if 0 <= ii < 5 and 0 <= jj < 6:
                            s += (x[0, ii, jj, :] * w[dy, dx, :, o]).sum()
                assert y[0, i, j, o] == pytest.approx(s, abs=1e-12)


def test_pool_and_upsample_are_adjoint_up_to_scale():
    """<up(a), b> = 4 <a, pool(b)>: nearest upsampling is 4x the adjoint of
    2x2 averaging."""
    rng = np.random.default_rng(5)
    a = rng.standard_normal((1, 3, 4, 2))
    b = rng.standard_normal((1, 6, 8, 2))
    assert (nn.up2(a) * b).sum() == pytest.approx(4 * (a * nn.pool2(b)).sum(), rel=1e-12)


def test_adam_first_step_moves_by_lr():
    """With bias correction the first Adam step is -lr * sign(g) (|g| >> eps)."""
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    nn.adam_step(p, g, {}, lr=0.01)
    np.testing.assert_allclose(p["w"], [0.99, -1.99, 2.99], rtol=0, atol=2e-7)  # eps/|g| = 1e-5


def test_parameter_count_of_the_warm_start_network():
    """4 levels, 32 base channels, 3 inputs, 3 outputs."""
    p = nn.init_params(0)
    n = sum(v.size for v in p.values())
    assert n == 1946947  # sum of 9 ci co + co over the conv3x3 layers, plus 32 x 3 + 3
