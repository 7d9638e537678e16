"""Pins of the preconditioner network's oracle (oracle/cnn.py) against facts that do not
come from the oracle itself: identity / shift kernels, an independent correlation routine,
transposes (dot-product tests), Taylor tests, closed forms."""
import math

import numpy as np
import pytest

from oracle import cnn


def _rng(seed=0):
    return np.random.default_rng(seed)


def test_conv_identity_and_shift_kernels():
    x = _rng(1).standard_normal((2, 7, 9, 4))
    W = np.zeros((3, 3, 4, 4))
    W[1, 1] = np.eye(4)
    assert np.allclose(cnn.conv3x3(x, W, np.zeros(4)), x, atol=0, rtol=0)
    W = np.zeros((3, 3, 4, 4))
    W[0, 1] = np.eye(4)          # reads the row above: y[h] = x[h - 1]
    y = cnn.conv3x3(x, W, np.zeros(4))
    assert np.all(y[:, 0] == 0)
    assert np.allclose(y[:, 1:], x[:, :-1])
    b = np.arange(4.0)
    assert np.allclose(cnn.conv3x3(np.zeros_like(x), W, b), np.broadcast_to(b, x.shape))


def test_conv_matches_independent_correlation():
    from scipy.signal import correlate2d
    rng = _rng(2)
    x = rng.standard_normal((1, 6, 11, 3))
    W = rng.standard_normal((3, 3, 3, 2))
    y = cnn.conv3x3(x, W, np.zeros(2))
    for co in range(2):
        ref = sum(correlate2d(x[0, :, :, ci], W[:, :, ci, co], mode="same", boundary="fill")
                  for ci in range(3))
        assert np.allclose(y[0, :, :, co], ref, rtol=1e-12, atol=1e-12)


def test_conv_backward_is_the_transpose():
    rng = _rng(3)
    x = rng.standard_normal((2, 5, 8, 3))
    W = rng.standard_normal((3, 3, 3, 4))
    gy = rng.standard_normal((2, 5, 8, 4))
    y = cnn.conv3x3(x, W, np.zeros(4))
    gx, gW, gb = cnn.conv3x3_backward(x, W, gy)
    assert abs(np.sum(y * gy) - np.sum(x * gx)) <= 1e-12 * abs(np.sum(y * gy))
    # linear in W too: <conv(x; W), gy> = <W, gW>
    assert abs(np.sum(y * gy) - np.sum(W * gW)) <= 1e-12 * abs(np.sum(y * gy))
    assert np.allclose(gb, gy.sum(axis=(0, 1, 2)))


@pytest.mark.parametrize("H,Wd", [(6, 8), (7, 9)])
def test_pool_and_upsample_transposes(H, Wd):
    rng = _rng(4)
    x = rng.standard_normal((2, H, Wd, 3))
    yp = rng.standard_normal((2, (H + 1) // 2, (Wd + 1) // 2, 3))
    assert abs(np.sum(cnn.pool2(x) * yp) - np.sum(x * cnn.pool2_backward(yp, H, Wd))) < 1e-12
    xc = rng.standard_normal((2, (H + 1) // 2, (Wd + 1) // 2, 3))
    yu = rng.standard_normal((2, H, Wd, 3))
    assert abs(np.sum(cnn.up2(xc, H, Wd) * yu) -
               np.sum(xc * cnn.up2_backward(yu, *xc.shape[1:3]))) < 1e-12
    # averaging a constant image gives the constant away from odd edges
    c = np.full((1, H, Wd, 1), 3.0)
    assert np.allclose(cnn.pool2(c)[0, :H // 2, :Wd // 2, 0], 3.0)


def test_unet_gradient_taylor():
    rng = _rng(5)
    p = cnn.init_params(7, scale=1.0)
    p["dec1.W"] = rng.standard_normal(p["dec1.W"].shape) * 0.1
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1
    x = rng.standard_normal((2, 13, 19, cnn.G))
    gy = rng.standard_normal((2, 13, 19, cnn.G))
    y, a = cnn.unet_forward(x, p)
    gx, g = cnn.unet_backward(gy, p, a)
    dp = {k: rng.standard_normal(v.shape) for k, v in p.items()}
    dx = rng.standard_normal(x.shape)

    def L(pp, xx):
        return float(np.sum(cnn.unet_forward(xx, pp)[0] * gy))
    h = 1e-6
    pp = {k: p[k] + h * dp[k] for k in p}
    pm = {k: p[k] - h * dp[k] for k in p}
    fd = (L(pp, x + h * dx) - L(pm, x - h * dx)) / (2 * h)
    an = sum(float(np.sum(g[k] * dp[k])) for k in p) + float(np.sum(gx * dx))
    assert abs(fd - an) <= 1e-6 * abs(an)


def test_untrained_preconditioner_is_the_diagonal_one():
    rng = _rng(6)
    p = cnn.init_params(11)
    nt, nz, nx = 2 * cnn.G, 9, 14
    r = rng.standard_normal((nt, nz, nx))
    D = rng.uniform(0.5, 2.0, (nz, nx))
    assert np.allclose(cnn.precondition(r, D, p), r * D[None], rtol=0, atol=0)


def test_pack_unpack_shapes_and_averages():
    nt, nz, nx = cnn.G, 6, 10
    s = np.ones((nt, nz, nx)) * np.arange(nt)[:, None, None]
    img = cnn.pack(s)
    assert img.shape == (1, 3, 5, cnn.G)
    assert np.allclose(img[0, :, :, 5], 5.0)
    y = np.zeros_like(img)
    y[0, 1, 2, 3] = 1.0
    z = cnn.unpack(s, y)
    assert np.allclose((z - s)[3, 2:4, 4:6], 1.0)
    assert np.count_nonzero(z - s) == 4


def test_cosine_loss_invariances_and_gradient():
    rng = _rng(8)
    z = rng.standard_normal(50)
    e = rng.standard_normal(50)
    l0 = cnn.cosine_loss(z, e)
    assert cnn.cosine_loss(3.7 * z, e) == pytest.approx(l0, rel=1e-12)
    assert cnn.cosine_loss(-2.0 * e, e) == pytest.approx(0.0, abs=1e-14)
    g = cnn.cosine_loss_grad(z, e)
    dz = rng.standard_normal(50)
    h = 1e-6
    fd = (cnn.cosine_loss(z + h * dz, e) - cnn.cosine_loss(z - h * dz, e)) / (2 * h)
    assert fd == pytest.approx(float(g @ dz), rel=1e-6)


def test_batch_gradient_taylor_and_param_vector_roundtrip():
    rng = _rng(9)
    p = cnn.init_params(3)
    p["dec1.W"] = rng.standard_normal(p["dec1.W"].shape) * 0.05
    v = cnn.param_vector(p)
    q = cnn.params_from_vector(v)
    assert all(np.array_equal(p[k], q[k]) for k in p)
    x = rng.standard_normal((3, 9, 11, cnn.G))
    e = rng.standard_normal((3, 9, 11, cnn.G))
    L, g = cnn.batch_loss_and_grad(x, e, p)
    gv = cnn.param_vector(g)
    dv = rng.standard_normal(v.shape)
    h = 1e-6
    Lp, _ = cnn.batch_loss_and_grad(x, e, cnn.params_from_vector(v + h * dv))
    Lm, _ = cnn.batch_loss_and_grad(x, e, cnn.params_from_vector(v - h * dv))
    assert (Lp - Lm) / (2 * h) == pytest.approx(float(gv @ dv), rel=1e-6)


def test_adam_first_step_closed_form():
    # from zero moments, the bias-corrected step is lr * g / (|g| + eps) ~ lr * sign(g)
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 1e-3])}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    cnn.adam_step(p, g, m, v, t=1, lr=0.01)
    assert np.allclose(p["w"], np.array([1.0, -2.0, 0.5]) - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8))


def test_normalized_network_is_positively_homogeneous():
    rng = _rng(10)
    p = cnn.init_params(12)
    p["dec1.W"] = rng.standard_normal(p["dec1.W"].shape) * 0.1
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1      # biases do not break it
    x = rng.standard_normal((2, 7, 9, cnn.G))
    y1, _, _ = cnn.normalized_forward(x, p)
    y2, _, _ = cnn.normalized_forward(1e-3 * x, p)
    assert np.allclose(1e-3 * y1, y2, rtol=1e-10, atol=0)
    y0, _, _ = cnn.normalized_forward(np.zeros_like(x), p)
    assert np.all(y0 == 0)
