"""Pins of the FP64 network oracle (oracle/mlp.py): back-propagation against
central finite differences of the loss (with the bfloat16 rounding points
switched off so the loss is smooth), and the closed-form derivatives of the
two losses."""
import numpy as np
import pytest

from oracle import mlp


@pytest.fixture
def smooth(monkeypatch):
    monkeypatch.setattr(mlp, "bf16", lambda a: np.asarray(a, dtype=np.float64))


@pytest.mark.parametrize("kind,din,hid,dout", [("bce", 12, 16, 1), ("mae", 12, 16, 10)])
def test_backprop_matches_finite_differences(smooth, kind, din, hid, dout):
    rng = np.random.default_rng(3)
    theta = mlp.init_params(din, hid, dout, rng)
    theta += rng.normal(0, 0.05, theta.shape)  # nonzero biases too
    u = rng.normal(size=(20, din))
    y = (rng.uniform(size=20) < 0.5).astype(float) if kind == "bce" else rng.normal(size=(20, dout))
    loss, g = mlp.loss_and_grad(theta, u, y, din, hid, dout, kind)
    idx = rng.choice(theta.size, 60, replace=False)
    for i in idx:
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, u, y, din, hid, dout, kind)[0] - mlp.loss_and_grad(tm, u, y, din, hid, dout, kind)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_loss_derivatives_closed_form():
    # d/dz [softplus(z) - y z] = sigmoid(z) - y ; d/do |o - t| = sign(o - t)
    z = np.linspace(-5, 5, 11)
    for y in (0.0, 1.0):
        h = 1e-6
        f = lambda v: np.logaddexp(0.0, v) - y * v
        fd = (f(z + h) - f(z - h)) / (2 * h)
        np.testing.assert_allclose(fd, 1 / (1 + np.exp(-z)) - y, atol=1e-8)


def test_bf16_rounding():
    # bfloat16 keeps 8 significant bits: 1 + 2^-8 rounds to 1 (tie to even), 1 + 3 * 2^-8 to 1 + 2^-6
    assert mlp.bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert mlp.bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    assert mlp.bf16(np.array([3.0]))[0] == 3.0


@pytest.mark.parametrize("kind", ["mae", "mae_theta"])
def test_residual_wide_backprop_matches_finite_differences(smooth, kind):
    """arch 1 (Sec. 4.2.1: residual blocks, wide concatenation) and the
    second-stage theta loss (Sec. 4.2.2)."""
    rng = np.random.default_rng(8)
    din, hid, dout, n = 7, 8, 5, 16
    theta = mlp.init_params(din, hid, dout, rng, arch=1)
    theta += rng.normal(0, 0.05, theta.shape)
    u = rng.normal(size=(n, din))
    y = rng.normal(0, 1.0, size=(n, dout))
    z = rng.dirichlet(np.ones(dout), size=n)
    th_t = rng.uniform(0.1, 0.9, size=n)
    kw = dict(arch=1, wth=0.7, z=z, th_target=th_t)
    loss, g = mlp.loss_and_grad(theta, u, y, din, hid, dout, kind, **kw)
    assert g.size == mlp.n_params(din, hid, dout, arch=1)
    for i in rng.choice(theta.size, 80, replace=False):
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, u, y, din, hid, dout, kind, **kw)[0] -
              mlp.loss_and_grad(tm, u, y, din, hid, dout, kind, **kw)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_rr_theta_ift_matches_finite_differences_and_binary_closed_form():
    rng = np.random.default_rng(2)
    for _ in range(20):
        nc = int(rng.integers(2, 9))
        z = rng.dirichlet(np.ones(nc))
        lnK = rng.normal(0, 1.5, nc)
        lnK[0], lnK[1] = abs(lnK[0]) + 0.1, -abs(lnK[1]) - 0.1  # K brackets 1
        th, d = mlp.rr_theta(z, lnK)
        for i in range(nc):
            h = 1e-6
            lp, lm = lnK.copy(), lnK.copy()
            lp[i] += h
            lm[i] -= h
            fd = (mlp.rr_theta(z, lp)[0] - mlp.rr_theta(z, lm)[0]) / (2 * h)
            assert d[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)
        if nc == 2:  # binary closed form theta = -(a z1 + b z2) / (a b), a = K1 - 1, b = K2 - 1
            a, b = np.exp(lnK) - 1.0
            assert th == pytest.approx(-(a * z[0] + b * z[1]) / (a * b), rel=1e-12)
