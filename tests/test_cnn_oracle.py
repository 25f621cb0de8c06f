"""Pins of the learned form's FP64 oracle (oracle/cnn_oracle.py): the
convolution against a library cross-correlation, every gradient against
central finite differences, Adam's first step, and the feature map's range."""
import numpy as np
import pytest

from oracle import cnn_oracle as co

scipy_signal = pytest.importorskip("scipy.signal")


def test_conv3x3_matches_library_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 7, 9))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = co.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(scipy_signal.correlate2d(x[n, c], w[o, c], mode="same", boundary="fill")
                             for c in range(3))
            assert np.allclose(y[n, o], ref, atol=1e-12)


def _num_grad(f, a, h=1e-6):
    g = np.zeros_like(a)
    it = np.nditer(a, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        old = a[i]
        a[i] = old + h
        fp = f()
        a[i] = old - h
        fm = f()
        a[i] = old
        g[i] = (fp - fm) / (2 * h)
    return g


def test_conv3x3_backward_is_the_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 3, 5, 6))
    w = rng.standard_normal((2, 3, 3, 3))
    b = rng.standard_normal(2)
    r = rng.standard_normal((2, 2, 5, 6))            # loss = sum(r * y)
    dx, dw, db = co.conv3x3_backward(x, w, r)
    f = lambda: float(np.sum(r * co.conv3x3(x, w, b)))
    assert np.allclose(dx, _num_grad(f, x), atol=1e-6)
    assert np.allclose(dw, _num_grad(f, w), atol=1e-6)
    assert np.allclose(db, _num_grad(f, b), atol=1e-6)


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    params = co.init_params(4, channels=(5, 4, 4, 1))
    x = rng.standard_normal((1, 5, 6, 5)) * 0.5
    t = rng.uniform(0.0, 1.0, (1, 6, 5))
    loss, grads = co.loss_and_grads(params, x, t)
    for li, (w, b) in enumerate(params):
        f = lambda: co.loss_and_grads(params, x, t)[0]
        assert np.allclose(grads[li][0], _num_grad(f, w), atol=1e-7, rtol=1e-5), li
        assert np.allclose(grads[li][1], _num_grad(f, b), atol=1e-7, rtol=1e-5), li
    assert loss > 0


def test_head_range_and_zero_loss_at_target():
    params = co.init_params(5, channels=(5, 4, 1))
    x = np.random.default_rng(6).standard_normal((2, 5, 4, 4))
    rho, _ = co.forward(params, x)
    assert np.all(rho >= 1e-3) and np.all(rho < 1.0)
    loss, _ = co.loss_and_grads(params, x, rho[:, 0].copy())
    assert loss == 0.0


def test_adam_first_step_and_convergence():
    p, m, v = np.array([1.0, -2.0]), np.zeros(2), np.zeros(2)
    g = np.array([0.3, -7.0])
    p1, m, v = co.adam_step(p.copy(), g, m, v, 1, lr=0.01)
    # bias correction makes the first step lr * sign(g) (up to the eps term)
    assert np.allclose(p1 - p, -0.01 * np.sign(g), atol=1e-9)
    x, m, v = np.array([10.0]), np.zeros(1), np.zeros(1)
    for t in range(1, 3001):
        x, m, v = co.adam_step(x, 2 * (x - 3.0), m, v, t, lr=0.05)
    assert abs(x[0] - 3.0) < 1e-2


def test_features_range_and_max():
    rng = np.random.default_rng(7)
    eb = rng.uniform(0, 1, (4, 6, 5))
    f = co.features(eb)
    assert f.shape == (5, 6, 5)
    assert np.all(f <= np.log10(1 + 1e-4) / 4 + 1e-15) and np.all(f >= -1.0)
    e = eb.sum(0)
    assert np.isclose(f[0].max(), np.log10(1 + 1e-4) / 4)
    assert np.isclose(f[0][np.unravel_index(np.argmin(e), e.shape)],
                      np.log10(e.min() / e.max() + 1e-4) / 4)


def test_loss_weight_closed_forms():
    # channel 0 = log10(E/max + 1e-4)/4: the brightest pixel has weight 1, an empty pixel the floor
    x = np.zeros((1, 5, 1, 3))
    x[0, 0, 0] = [np.log10(1 + 1e-4) / 4, np.log10(0.5 + 1e-4) / 4, np.log10(1e-4) / 4]
    w = co.loss_weights(x)[0, 0, 0]
    assert np.allclose(w, [1.0, co.WEIGHT_FLOOR + (1 - co.WEIGHT_FLOOR) * 0.5, co.WEIGHT_FLOOR], atol=1e-12)
    # the weighted loss of a uniform error d is d^2 times the mean weight
    params = co.init_params(9, channels=(5, 3, 1))
    rho, _ = co.forward(params, x)
    loss, _ = co.loss_and_grads(params, x, rho[:, 0] - 0.1)
    assert np.isclose(loss, 0.01 * w.mean())
