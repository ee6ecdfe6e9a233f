"""The oracle's conv-net gradient against central finite differences."""
import numpy as np
import pytest

from oracle import conv3d


@pytest.mark.parametrize("weighted", [False, True])
def test_conv_gradient_matches_finite_differences(weighted):
    rng = np.random.default_rng(0)
    cin, cout = [2, 3, 3], [3, 3, 1]
    params = [(rng.normal(size=(co, ci, 3, 3, 3)) * 0.4, rng.normal(size=co) * 0.1) for ci, co in zip(cin, cout)]
    x = rng.normal(size=(2, 2, 3, 4, 2))
    t = rng.uniform(size=(2, 1, 3, 4, 2))
    w = rng.uniform(size=t.shape) * (rng.uniform(size=t.shape) < 0.4) if weighted else None
    loss, grads = conv3d.loss_and_grad(params, x, t, w)
    flat = np.concatenate([np.concatenate([wl.ravel(), bl.ravel()]) for wl, bl in params])
    g = conv3d.flatten(grads)
    eps = 1e-6
    idx = rng.choice(flat.size, size=40, replace=False)
    for i in idx:
        fp = flat.copy(); fp[i] += eps
        fm = flat.copy(); fm[i] -= eps
        lp = conv3d.loss_and_grad(conv3d.unflatten(fp, cin, cout), x, t, w)[0]
        lm = conv3d.loss_and_grad(conv3d.unflatten(fm, cin, cout), x, t, w)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i]), abs(fd)), (i, fd, g[i])


def test_face_flux_term_is_the_squared_flux_error():
    """mean((1 + w)(y - t)^2) with w = T_R^2 adds (T_R (y - t))^2, the squared
    error of the outward flux T_R (p_c - g) through the face (g cancels)."""
    rng = np.random.default_rng(3)
    cin, cout = [1, 2], [2, 1]
    params = [(rng.normal(size=(co, ci, 3, 3, 3)) * 0.3, np.zeros(co)) for ci, co in zip(cin, cout)]
    x = rng.normal(size=(1, 1, 2, 2, 2))
    t = rng.uniform(size=(1, 1, 2, 2, 2))
    TR = 0.7
    w = np.zeros_like(t)
    w[0, 0, 0, 0, 0] = TR ** 2
    y = conv3d.forward(params, x)[-1]
    g = 0.3                                       # any Robin datum of the face
    flux_err = TR * (y[0, 0, 0, 0, 0] - g) - TR * (t[0, 0, 0, 0, 0] - g)
    expect = (np.sum((y - t) ** 2) + flux_err ** 2) / y.size
    assert abs(conv3d.loss_and_grad(params, x, t, w)[0] - expect) <= 1e-14


def test_conv_is_cross_correlation_with_zero_padding():
    # a single tap reproduces a shifted copy of the input (zero outside)
    x = np.arange(2 * 3 * 4, dtype=float).reshape(1, 1, 2, 3, 4)
    w = np.zeros((1, 1, 3, 3, 3))
    w[0, 0, 1, 1, 2] = 1.0                 # tap (dz, dy, dx) = (0, 0, +1)
    y = conv3d.conv3d_same(x, w, np.zeros(1))
    assert np.array_equal(y[..., :-1], x[..., 1:]) and np.all(y[..., -1] == 0)
