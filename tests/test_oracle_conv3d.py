"""The oracle's conv-net gradient against central finite differences."""
import numpy as np

from oracle import conv3d


def test_conv_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    cin, cout = [2, 3, 3], [3, 3, 1]
    params = [(rng.normal(size=(co, ci, 3, 3, 3)) * 0.4, rng.normal(size=co) * 0.1) for ci, co in zip(cin, cout)]
    x = rng.normal(size=(2, 2, 3, 4, 2))
    t = rng.uniform(size=(2, 1, 3, 4, 2))
    loss, grads = conv3d.loss_and_grad(params, x, t)
    flat = np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])
    g = conv3d.flatten(grads)
    eps = 1e-6
    idx = rng.choice(flat.size, size=40, replace=False)
    for i in idx:
        fp = flat.copy(); fp[i] += eps
        fm = flat.copy(); fm[i] -= eps
        lp = conv3d.loss_and_grad(conv3d.unflatten(fp, cin, cout), x, t)[0]
        lm = conv3d.loss_and_grad(conv3d.unflatten(fm, cin, cout), x, t)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i]), abs(fd)), (i, fd, g[i])


def test_conv_is_cross_correlation_with_zero_padding():
    # a single tap reproduces a shifted copy of the input (zero outside)
    x = np.arange(2 * 3 * 4, dtype=float).reshape(1, 1, 2, 3, 4)
    w = np.zeros((1, 1, 3, 3, 3))
    w[0, 0, 1, 1, 2] = 1.0                 # tap (dz, dy, dx) = (0, 0, +1)
    y = conv3d.conv3d_same(x, w, np.zeros(1))
    assert np.array_equal(y[..., :-1], x[..., 1:]) and np.all(y[..., -1] == 0)
