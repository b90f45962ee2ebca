"""The CPU reference of the cost model against finite differences and a
closed form (no GPU)."""
import numpy as np

from oracle import mlp as M


def _random(hidden, n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, M.D)) * 3 + 1
    t = rng.normal(size=n)
    w = np.zeros(2 * M.D + M.D * hidden + 2 * hidden + 1)
    w[:M.D] = x.mean(axis=0)
    w[M.D:2 * M.D] = x.std(axis=0)
    w[2 * M.D:] = rng.normal(size=w.size - 2 * M.D) * 0.5
    return x, t, w


def test_gradient_matches_finite_differences():
    x, t, w = _random(8, 50, 0)
    g, L = M.grad(x, t, w, 8)
    assert abs(L - M.loss(x, t, w, 8)) < 1e-12
    eps = 1e-6
    for k in range(2 * M.D, w.size):
        wp, wm = w.copy(), w.copy()
        wp[k] += eps
        wm[k] -= eps
        fd = (M.loss(x, t, wp, 8) - M.loss(x, t, wm, 8)) / (2 * eps)
        assert abs(fd - g[k]) < 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])
    assert not g[:2 * M.D].any()


def test_single_active_unit_is_linear_regression():
    # with one hidden unit that is active everywhere the model is linear:
    # y = b2 + w2 (xs W1 + b1), and the loss gradient w.r.t. b2 is 2 mean(r)
    rng = np.random.default_rng(1)
    n = 40
    x = rng.normal(size=(n, M.D))
    t = rng.normal(size=n)
    w = np.zeros(2 * M.D + M.D + 3)
    w[M.D:2 * M.D] = 1.0
    W1 = rng.normal(size=M.D) * 0.01
    w[2 * M.D:3 * M.D] = W1
    w[3 * M.D] = 100.0      # b1: keeps the unit active
    w[3 * M.D + 1] = 0.5    # w2
    w[3 * M.D + 2] = -1.0   # b2
    y = -1.0 + 0.5 * (x @ W1 + 100.0)
    assert np.allclose(M.forward(x, w, 1), y)
    g, L = M.grad(x, t, w, 1)
    r = y - t
    assert np.isclose(L, np.mean(r ** 2))
    assert np.isclose(g[-1], 2 * r.mean())                       # b2
    assert np.isclose(g[3 * M.D + 1], 2 * np.mean(r * (x @ W1 + 100.0)))  # w2
