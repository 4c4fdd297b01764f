"""Pins of the rank-rule and predictor oracle (oracle/learned_ref.py)
against hand-worked values, the matrix rank, finite differences and the
closed form of Adam's first step."""
import numpy as np

from oracle import learned_ref as R


def test_rank_rule_by_hand():
    # squares 9, 4, 1, 0.25 (total 14.25); discarded energy after r = 1, 2, 3, 4:
    # 5.25, 1.25, 0.25, 0.  tol 0.3 -> threshold 0.09 * 14.25 = 1.2825 -> r = 2
    sig = np.array([[3.0, 2.0, 1.0, 0.5], [0.0, 0.0, 0.0, 0.0]])
    assert list(R.rank_rule(sig, 0.3, 4)) == [2, 0]
    assert list(R.rank_rule(sig, 0.3, 1)) == [1, 0]      # capped
    assert list(R.rank_rule(sig, 0.0, 4)) == [4, 0]      # nothing may be dropped
    assert list(R.rank_rule(sig, 0.999, 4)) == [1, 0]


def test_rank_rule_limit_is_the_matrix_rank():
    # Section 2 multi-rank: with tol -> 0 the rule returns the rank of the slice
    g = np.random.default_rng(0)
    for r in (1, 3, 7):
        M = g.standard_normal((20, r)) @ g.standard_normal((r, 15))
        s = np.linalg.svd(M, compute_uv=False)
        s[r:] = 0.0                                       # exact zeros past the rank
        assert R.rank_rule(s[None, :], 1e-12, 15)[0] == np.linalg.matrix_rank(M) == r


def test_features_by_hand():
    sig = np.zeros((1, 17))
    sig[0, :3] = [10.0, 1.0, 0.1]
    f = R.features(sig)
    assert f.shape == (1, 16)
    assert np.allclose(f[0, :2], [-1 / 8, -2 / 8]) and np.all(f[0, 2:] == -1.0)


def test_backprop_matches_finite_differences():
    g = np.random.default_rng(1)
    theta = 0.3 * g.standard_normal(R.N_PARAMS)
    X = g.standard_normal((7, R.N_IN))
    T = g.standard_normal((7, R.N_OUT))
    _, grad = R.loss_and_grad(theta, X, T)
    idx = g.choice(R.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, np.arange(R.N_PARAMS - 258, R.N_PARAMS)])   # all of W3, b3
    h = 1e-6
    for i in idx:
        tp_, tm = theta.copy(), theta.copy()
        tp_[i] += h
        tm[i] -= h
        fd = (R.loss_and_grad(tp_, X, T)[0] - R.loss_and_grad(tm, X, T)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_linear_regime_and_zero_output_layer():
    g = np.random.default_rng(2)
    theta = np.abs(g.standard_normal(R.N_PARAMS)) * 0.1     # all positive: no ReLU clips
    X = np.abs(g.standard_normal((5, R.N_IN)))
    W1, b1, W2, b2, W3, b3 = R.unpack(theta)
    y, _, _ = R.forward(theta, X)
    lin = ((X @ W1.T + b1) @ W2.T + b2) @ W3.T + b3
    np.testing.assert_allclose(y, lin, rtol=1e-13)
    theta0 = theta.copy()
    theta0[R.N_PARAMS - 258:R.N_PARAMS - 2] = 0.0           # W3 = 0
    _, grad = R.loss_and_grad(theta0, X, g.standard_normal((5, 2)))
    assert np.all(grad[:R.N_PARAMS - 258] == 0.0)


def test_adam_first_step_moves_by_lr_times_sign():
    g = np.array([3.0, -0.5, 1e-3])
    th, m, v = R.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, 0.01)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-4)
