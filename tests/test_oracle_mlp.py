"""Pins of the MLP oracle: gradients against central differences, Adam against
its closed-form first step, the forward pass against a hand-built net."""
import numpy as np

from oracle import mlp as M


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    sizes = [5, 7, 6, 3]
    params = M.init_params(sizes, seed=1)
    for W, b in params:
        b[:] = 0.1 * rng.standard_normal(b.shape)
    X = rng.standard_normal((11, 5))
    T = rng.standard_normal((11, 3))
    w = np.array([1.0, 2.0, 0.5])
    _, grads = M.loss_and_grads(params, X, T, w)
    h = 1e-6
    for l in range(len(params)):
        for q in range(2):
            P = params[l][q]
            it = np.nditer(P, flags=["multi_index"])
            for _ in range(min(P.size, 12)):
                idx = it.multi_index
                old = P[idx]
                P[idx] = old + h
                lp, _ = M.loss_and_grads(params, X, T, w)
                P[idx] = old - h
                lm, _ = M.loss_and_grads(params, X, T, w)
                P[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - grads[l][q][idx]) <= 1e-7 * max(1.0, abs(fd))
                it.iternext()


def test_forward_is_affine_tanh_chain():
    params = [[np.array([[2.0, -1.0]]), np.array([0.5])], [np.array([[3.0]]), np.array([-1.0])]]
    X = np.array([[0.3, 0.1]])
    y, _, _ = M.forward(params, X)
    assert np.isclose(y[0, 0], 3.0 * np.tanh(2 * 0.3 - 0.1 + 0.5) - 1.0)


def test_adam_first_step_closed_form():
    """After one step from zero moments: p -= lr * g / (|g| + eps)."""
    params = [[np.array([[1.0, -2.0]]), np.array([0.5])]]
    grads = [[np.array([[0.3, -4.0]]), np.array([1e-3])]]
    st = {}
    M.adam_step(params, grads, st, lr=0.01, eps=1e-8)
    assert np.allclose(params[0][0], [[1.0 - 0.01 * 0.3 / (0.3 + 1e-8), -2.0 + 0.01 * 4.0 / (4.0 + 1e-8)]])
    assert np.allclose(params[0][1], [0.5 - 0.01 * 1e-3 / (1e-3 + 1e-8)])


def test_adam_bias_correction_over_many_steps():
    """Under a constant gradient g the bias-corrected moments are exactly g
    and g^2 at every step t (m_t = (1 - b1^t) g, v_t = (1 - b2^t) g^2), so every
    step moves a parameter by lr g / (|g| + eps).  A wrong exponent of b1^t or
    b2^t changes the step size after the first step and fails this."""
    g = np.array([[0.3, -4.0, 2e-2]])
    gb = np.array([-0.7])
    params = [[np.array([[1.0, -2.0, 0.25]]), np.array([0.5])]]
    st = {}
    lr, eps = 0.01, 1e-8
    for t in range(1, 8):
        w0, b0 = params[0][0].copy(), params[0][1].copy()
        M.adam_step(params, [[g, gb]], st, lr=lr, b1=0.8, b2=0.95, eps=eps)
        assert np.allclose(params[0][0] - w0, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
        assert np.allclose(params[0][1] - b0, -lr * gb / (np.abs(gb) + eps), rtol=1e-12, atol=0)
    assert st["t"] == 7


def test_training_reduces_loss_on_a_smooth_map():
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, size=(256, 3))
    T = np.stack([np.sin(X[:, 0]) * X[:, 1], X[:, 2] ** 2], axis=1)
    params = M.init_params([3, 32, 32, 2], seed=2)
    st = {}
    l0, _ = M.loss_and_grads(params, X, T)
    for _ in range(300):
        _, g = M.loss_and_grads(params, X, T)
        M.adam_step(params, g, st, lr=3e-3)
    l1, _ = M.loss_and_grads(params, X, T)
    assert l1 < 0.1 * l0
