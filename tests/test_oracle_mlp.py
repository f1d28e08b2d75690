"""Pins of the warm-start network oracle against facts it does not compute
itself: hand-worked bfloat16 roundings, central finite differences of the
loss, closed forms of degenerate networks and the first Adam step."""
import numpy as np

from oracle import mlp as M


def _params(rng, n_in=5, width=7, scale=0.5):
    return M.Params(rng.standard_normal((width, n_in)) * scale, rng.standard_normal(width) * 0.1,
                    rng.standard_normal((width, width)) * scale / np.sqrt(width),
                    rng.standard_normal(width) * 0.1,
                    rng.standard_normal((1, width)) * scale, rng.standard_normal(1) * 0.1,
                    rng.standard_normal((1, n_in)) * scale)


def test_bf16_rounding_hand_values():
    # bfloat16 keeps 7 fraction bits: neighbours of 1 are 1 - 2^-8 and 1 + 2^-7
    v = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -20,
                  -(1 + 2.0 ** -8), 3.0, 0.0, 2.0 ** -130, 65280.0 + 128.0])
    want = np.array([1.0, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, -1.0, 3.0, 0.0,
                     2.0 ** -130, 65536.0])
    got = M.bf16_round(v)
    assert np.array_equal(got, want)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    P = _params(rng)
    X = rng.standard_normal((11, 5))
    t = rng.standard_normal(11)
    _, G = M.loss_and_grad(P, X, t, bf16=False)
    theta = P.flat()
    g = G.flat()
    eps = 1e-6
    for k in rng.choice(theta.size, 40, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        Lp, _ = M.loss_and_grad(M.Params.from_flat(tp, 5, 7), X, t, bf16=False)
        Lm, _ = M.loss_and_grad(M.Params.from_flat(tm, 5, 7), X, t, bf16=False)
        fd = (Lp - Lm) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_bf16_gradient_is_the_gradient_at_the_rounded_weights():
    rng = np.random.default_rng(2)
    P = _params(rng)
    X = rng.standard_normal((9, 5))
    t = rng.standard_normal(9)
    L1, G1 = M.loss_and_grad(P, X, t, bf16=True)
    R = M.Params(M.bf16_round(P.W1), P.b1, M.bf16_round(P.W2), P.b2, M.bf16_round(P.W3), P.b3,
                 P.WL)
    L2, G2 = M.loss_and_grad(R, X, t, bf16=False)
    assert L1 == L2
    assert np.array_equal(G1.flat(), G2.flat())
    # and rounding changed something (the test is not vacuous)
    assert not np.array_equal(M.bf16_round(P.W2), P.W2)


def test_degenerate_networks_closed_form():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((6, 4))
    t = rng.standard_normal(6)
    w = 3
    # all weights zero: y = b3, dL/db3 = mean(b3 - t), dL/dW3 = mean(y - t) tanh(b2)
    P = M.Params(np.zeros((w, 4)), np.full(w, 0.2), np.zeros((w, w)), np.array([0.1, -0.3, 0.5]),
                 np.zeros((1, w)), np.array([0.7]))
    y, _ = M.forward(P, X)
    assert np.allclose(y, 0.7, rtol=0, atol=0)
    L, G = M.loss_and_grad(P, X, t)
    assert np.isclose(L, 0.5 * np.mean((0.7 - t) ** 2), rtol=1e-15)
    assert np.isclose(G.b3[0], np.mean(0.7 - t), rtol=1e-14)
    assert np.allclose(G.W3[0], np.mean(0.7 - t) * np.tanh([0.1, -0.3, 0.5]), rtol=1e-14)
    assert np.array_equal(G.W1, np.zeros((w, 4)))
    # the linear skip alone: y = WL x + b3, dL/dWL = mean((y - t) x)
    P.WL = np.array([[0.5, -1.0, 0.0, 2.0]])
    y, _ = M.forward(P, X)
    assert np.allclose(y, X @ P.WL[0] + 0.7, rtol=1e-14)
    _, G = M.loss_and_grad(P, X, t)
    assert np.allclose(G.WL[0], ((X @ P.WL[0] + 0.7 - t)[:, None] * X).mean(0), rtol=1e-13)
    P.WL = np.zeros((1, 4))
    # W2 = 0: y = W3 tanh(b2) + b3 whatever the input
    P.W3 = np.array([[0.5, 0.25, -1.0]])
    y, _ = M.forward(P, X)
    assert np.allclose(y, 0.5 * np.tanh(0.1) + 0.25 * np.tanh(-0.3) - np.tanh(0.5) + 0.7,
                       rtol=1e-15)


def test_first_adam_step_moves_by_lr_against_the_gradient_sign():
    g = np.array([3.0, -2e-3, 1e-1, -7.0])
    th, m, v = M.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=1e-12)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=1e-9)
    # second step with the same gradient: still lr (moments equal g, g^2)
    th2, _, _ = M.adam_step(th, g, m, v, 2, lr=0.01, eps=1e-12)
    assert np.allclose(th2, -0.02 * np.sign(g), rtol=1e-9)
