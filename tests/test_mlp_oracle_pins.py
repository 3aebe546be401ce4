"""Pins of the closure MLP oracle: analytic gradients against central finite
differences, a linear special case against least squares, Adam's first step."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = M.init(1) * 0.5 + 0.01 * rng.standard_normal(M.n_params())
    X = rng.standard_normal((7, 85))
    T = rng.standard_normal((7, 9))
    L, g = M.loss_and_grad(w, X, T)
    idx = rng.choice(M.n_params(), 60, replace=False)
    for i in idx:
        h = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (M.loss_and_grad(wp, X, T)[0] - M.loss_and_grad(wm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_parameter_count_and_layout():
    assert M.n_params() == 85 * 64 + 64 + 2 * (64 * 64 + 64) + 64 * 9 + 9
    w = np.arange(M.n_params(), dtype=np.float64)
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = M.unpack(w)
    assert W1[0, 1] == 1 and b1[0] == 85 * 64 and W4.shape == (64, 9) and b4[-1] == M.n_params() - 1


def test_identity_hidden_path_reduces_to_linear_model():
    # with ReLU units fed strictly positive values, the net is affine: check
    # the forward pass against the product of the layer matrices
    rng = np.random.default_rng(2)
    w = np.abs(M.init(3)) * 0.1
    X = np.abs(rng.standard_normal((5, 85)))
    Y, _ = M.forward(w, X)
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = M.unpack(w)
    lin = (((X @ W1 + b1) @ W2 + b2) @ W3 + b3) @ W4 + b4
    assert np.allclose(Y, lin, rtol=1e-12)


def test_adam_first_step_is_signed_lr():
    w = np.zeros(4)
    g = np.array([1.0, -2.0, 0.5, 0.0])
    w1, m, v = M.adam(w, g, np.zeros(4), np.zeros(4), 1, 1e-3)
    assert np.allclose(w1[:3], -1e-3 * np.sign(g[:3]), rtol=1e-6)
    assert w1[3] == 0.0


def test_bf16_rounding_matches_torch_and_ties_to_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(200000) * 3.7).astype(np.float32)
    x[:4] = [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 0.0]  # ties: to even
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    r = M.round_bf16(x)
    assert np.array_equal(r, ref)
    assert r[0] == 1.0 and r[1] == 1.0 + 2.0 ** -6 and r[2] == -1.0


def test_tensor_core_model_reduces_to_exact_network():
    """With rounding switched off, the operand-precision model of the
    tensor-core kernels is the exact network and gradient (pinned above by
    finite differences); with bfloat16 rounding it stays within bfloat16
    error of it."""
    rng = np.random.default_rng(2)
    w = M.init(3)
    X, T = rng.standard_normal((60, 85)), rng.standard_normal((60, 9))
    w32 = w.astype(np.float32).astype(np.float64)
    ident = lambda a: np.asarray(a, dtype=np.float64)  # noqa: E731
    Y0, _ = M.forward(w32, X)
    Y1, _ = M.forward_tc(w, X, rnd=ident)
    assert np.array_equal(Y0, Y1)
    L0, g0 = M.loss_and_grad(w32, X, T)
    L1, g1 = M.loss_and_grad_tc(w, X, T, rnd=ident)
    assert L0 == L1 and np.array_equal(g0, g1)
    L2, g2 = M.loss_and_grad_tc(w, X, T)
    assert abs(L2 - L0) < 1e-2 * L0
    assert np.linalg.norm(g2 - g0) < 5e-2 * np.linalg.norm(g0)
    Y2, _ = M.forward_tc(w, X)
    assert np.linalg.norm(Y2 - Y0) < 2e-2 * np.linalg.norm(Y0)
