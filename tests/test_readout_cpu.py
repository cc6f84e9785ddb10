"""The differentiable readout objective (paper_2312_01121_b300.autograd.
ridge_objective, torch on the CPU) against the oracle's ridge readout
(oracle/readout.py).  No GPU needed.

ridge_objective(states, y, washout, beta) = mean_t (Phi_t w - y_t)^2 +
beta |w_states|^2 at its own minimiser w.  Its normal equations are
(Phi^T Phi + n beta D) w = Phi^T y (n samples), the oracle's with
beta_rel = n beta (N + 1) / trace(Phi^T Phi).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def problem(T=400, N=20, seed=3):
    g = np.random.default_rng(seed)
    X = g.uniform(-1.0, 1.0, (T, N)).astype(np.float32)
    y = X.astype(np.float64) @ g.standard_normal(N) + 0.3 + 0.1 * g.standard_normal(T)
    return X, y


def oracle_objective(X, y, washout, beta):
    from oracle import readout
    Xt, yt = X[washout:].astype(np.float64), y[washout:]
    n, N = Xt.shape
    Phi = np.hstack([Xt, np.ones((n, 1))])
    beta_rel = n * beta * (N + 1) / np.trace(Phi.T @ Phi)
    w = readout.ridge_fit(Xt, yt, beta_rel)
    r = readout.predict(Xt, w) - yt
    return float(np.mean(r * r) + beta * np.sum(w[:-1] ** 2)), w, r


@pytest.mark.parametrize("beta", [1e-6, 1e-3, 1e-1])
def test_ridge_objective_value_equals_oracle_fit(beta):
    from paper_2312_01121_b300.autograd import ridge_objective
    X, y = problem()
    L_o, _, _ = oracle_objective(X, y, 50, beta)
    L = ridge_objective(torch.from_numpy(X), torch.from_numpy(y), 50, beta).item()
    assert abs(L - L_o) <= 1e-10 * L_o


def test_ridge_objective_gradient_is_the_envelope_gradient():
    """Differentiating through the solve gives the gradient at fixed w
    (envelope theorem): dL/dstates[t] = 2 r_t w_states / n for t >= washout,
    0 before it; r and w from the oracle's fit."""
    from paper_2312_01121_b300.autograd import ridge_objective
    X, y = problem(T=300, N=12, seed=5)
    washout, beta = 40, 1e-3
    _, w, r = oracle_objective(X, y, washout, beta)
    Xt = torch.from_numpy(X.astype(np.float64)).requires_grad_(True)
    ridge_objective(Xt, torch.from_numpy(y), washout, beta).backward()
    n = X.shape[0] - washout
    expect = np.zeros_like(X, dtype=np.float64)
    expect[washout:] = 2.0 * np.outer(r, w[:-1]) / n
    assert np.max(np.abs(Xt.grad.numpy() - expect)) <= 1e-10 * np.max(np.abs(expect))
