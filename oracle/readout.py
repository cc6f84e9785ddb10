"""FP64 ridge readout for the reservoir states (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 1 of the paper says only the readout of a reservoir is trained and does
not specify it further.  The reading used throughout the repository: a linear
readout with a bias column, fitted by ridge regression on the states after a
washout, trained on the first half of the remaining samples and scored by the
normalised mean squared error on the second half.  The ridge strength is
beta = beta_rel * trace(Phi^T Phi) / (N + 1) and does not act on the bias.
"""
from __future__ import annotations

import numpy as np


def delay_target(u, delay: int = 5) -> np.ndarray:
    """y_t = u_{t - delay} (first input channel); zero before the input starts."""
    u = np.asarray(u, dtype=np.float64)
    u = u.reshape(u.shape[0], -1)[:, 0]
    y = np.zeros_like(u)
    y[delay:] = u[:-delay] if delay > 0 else u
    return y


def split(T: int, washout: int):
    """Index ranges (train, test) after the washout: first half / second half."""
    n = T - washout
    if n < 4:
        raise ValueError("too few samples after the washout")
    half = washout + n // 2
    return np.arange(washout, half), np.arange(half, T)


def ridge_fit(states, y, beta_rel: float = 1e-6):
    """Solve (Phi^T Phi + beta D) w = Phi^T y with Phi = [states, 1] by Cholesky.

    D is the identity on the state columns and 0 on the bias.  Returns w of
    length N + 1 (bias last)."""
    X = np.asarray(states, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    Phi = np.hstack([X, np.ones((X.shape[0], 1))])
    G = Phi.T @ Phi
    n = G.shape[0]
    beta = beta_rel * np.trace(G) / n
    D = np.eye(n)
    D[-1, -1] = 0.0
    A = G + beta * D
    L = np.linalg.cholesky(A)
    z = np.linalg.solve(L, Phi.T @ y)
    return np.linalg.solve(L.T, z)


def predict(states, w) -> np.ndarray:
    X = np.asarray(states, dtype=np.float64)
    return X @ w[:-1] + w[-1]


def nmse(y_hat, y) -> float:
    y = np.asarray(y, dtype=np.float64)
    return float(np.mean((np.asarray(y_hat) - y) ** 2) / np.var(y))


def evaluate(states, u, washout: int = 100, delay: int = 5, beta_rel: float = 1e-6):
    """Fit on the train half, return (w, nmse_test) for the delay-`delay` task."""
    states = np.asarray(states, dtype=np.float64)
    y = delay_target(u, delay)
    tr, te = split(states.shape[0], washout)
    w = ridge_fit(states[tr], y[tr], beta_rel)
    return w, nmse(predict(states[te], w), y[te])
