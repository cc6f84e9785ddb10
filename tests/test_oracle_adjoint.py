"""Pins of the oracle's discrete adjoint: central finite differences of the
oracle's own forward run (FP64), independent of the adjoint code."""
import numpy as np
import pytest

import oracle
from oracle import readout
from paper_2312_01121_b300 import inputs


def _system(N, T, seed, n_in=1):
    return (inputs.coupling_paper(N, seed), inputs.input_weights(N, n_in, seed),
            inputs.random_unit_states(N, seed), inputs.input_series(T, n_in, seed))


def _fd(f, x, h):
    return (f(x + h) - f(x - h)) / (2.0 * h)


@pytest.mark.parametrize("N,T,comp", [(1, 5, 0), (5, 6, 0), (16, 8, 0), (7, 5, 2)])
def test_adjoint_matches_finite_differences(N, T, comp):
    P = oracle.OracleParams(substeps=10, A_cp=80.0, A_in=40.0, alpha=0.02, component=comp)
    W, w_in, m0, u = _system(N, T, seed=N)
    G = np.random.default_rng(N).standard_normal((T, N))
    g = oracle.adjoint(P, W, w_in, m0, u, G)

    def L(P_=P, w_=w_in, m_=m0):
        return float(np.sum(G * oracle.run(P_, W, w_, m_, u)[1]))

    def close(a, b, tol=1e-6):
        assert abs(a - b) <= tol * max(abs(b), 1e-12 * abs(L())), (a, b)

    close(g["A_cp"], _fd(lambda a: L(P.replace(A_cp=a)), P.A_cp, 1e-6 * P.A_cp))
    close(g["current"], _fd(lambda a: L(P.replace(I=a)), P.I, 1e-6 * P.I))
    for k in range(min(N, 3)):
        def fw(a, k=k):
            w2 = w_in.copy()
            w2[k, 0] = a
            return L(w_=w2)
        close(g["w_in"][k, 0], _fd(fw, w_in[k, 0], 1e-6))
    for c, k in [(0, 0), (1, N - 1), (2, N // 2)]:
        def fm(a, c=c, k=k):
            m2 = m0.copy()
            m2[c, k] = a
            return L(m_=m2)
        close(g["m0"][c, k], _fd(fm, m0[c, k], 1e-6))


def test_adjoint_of_readout_loss_envelope():
    """Loss = ridge objective at the refitted readout (fixed beta).  By the
    envelope theorem its gradient is the adjoint of dL/dstates taken at the
    fitted weights; checked against FD that refits per perturbation."""
    N, T, washout = 6, 40, 10
    P = oracle.OracleParams(substeps=5, A_cp=60.0, A_in=80.0, alpha=0.05)
    W, w_in, m0, u = _system(N, T, seed=3)
    y = readout.delay_target(u, 2)
    tr = np.arange(washout, T)
    beta = 1e-3

    def objective(states):
        X = np.hstack([states[tr], np.ones((len(tr), 1))])
        D = np.eye(N + 1)
        D[-1, -1] = 0.0
        w = np.linalg.solve(X.T @ X / len(tr) + beta * D, X.T @ y[tr] / len(tr))
        r = X @ w - y[tr]
        return float(np.mean(r ** 2) + beta * np.sum(w[:-1] ** 2)), w

    def L(P_=P):
        return objective(oracle.run(P_, W, w_in, m0, u)[1])[0]

    _, st = oracle.run(P, W, w_in, m0, u)
    val, w = objective(st)
    G = np.zeros((T, N))
    G[tr] = 2.0 / len(tr) * (np.hstack([st[tr], np.ones((len(tr), 1))]) @ w - y[tr])[:, None] * w[None, :-1]
    g = oracle.adjoint(P, W, w_in, m0, u, G)
    fd = _fd(lambda a: L(P.replace(A_cp=a)), P.A_cp, 1e-5 * P.A_cp)
    assert abs(g["A_cp"] - fd) <= 1e-5 * abs(fd)
    fd = _fd(lambda a: L(P.replace(I=a)), P.I, 1e-5 * P.I)
    assert abs(g["current"] - fd) <= 1e-5 * abs(fd)
