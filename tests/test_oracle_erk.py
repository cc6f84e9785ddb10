"""Pins of the oracle's general explicit Runge-Kutta stepping."""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle
from paper_2312_01121_b300 import inputs


def _system(N, seed):
    return (inputs.coupling_paper(N, seed), inputs.input_weights(N, 1, seed),
            inputs.random_unit_states(N, seed), inputs.input_series(3, 1, seed))


@pytest.mark.parametrize("name,order", [("euler", 1), ("heun", 2), ("kutta3", 3), ("rk4", 4),
                                        ("rk38", 4)])
def test_local_error_order(name, order):
    """One step against DOP853: the local error of an order-p method shrinks
    2^(p+1) x per halving of dt."""
    N = 4
    W, w_in, m0, u = _system(N, 2)
    P = oracle.OracleParams(A_cp=50.0)
    hin = oracle.input_field(P, w_in, u[0])
    rhs = lambda _t, yy: oracle.field(P, W, yy.reshape(3, N), hin)[0].reshape(-1)
    a, b = oracle.TABLEAUS[name]
    e = []
    hs = (8e-12, 4e-12, 2e-12) if order >= 3 else (4e-13, 2e-13, 1e-13)
    for h in hs:
        ref = solve_ivp(rhs, (0.0, h), m0.reshape(-1), method="DOP853", rtol=2.3e-14,
                        atol=1e-18).y[:, -1].reshape(3, N)
        e.append(np.linalg.norm(oracle.erk_step(P.replace(dt=h), W, m0, a, b, hin) - ref))
    want = 2.0 ** (order + 1)
    assert 0.85 * want < e[0] / e[1] < 1.15 * want
    assert 0.85 * want < e[1] / e[2] < 1.15 * want


def test_rk4_tableau_reproduces_run():
    N = 6
    W, w_in, m0, u = _system(N, 3)
    P = oracle.OracleParams(substeps=7, A_cp=20.0)
    a, b = oracle.TABLEAUS["rk4"]
    m1, s1 = oracle.run(P, W, w_in, m0, u)
    m2, s2 = oracle.run_erk(P, W, w_in, m0, u, a, b)
    assert np.max(np.abs(m1 - m2)) < 1e-13 and np.max(np.abs(s1 - s2)) < 1e-13
