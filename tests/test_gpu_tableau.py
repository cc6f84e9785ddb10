"""Explicit Runge-Kutta tableaus other than classic RK4 on the CUDA path,
against the oracle's tableau stepper.

Tolerances as for RK4: one step's increment to 1e-5 relative to its largest
component; sampled states over a short horizon to 1e-4 absolute.
"""
import numpy as np
import pytest

import helpers
import oracle
from helpers import make_system

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2312_01121_b300 import build, sto
    build.build()
    sto.load_library()


def _run(P, W, w_in, m0, u, tableau, grid=0):
    from paper_2312_01121_b300 import sto
    N = W.shape[0]
    T = u.shape[0]
    st = np.zeros((T, N), dtype=np.float32)
    with sto.Reservoir(W, w_in, P, m0=m0, grid=grid) as r:
        if tableau is not None:
            r.set_tableau(*oracle.TABLEAUS[tableau])
        r.run(u, st, T=T)
        return r.state(), st


def _oracle(P, W, w_in, m0, u, tableau):
    a, b = oracle.TABLEAUS[tableau]
    return oracle.run_erk(helpers.oracle_params(P), np.asarray(W, np.float64),
                          np.asarray(w_in, np.float64), np.asarray(m0, np.float64),
                          np.asarray(u, np.float64), a, b, nthreads=helpers.NTHREADS)


@pytest.mark.parametrize("tableau", ["euler", "heun", "kutta3", "rk38"])
@pytest.mark.parametrize("N,kind,grid", [(8, "paper", 0), (1000, "gauss", 0), (2500, "gauss", 0),
                                         (1001, "gauss", 7)])
def test_one_step_increment(tableau, N, kind, grid):
    from paper_2312_01121_b300 import sto
    W, w_in, m0, u = make_system(N, kind, seed=N)
    P = sto.Params(substeps=1, A_cp=300.0)
    m_gpu, _ = _run(P, W, w_in, m0, u[:1], tableau, grid)
    m_orc, _ = _oracle(P, W, w_in, m0, u[:1], tableau)
    d_gpu = m_gpu - m0.astype(np.float64)
    d_orc = m_orc - m0.astype(np.float64)
    rel = np.max(np.abs(d_gpu - d_orc)) / np.max(np.abs(d_orc))
    assert rel <= 1e-5, rel


@pytest.mark.parametrize("tableau,T", [("heun", 40), ("kutta3", 40), ("rk38", 40), ("euler", 5)])
def test_sampled_states(tableau, T):
    from paper_2312_01121_b300 import sto
    W, w_in, m0, u = make_system(100, "gauss", seed=1, T=T)
    P = sto.Params(substeps=100)
    m_gpu, st_gpu = _run(P, W, w_in, m0, u, tableau)
    m_orc, st_orc = _oracle(P, W, w_in, m0, u, tableau)
    assert np.max(np.abs(st_gpu - st_orc)) <= 1e-4
    assert np.max(np.abs(m_gpu - m_orc)) <= 1e-4


def test_rk4_tableau_matches_classic_path_and_reset():
    """The classic tableau through the generic program gives the classic
    stepper's samples; stages = 0 goes back to the classic program."""
    from paper_2312_01121_b300 import sto
    W, w_in, m0, u = make_system(300, "gauss", seed=4, T=20)
    P = sto.Params(substeps=20)
    _, st_classic = _run(P, W, w_in, m0, u, None)
    _, st_tab = _run(P, W, w_in, m0, u, "rk4")
    assert np.max(np.abs(st_tab - st_classic)) <= 1e-5
    st = np.zeros_like(st_classic)
    with sto.Reservoir(W, w_in, P, m0=m0) as r:
        r.set_tableau(*oracle.TABLEAUS["euler"])
        r.set_tableau()
        r.run(u, st, T=u.shape[0])
    assert np.array_equal(st, st_classic)


def test_invalid_tableaus_and_adjoint_refused():
    from paper_2312_01121_b300 import sto
    W, w_in, m0, u = make_system(16, "gauss", seed=5, T=3)
    P = sto.Params(substeps=2)
    with sto.Reservoir(W, w_in, P, m0=m0) as r:
        with pytest.raises(sto.StoError):  # implicit (diagonal entry)
            r.set_tableau([[0.5]], [1.0])
        with pytest.raises(sto.StoError):  # five stages
            r.set_tableau(np.zeros((5, 5)), np.full(5, 0.2))
        with pytest.raises(sto.StoError):
            r.set_tableau([[0.0, 0.0], [np.nan, 0.0]], [0.5, 0.5])
        r.set_tableau(*oracle.TABLEAUS["heun"])
        with pytest.raises(sto.StoError):
            r.adjoint(u, np.ones((3, 16), np.float32))
