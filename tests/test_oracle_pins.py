"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself or with the CUDA path.  Each
test names the part of the oracle it pins and the mistake it would catch.
Closed forms used here are derived from Eq. (gov) for special parameter
choices (all of them valid inputs of the method); the derivations are in the
test docstrings.
"""
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad, solve_ivp
from scipy.optimize import brentq

import oracle
from oracle import readout
from paper_2312_01121_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
P0 = oracle.OracleParams()


def _golden_table():
    vals = {}
    with open(os.path.join(GOLDEN, "table_parameters.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


def _traj(params, W, w_in, m0, u):
    """Full 3-component state after every input sample (oracle.run per sample)."""
    m = np.array(m0, dtype=np.float64)
    out = []
    for t in range(u.shape[0]):
        m, _ = oracle.run(params, W, w_in, m, u[t:t + 1])
        out.append(m.copy())
    return np.array(out)  # (T, 3, N)


def _consts(P):
    """gamma', H_K - 4 pi M and H_s0 computed here from the parameters, so the
    closed forms below do not reuse the oracle's own derived constants."""
    gp = P.gamma / (1.0 + P.alpha ** 2)
    hkp = P.H_K - 4.0 * math.pi * P.M
    hs0 = P.hbar * P.eta * P.I / (2.0 * P.e * P.M * P.V) * 1e7
    return gp, hkp, hs0


def _no_field_params(**kw):
    """H_appl = 0 and H_K = 4 pi M, so that H(m) = 0 (Eq. gov, first field)."""
    base = dict(H_appl=0.0, H_K=4.0 * np.pi * P0.M, A_cp=0.0, I=0.0)
    base.update(kw)
    return P0.replace(**base)


# --------------------------------------------------------------------------
# Table values and derived constants


def test_defaults_match_paper_table():
    """Pins the parameter transcription against Table "Summary of parameters"."""
    g = _golden_table()
    P = P0
    for name, attr in [("gamma", "gamma"), ("alpha", "alpha"), ("M", "M"), ("H_K", "H_K"),
                       ("H_appl", "H_appl"), ("eta", "eta"), ("lambda", "lambda_"),
                       ("I", "I"), ("V", "V"), ("e", "e"), ("hbar", "hbar"),
                       ("A_cp", "A_cp"), ("A_in", "A_in"), ("dt", "dt")]:
        assert getattr(P, attr) == pytest.approx(g[name], rel=1e-15), name
    assert tuple(P.p) == (g["p_x"], g["p_y"], g["p_z"])
    d = oracle.derived(P)
    # gamma' = gamma / (1 + alpha^2); 4 pi M in CGS (reading of the table units)
    assert d["gamma_p"] == pytest.approx(g["gamma"] / (1 + g["alpha"] ** 2), rel=1e-15)
    assert d["HK_p"] == pytest.approx(18616.0 - 18199.874560776386, abs=1e-9)


def test_spin_torque_unit_reading():
    """H_s0 = hbar eta I / (2 e M V) in Oe: SI hbar/e, CGS M, V, times 1e7 J->erg.

    The value is fixed by the Table constants and that unit reading; the
    independent anchor is the paper's statement that the parameters make the
    oscillator oscillate (checked in test_driven_single_oscillator_oscillates)."""
    g = _golden_table()
    d = oracle.derived(P0)
    joule_per_emu = g["hbar"] * g["eta"] * g["I"] / (2 * g["e"] * g["M"] * g["V"])
    assert d["Hs0"] == pytest.approx(joule_per_emu * 1e7, rel=1e-14)
    assert d["Hs0"] == pytest.approx(134.868, abs=1e-3)
    # H_s0 scales linearly with the current.
    assert oracle.derived(P0.replace(I=1e-3))["Hs0"] == pytest.approx(d["Hs0"] / 2.5, rel=1e-14)


def test_initial_state_eq_initial():
    """Eq. (initial): |m_k(0)| = 1 and m_k(0) ~ (0, 0, 1), same for every k."""
    m = oracle.initial_state(5)
    phi0 = np.deg2rad(_golden_table()["phi0_deg"])
    assert np.allclose(np.linalg.norm(m, axis=0), 1.0, atol=1e-15)
    assert np.allclose(m[2], np.cos(phi0), atol=0)
    assert np.allclose(m[0], np.sin(phi0) * np.cos(phi0))
    assert np.allclose(m[1], np.sin(phi0) ** 2)
    assert np.all(m == m[:, :1])


# --------------------------------------------------------------------------
# Vector field


def test_field_orthogonal_to_m():
    """m_k . dm_k/dt = 0 for every term of Eq. (gov) (all are m x (...)).

    Catches a torque term that is not a cross product with m (e.g. b instead
    of m x b)."""
    N = 7
    W = inputs.coupling_paper(N, seed=3)
    m = inputs.random_unit_states(N, seed=3) * 1.3  # any m, not only unit
    hin = np.linspace(-50, 50, N)
    for P in [P0, P0.replace(I=4e-3, A_cp=30.0, alpha=0.3)]:
        f, _ = oracle.field(P, W, m, hin)
        dot = np.sum(m * f, axis=0)
        scale = np.linalg.norm(m, axis=0) * np.linalg.norm(f, axis=0)
        assert np.max(np.abs(dot) / scale) < 1e-14


def test_coupling_is_matrix_vector_product():
    """h_cp = A_cp W m^x (Eq. coup with the source index, Sec. 3.3) vs BLAS dgemv."""
    N = 37
    W = inputs.coupling_paper(N, seed=1)
    x = inputs.random_unit_states(N, seed=2)[0]
    P = P0.replace(A_cp=2.5)
    h = oracle.coupling(P, W, x, nthreads=2)
    ref = 2.5 * (W @ x)
    assert np.max(np.abs(h - ref)) <= 1e-14 * np.max(np.abs(W) @ np.abs(x)) * 2.5


def test_coupling_and_input_share_the_x_channel():
    """H_cp and H_in both point along e_x (Eq. coup, Eq. in): a state whose
    coupling field is h gives the same dm/dt as no coupling with H_in = h."""
    N = 6
    W = inputs.coupling_paper(N, seed=4)
    m = inputs.random_unit_states(N, seed=5)
    P = P0.replace(A_cp=40.0)
    f1, h = oracle.field(P, W, m)
    f2, _ = oracle.field(P.replace(A_cp=0.0), W, m, hin=h)
    assert np.max(np.abs(f1 - f2)) <= 1e-12 * np.max(np.abs(f1))


def test_field_affine_in_input():
    """dm/dt is affine in the input field: u enters only through b_x."""
    N = 5
    W = inputs.coupling_paper(N, seed=6)
    m = inputs.random_unit_states(N, seed=6)
    a = np.linspace(1, 3, N) * 10
    b = np.linspace(-2, 1, N) * 10
    f0, _ = oracle.field(P0, W, m, np.zeros(N))
    fa, _ = oracle.field(P0, W, m, a)
    fb, _ = oracle.field(P0, W, m, b)
    fab, _ = oracle.field(P0, W, m, a + b)
    assert np.max(np.abs((fab - f0) - (fa - f0) - (fb - f0))) <= 1e-12 * np.max(np.abs(f0))
    assert np.max(np.abs(fa - f0)) > 1e-3 * np.max(np.abs(f0))


def test_input_field_weights_and_gain():
    """H_in_k = g A_in sum_j w_in[k,j] u_j (Eq. in), several channels."""
    P = P0.replace(n_in=3, A_in=2.0, g=1.5)
    w_in = inputs.input_weights(4, 3, seed=1)
    u_t = np.array([0.25, -1.0, 0.5])
    hin = oracle.input_field(P, w_in, u_t)
    assert np.allclose(hin, 3.0 * (w_in @ u_t), rtol=1e-15, atol=1e-15)


# --------------------------------------------------------------------------
# Closed-form trajectories


def test_undriven_relaxation_closed_form():
    """I = 0, no coupling, no input: b = (H_appl + H_K' m_z) e_z.

    From Eq. (gov): dtheta/dt = -alpha gamma' B(theta) sin(theta) and
    dphi/dt = +gamma' B(theta), B = H_appl + H_K' cos(theta).  Hence exactly
        phi - phi0 = -(1/alpha) ln(tan(theta/2) / tan(theta0/2))
        t(theta)   = int_theta^theta0 dth / (alpha gamma' B(th) sin(th)).
    Pins gamma' (incl. the 1/(1+alpha^2) factor: 0.25 % at alpha = 0.05), alpha,
    H_appl, H_K - 4 pi M and the sense of precession."""
    P = P0.replace(I=0.0, A_cp=0.0, alpha=0.05, dt=1e-12, substeps=100)
    th0 = np.deg2rad(60.0)
    m0 = np.array([[np.sin(th0)], [0.0], [np.cos(th0)]])
    T = 60
    tr = _traj(P, np.zeros((1, 1)), np.zeros((1, 1)), m0, np.zeros((T, 1)))
    m = tr[:, :, 0]
    th = np.arccos(m[:, 2] / np.linalg.norm(m, axis=1))
    ph = np.unwrap(np.concatenate([[0.0], np.arctan2(m[:, 1], m[:, 0])]))[1:]
    t = (np.arange(T) + 1) * P.substeps * P.dt
    gp, hkp, _ = _consts(P)
    # relaxation towards +z (easy axis, H_K > 4 pi M) and counter-clockwise precession
    assert np.all(np.diff(th) < 0) and th[-1] < 0.5 * th0
    assert np.all(np.diff(ph) > 0)
    ph_exact = -(1.0 / P.alpha) * np.log(np.tan(th / 2) / np.tan(th0 / 2))
    assert np.max(np.abs(ph - ph_exact)) < 1e-7
    B = lambda x: P.H_appl + hkp * np.cos(x)
    t_exact = np.array([quad(lambda x: 1.0 / (P.alpha * gp * B(x) * np.sin(x)), a, th0,
                             epsabs=0, epsrel=1e-13)[0] for a in th])
    assert np.max(np.abs(t_exact - t) / t) < 1e-8
    # the same with gamma instead of gamma' would be off by alpha^2 = 0.25 %
    assert 0.0025 * 0.5 > 1e-8


def test_spin_torque_closed_form():
    """Only the spin torque: H_appl = 0, H_K = 4 pi M, no coupling, no input,
    p = e_x.  With s = m.p, Eq. (gov) gives
        ds/dt   = -gamma' H_s0 (1 - s^2) / (1 + lambda s)
        dpsi/dt = +alpha gamma' H_s0 / (1 + lambda s)   (azimuth about p, y -> z)
    so exactly  atanh(s) - (lambda/2) ln(1 - s^2) = F(s0) - gamma' H_s0 t
    and         psi - psi0 = -alpha (atanh(s) - atanh(s0)).
    Pins H_s0 (units), the sign of the current, lambda and the alpha part of
    the spin torque."""
    P = _no_field_params(I=2.5e-3, p=(1.0, 0.0, 0.0), alpha=0.05, dt=1e-12, substeps=50)
    s0 = 0.9
    m0 = np.array([[s0], [np.sqrt(1 - s0 ** 2)], [0.0]])
    T = 60
    tr = _traj(P, np.zeros((1, 1)), np.zeros((1, 1)), m0, np.zeros((T, 1)))
    m = tr[:, :, 0]
    s = m[:, 0]
    psi = np.unwrap(np.concatenate([[0.0], np.arctan2(m[:, 2], m[:, 1])]))[1:]
    t = (np.arange(T) + 1) * P.substeps * P.dt
    gp, _, hs0 = _consts(P)
    F = lambda x: np.arctanh(x) - 0.5 * P.lambda_ * np.log(1 - x * x)
    assert np.all(np.diff(s) < 0) and s[-1] < 0.0   # pushed away from p
    # invert F for the exact s(t) and compare in s (F is steep near s = -1)
    s_exact = np.array([brentq(lambda x: F(x) - F(s0) + gp * hs0 * tt,
                               -1 + 1e-15, s0, xtol=1e-15, rtol=1e-15) for tt in t])
    assert np.max(np.abs(s - s_exact)) < 1e-10
    # atanh(s) is steep near s = -1; compare where it amplifies errors < 50x
    w = np.abs(s) < 0.99
    assert w.sum() > 20
    assert np.max(np.abs(psi + P.alpha * (np.arctanh(s) - np.arctanh(s0)))[w]) < 1e-9
    assert np.all(np.diff(psi) > 0)


def test_input_drive_closed_form_and_hold():
    """Only the input field: b = g A_in w u_t e_x, held over each input sample.

    Relaxation about e_x gives atanh(m_x) = atanh(m_x0) + alpha gamma' int B dt,
    so after sample t: m_x = tanh(atanh(m_x0) + alpha gamma' g A_in w S dt
    sum_{tau <= t} u_tau).  Pins A_in, g, w_in, the e_x direction, the
    zero-order hold and that states[t] is taken after sample t's substeps."""
    P = _no_field_params(A_in=500.0, g=1.5, alpha=0.05, dt=1e-12, substeps=100)
    w = 0.8
    u = inputs.input_series(50, 1, seed=11)
    m0 = np.array([[-0.2], [np.sqrt(1 - 0.04)], [0.0]])
    m, states = oracle.run(P, np.zeros((1, 1)), np.array([[w]]), m0, u)
    gp = _consts(P)[0]
    expect = np.tanh(np.arctanh(-0.2) + P.alpha * gp * P.g * P.A_in * w * P.substeps * P.dt
                     * np.cumsum(u[:, 0]))
    assert np.max(np.abs(states[:, 0] - expect)) < 1e-9
    # off-by-one in the schedule would shift the cumulative sum by one sample
    wrong = np.tanh(np.arctanh(-0.2) + P.alpha * gp * P.g * P.A_in * w * P.substeps * P.dt
                    * np.concatenate([[0.0], np.cumsum(u[:-1, 0])]))
    assert np.max(np.abs(states[:, 0] - wrong)) > 1e-3


def test_one_way_coupling_closed_form():
    """W = [[0, c], [0, 0]]: row k is the target, column i the source.

    With no other field, oscillator 1 feels nothing and stays exactly at its
    initial state; oscillator 0 feels B = A_cp c m_1^x along e_x, so
    m_0^x(t) = tanh(atanh(m_0^x(0)) + alpha gamma' B t).  Pins the reading
    of Eq. (coup) with the source index (the printed m_k^x would give node 0
    a field proportional to its own m^x) and catches a transposed W."""
    c = 0.75
    P = _no_field_params(A_cp=400.0, alpha=0.05, dt=1e-12, substeps=100)
    W = np.array([[0.0, c], [0.0, 0.0]])
    m0 = np.array([[0.1, 0.6], [np.sqrt(0.99), 0.0], [0.0, 0.8]])
    T = 40
    tr = _traj(P, W, np.zeros((2, 1)), m0, np.zeros((T, 1)))
    assert np.all(tr[:, :, 1] == m0[:, 1])
    gp = _consts(P)[0]
    t = (np.arange(T) + 1) * P.substeps * P.dt
    expect = np.tanh(np.arctanh(0.1) + P.alpha * gp * P.A_cp * c * 0.6 * t)
    assert np.max(np.abs(tr[:, 0, 0] - expect)) < 1e-9


# --------------------------------------------------------------------------
# Integrator


def _paper_system(N, seed=0):
    W = inputs.coupling_paper(N, seed=seed)
    w_in = inputs.input_weights(N, 1, seed=seed)
    m0 = inputs.random_unit_states(N, seed=seed)
    u = inputs.input_series(4, 1, seed=seed)
    return W, w_in, m0, u


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_rk4_local_error_order(seed):
    """Classic RK4 (Sec. 3.2) has local error C h^5: one step from the same
    state, against DOP853 at rtol ~2e-14, shrinks 32x per halving of h.  A
    wrong stage weight or stage point leaves an h^2..h^4 local error."""
    N = 4
    W, w_in, m0, u = _paper_system(N, seed=seed)
    P = P0.replace(A_cp=50.0)
    hin = oracle.input_field(P, w_in, u[0])
    rhs = lambda _t, yy: oracle.field(P, W, yy.reshape(3, N), hin)[0].reshape(-1)
    e = []
    for h in (8e-12, 4e-12, 2e-12):
        ref = solve_ivp(rhs, (0.0, h), m0.reshape(-1), method="DOP853",
                        rtol=2.3e-14, atol=1e-17).y[:, -1].reshape(3, N)
        e.append(np.linalg.norm(oracle.rk4_step(P.replace(dt=h), W, m0, hin) - ref))
    assert 30.0 < e[0] / e[1] < 34.0 and 30.0 < e[1] / e[2] < 34.0


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_brute_force_small_n(N):
    """N = 1..4 against an independent integration (scipy DOP853, rtol 1e-13)
    of the same vector field with the same piecewise-constant input.  The
    oracle's deviation must equal its own Richardson error estimate
    (x_dt - x_dt/2) * 16/15 to within 20 %, i.e. the only error is RK4's."""
    W, w_in, m0, u = _paper_system(N, seed=N)
    P = P0.replace(A_cp=50.0, A_in=30.0)
    T = 3
    m_dt, st_dt = oracle.run(P, W, w_in, m0, u[:T])
    m_h, _ = oracle.run(P.replace(substeps=2 * P.substeps, dt=P.dt / 2), W, w_in, m0, u[:T])
    y = m0.reshape(-1).copy()
    for t in range(T):
        hin = oracle.input_field(P, w_in, u[t])
        rhs = lambda _t, yy: oracle.field(P, W, yy.reshape(3, N), hin)[0].reshape(-1)
        sol = solve_ivp(rhs, (0.0, P.substeps * P.dt), y, method="DOP853",
                        rtol=1e-13, atol=1e-15)
        y = sol.y[:, -1]
    ref = y.reshape(3, N)
    err = m_dt - ref
    est = (m_dt - m_h) * 16.0 / 15.0
    assert np.linalg.norm(est) > 1e-9   # the truncation error is measurable
    assert np.linalg.norm(err - est) < 0.2 * np.linalg.norm(est)


def test_norm_drift_is_rk4_truncation():
    """|m_k| = 1 is conserved by the ODE (Sec. 3.1); RK4 breaks it only by its
    truncation error: the drift is far above rounding (no renormalisation
    hides it) and halving dt shrinks it by at least 2^4 (measured ~2^5: on
    the dominant precession RK4's amplification |R(iy)| = 1 - y^6/144 + ...)."""
    W, w_in, m0, u = _paper_system(4, seed=7)
    u = inputs.input_series(20, 1, seed=7)
    drift = []
    for S in (100, 200):
        P = P0.replace(substeps=S, dt=1e-9 / S, A_cp=20.0)
        tr = _traj(P, W, w_in, m0, u)
        drift.append(np.max(np.abs(np.linalg.norm(tr, axis=1) - 1.0)))
    assert 1e-12 < drift[0] < 1e-5
    assert 14.0 < drift[0] / drift[1] < 40.0


def test_driven_single_oscillator_oscillates():
    """Sec. 3.1: the parameters make the solution oscillate.  A single STO at
    I = 2.5 mA reaches a limit cycle (large, steady m^x swing, period
    converged under dt halving); at I = 0 it relaxes to +z; with H_s0 ten
    times smaller (the other unit reading) it never leaves +z.
    Partially pinned: the paper prints no frequency or amplitude."""
    def series(P, T=300):
        m0 = oracle.initial_state(1)
        _, st = oracle.run(P, np.zeros((1, 1)), np.zeros((1, 1)), m0, np.zeros((T, 1)))
        return st[:, 0]

    P = P0.replace(substeps=10)  # samples every 0.1 ns
    x = series(P)
    tail = x[150:]
    assert tail.max() > 0.8 and tail.min() < -0.8
    def period(xs, dt_s):
        up = np.where((xs[:-1] < 0) & (xs[1:] >= 0))[0]
        frac = -xs[up] / (xs[up + 1] - xs[up])
        tz = (up + frac) * dt_s
        return np.mean(np.diff(tz))
    p1 = period(tail, 1e-10)
    x2 = series(P.replace(substeps=20, dt=5e-12))
    p2 = period(x2[150:], 1e-10)
    assert abs(p1 - p2) / p2 < 2e-3
    assert 1e-9 < p1 < 5e-9   # an oscillation in the GHz range
    assert np.max(np.abs(series(P.replace(I=0.0))[150:])) < 0.05
    assert np.max(np.abs(series(P.replace(I=0.25e-3))[150:])) < 0.05


# --------------------------------------------------------------------------
# Structure


def test_decoupled_nodes_equal_single_node():
    """A_cp = 0: every oscillator with the Eq. (initial) start follows the
    N = 1 trajectory bit for bit (no leakage between nodes)."""
    N = 5
    W = inputs.coupling_paper(N, seed=2)
    P = P0.replace(A_cp=0.0)
    u = np.zeros((5, 1))
    m, st = oracle.run(P, W, np.zeros((N, 1)), oracle.initial_state(N), u)
    m1, st1 = oracle.run(P, np.zeros((1, 1)), np.zeros((1, 1)), oracle.initial_state(1), u)
    assert np.all(st == st1) and np.all(m == m1)


def test_permutation_equivariance_and_paper_order_check():
    """Relabelling oscillators permutes the trajectory (P W P^T, P m0, P w_in).
    The residual difference comes only from the changed summation order; the
    paper's own cross-implementation criterion (Sec. 3.3) is that such
    differences are at least 1e-6 times smaller than | |m| - 1 |."""
    N = 6
    W, w_in, m0, _ = _paper_system(N, seed=9)
    u = inputs.input_series(5, 1, seed=9)
    perm = np.array([3, 0, 5, 1, 4, 2])
    P = P0
    tr = _traj(P, W, w_in, m0, u)
    trp = _traj(P, W[np.ix_(perm, perm)], w_in[perm], m0[:, perm], u)
    diff = np.max(np.abs(trp - tr[:, :, perm]))
    assert diff < 1e-12
    norm_err = np.max(np.abs(np.linalg.norm(tr, axis=1) - 1.0))
    assert diff <= 1e-6 * norm_err


def test_run_is_resumable():
    """Running T samples at once equals running them in two calls (the state
    is the whole memory of the method; sampling does not perturb it)."""
    W, w_in, m0, _ = _paper_system(3, seed=4)
    u = inputs.input_series(6, 1, seed=4)
    m, st = oracle.run(P0, W, w_in, m0, u)
    ma, sa = oracle.run(P0, W, w_in, m0, u[:2])
    mb, sb = oracle.run(P0, W, w_in, ma, u[2:])
    assert np.all(m == mb) and np.all(st == np.vstack([sa, sb]))


def test_sampled_component():
    W, w_in, m0, _ = _paper_system(3, seed=5)
    u = inputs.input_series(3, 1, seed=5)
    tr = _traj(P0, W, w_in, m0, u)
    for c in range(3):
        _, st = oracle.run(P0.replace(component=c), W, w_in, m0, u)
        assert np.all(st == tr[:, c, :])


def test_openmp_rows_do_not_change_results():
    """Threads split rows only; each row is still summed in ascending order."""
    W, w_in, m0, u = _paper_system(40, seed=8)
    a = oracle.run(P0, W, w_in, m0, u[:2], nthreads=1)
    b = oracle.run(P0, W, w_in, m0, u[:2], nthreads=4)
    assert np.all(a[0] == b[0]) and np.all(a[1] == b[1])


# --------------------------------------------------------------------------
# Readout


def test_ridge_limit_is_least_squares():
    """beta -> 0: ridge with a bias column equals lstsq on [X, 1]."""
    g = np.random.default_rng(0)
    X = g.standard_normal((200, 12))
    y = X @ g.standard_normal(12) + 0.3 + 0.01 * g.standard_normal(200)
    w = readout.ridge_fit(X, y, beta_rel=1e-14)
    ref = np.linalg.lstsq(np.hstack([X, np.ones((200, 1))]), y, rcond=None)[0]
    assert np.allclose(w, ref, rtol=1e-8, atol=1e-10)
    assert readout.nmse(readout.predict(X, w), y) < 1e-3


def test_ridge_shrinks_weights_not_bias():
    g = np.random.default_rng(1)
    X = g.standard_normal((100, 5))
    y = np.full(100, 7.0)
    w = readout.ridge_fit(X, y, beta_rel=10.0)
    assert abs(w[-1] - 7.0) < 0.2 and np.max(np.abs(w[:-1])) < 0.2


def test_delay_target_and_split():
    u = np.arange(10.0).reshape(-1, 1)
    y = readout.delay_target(u, 5)
    assert np.all(y[5:] == np.arange(5.0)) and np.all(y[:5] == 0)
    tr, te = readout.split(110, 100)
    assert tr[0] == 100 and te[-1] == 109 and len(tr) == 5
