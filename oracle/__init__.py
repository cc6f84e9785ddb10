"""FP64 CPU oracle for the coupled spin-torque-oscillator reservoir (arXiv 2312.01121).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library and never imports it.

The arithmetic lives in ``sto_oracle.c`` (plain C, FP64); this module compiles
it with gcc on first use and wraps it with ctypes.  ``readout.py`` holds the
FP64 ridge readout.

Parity status of each function (the pins are in ``tests/test_oracle_pins.py``):
  derived        pinned: Table "Summary of parameters" fixture + closed forms
  field          pinned: m.f = 0, closed-form relaxation / spin-torque / input /
                 one-way coupling trajectories, linearity in u, BLAS matvec
  rk4 / run      pinned: order-4 convergence, DOP853 brute force at N = 1..4,
                 closed-form trajectories, norm drift O(dt^4)
  initial_state  pinned: Eq. (initial) unit norm and the stated limit (0,0,1)
  readout        pinned: ridge at beta -> 0 equals numpy lstsq
  erk            pinned: local error order p+1 of Euler, Heun, Kutta-3 and RK4
                 tableaus against DOP853; the RK4 tableau reproduces `run`
  adjoint        pinned: central finite differences of `run` (FP64) for A_cp,
                 I, w_in and m0, including the refitted-readout objective
                 (tests/test_oracle_adjoint.py)
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sto_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sto_oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP).

    No fast-math and the default x86-64 target, so no FMA contraction: every
    operation is the IEEE double operation written in the source."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _CParams(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double), ("alpha", ctypes.c_double), ("M", ctypes.c_double),
        ("H_K", ctypes.c_double), ("H_appl", ctypes.c_double), ("eta", ctypes.c_double),
        ("lambda_", ctypes.c_double), ("I", ctypes.c_double), ("V", ctypes.c_double),
        ("e", ctypes.c_double), ("hbar", ctypes.c_double), ("p", ctypes.c_double * 3),
        ("A_cp", ctypes.c_double), ("A_in", ctypes.c_double), ("g", ctypes.c_double),
        ("dt", ctypes.c_double), ("substeps", ctypes.c_int), ("n_in", ctypes.c_int),
        ("component", ctypes.c_int), ("pad", ctypes.c_int),
    ]


@dataclasses.dataclass
class OracleParams:
    """Model parameters; defaults are Table "Summary of parameters" (Sec. 3.1).

    V = pi * 60^2 * 2 nm^3 expressed in cm^3 (1 nm^3 = 1e-21 cm^3).  dt is the
    Sec. 3.2 step.  substeps (RK4 steps per input sample), g (input gain),
    n_in and component are not fixed by the paper; the defaults are the
    readings documented in the design notes (100 substeps, g = 1, one input
    channel, the x component)."""
    gamma: float = 1.764e7
    alpha: float = 0.005
    M: float = 1448.3
    H_K: float = 18616.0
    H_appl: float = 200.0
    eta: float = 0.537
    lambda_: float = 0.288
    I: float = 2.5e-3
    V: float = np.pi * 60.0 ** 2 * 2.0 * 1e-21
    e: float = 1.60217733e-19
    hbar: float = 1.05457266e-34
    p: tuple = (1.0, 0.0, 6.123234e-17)
    A_cp: float = 1.0
    A_in: float = 1.0
    g: float = 1.0
    dt: float = 1e-11
    substeps: int = 100
    n_in: int = 1
    component: int = 0

    def replace(self, **kw) -> "OracleParams":
        return dataclasses.replace(self, **kw)

    def _c(self) -> _CParams:
        c = _CParams()
        for f in dataclasses.fields(self):
            if f.name == "p":
                c.p = (ctypes.c_double * 3)(*[float(v) for v in self.p])
            else:
                setattr(c, f.name, getattr(self, f.name))
        return c


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.POINTER(ctypes.c_double)
            P = ctypes.POINTER(_CParams)
            lib.orc_derived.argtypes = [P, D]
            lib.orc_coupling.argtypes = [ctypes.c_int, P, D, D, D, ctypes.c_int]
            lib.orc_field.argtypes = [ctypes.c_int, P, D, D, D, D, D, ctypes.c_int]
            lib.orc_input_field.argtypes = [ctypes.c_int, P, D, D, D]
            lib.orc_rk4_step.argtypes = [ctypes.c_int, P, D, D, D, ctypes.c_int]
            lib.orc_run.argtypes = [ctypes.c_int, P, D, D, D, D, ctypes.c_int, D, ctypes.c_int]
            lib.orc_run.restype = ctypes.c_int
            lib.orc_initial_state.argtypes = [ctypes.c_int, D]
            lib.orc_max_threads.restype = ctypes.c_int
            lib.orc_adjoint.argtypes = [ctypes.c_int, P, D, D, D, D, ctypes.c_int, D, D,
                                        ctypes.c_int]
            lib.orc_adjoint.restype = ctypes.c_int
            lib.orc_erk_step.argtypes = [ctypes.c_int, P, D, D, D, ctypes.c_int, D, D, ctypes.c_int]
            lib.orc_run_erk.argtypes = [ctypes.c_int, P, D, D, D, D, ctypes.c_int, D, ctypes.c_int,
                                        D, D, ctypes.c_int]
            lib.orc_run_erk.restype = ctypes.c_int
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def max_threads() -> int:
    return int(_load().orc_max_threads())


def derived(params: OracleParams) -> dict:
    """gamma' = gamma/(1+alpha^2), H_K' = H_K - 4 pi M, H_s0 (Oe) of Eq. (gov)."""
    out = np.zeros(3)
    c = params._c()
    _load().orc_derived(ctypes.byref(c), _d(out))
    return {"gamma_p": out[0], "HK_p": out[1], "Hs0": out[2]}


def initial_state(N: int) -> np.ndarray:
    """Eq. (initial) for every oscillator, shape (3, N)."""
    m = np.zeros((3, N))
    _load().orc_initial_state(N, _d(m))
    return m


def coupling(params: OracleParams, W, x, nthreads: int = 1) -> np.ndarray:
    W = _f64(W)
    N = W.shape[0]
    x = _f64(x, (N,))
    h = np.zeros(N)
    c = params._c()
    _load().orc_coupling(N, ctypes.byref(c), _d(W), _d(x), _d(h), nthreads)
    return h


def field(params: OracleParams, W, m, hin=None, nthreads: int = 1):
    """dm/dt of Eq. (gov) at state m (3, N); returns (f (3, N), h_cp (N,))."""
    W = _f64(W)
    N = W.shape[0]
    m = _f64(m, (3, N))
    f = np.zeros((3, N))
    h = np.zeros(N)
    hin_a = _f64(hin, (N,)) if hin is not None else None
    c = params._c()
    _load().orc_field(N, ctypes.byref(c), _d(W), _d(m),
                      _d(hin_a) if hin_a is not None else None, _d(f), _d(h), nthreads)
    return f, h


def input_field(params: OracleParams, w_in, u_t) -> np.ndarray:
    w_in = _f64(w_in)
    N = w_in.shape[0]
    w_in = w_in.reshape(N, params.n_in)
    u_t = _f64(u_t, (params.n_in,))
    hin = np.zeros(N)
    c = params._c()
    _load().orc_input_field(N, ctypes.byref(c), _d(w_in), _d(u_t), _d(hin))
    return hin


def rk4_step(params: OracleParams, W, m, hin=None, nthreads: int = 1) -> np.ndarray:
    W = _f64(W)
    N = W.shape[0]
    m = _f64(m, (3, N)).copy()
    hin_a = _f64(hin, (N,)) if hin is not None else np.zeros(N)
    c = params._c()
    _load().orc_rk4_step(N, ctypes.byref(c), _d(W), _d(hin_a), _d(m), nthreads)
    return m


def run(params: OracleParams, W, w_in, m0, u, T: int | None = None, nthreads: int = 1):
    """Advance m0 over T input samples (T defaults to len(u)).

    Returns (m_final (3, N), states (T, N)) with states[t] the sampled
    component after input sample t."""
    W = _f64(W)
    N = W.shape[0]
    if W.shape != (N, N):
        raise ValueError("W must be N x N")
    u = _f64(u)
    if u.ndim == 1:
        u = u.reshape(-1, 1)
    if T is None:
        T = u.shape[0]
    u = np.ascontiguousarray(u[:T].reshape(T, params.n_in)) if T > 0 else np.zeros((1, params.n_in))
    w_in = _f64(w_in).reshape(N, params.n_in)
    m = _f64(m0, (3, N)).copy()
    states = np.zeros((max(T, 1), N))
    c = params._c()
    rc = _load().orc_run(N, ctypes.byref(c), _d(W), _d(w_in), _d(m), _d(u), T,
                         _d(states), nthreads)
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return m, states[:T]


def adjoint(params: OracleParams, W, w_in, m0, u, dL_dstates, nthreads: int = 1) -> dict:
    """Exact gradients of L = sum(dL_dstates * states) for one run from m0
    (discrete adjoint of the RK4 stepper).  Returns dA_cp, dI, dw_in (N, n_in)
    and dm0 (3, N)."""
    W = _f64(W)
    N = W.shape[0]
    u = _f64(u)
    if u.ndim == 1:
        u = u.reshape(-1, 1)
    T = u.shape[0]
    u = np.ascontiguousarray(u.reshape(T, params.n_in))
    w_in = _f64(w_in).reshape(N, params.n_in)
    m0 = _f64(m0, (3, N))
    g = _f64(dL_dstates, (T, N))
    out = np.zeros(2 + N * params.n_in + 3 * N)
    c = params._c()
    rc = _load().orc_adjoint(N, ctypes.byref(c), _d(W), _d(w_in), _d(m0), _d(u), T, _d(g),
                             _d(out), nthreads)
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    nw = N * params.n_in
    return {"A_cp": out[0], "current": out[1], "w_in": out[2:2 + nw].reshape(N, params.n_in),
            "m0": out[2 + nw:].reshape(3, N)}


# Explicit Runge-Kutta tableaus (a strictly lower triangular, weights b).
TABLEAUS = {
    "euler": ([[0.0]], [1.0]),
    "heun": ([[0.0, 0.0], [1.0, 0.0]], [0.5, 0.5]),
    "kutta3": ([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [-1.0, 2.0, 0.0]], [1 / 6, 2 / 3, 1 / 6]),
    "rk4": ([[0, 0, 0, 0], [0.5, 0, 0, 0], [0, 0.5, 0, 0], [0, 0, 1.0, 0]],
            [1 / 6, 1 / 3, 1 / 3, 1 / 6]),
    # Kutta's 3/8 rule: order 4 with every entry below the diagonal in use
    "rk38": ([[0, 0, 0, 0], [1 / 3, 0, 0, 0], [-1 / 3, 1.0, 0, 0], [1.0, -1.0, 1.0, 0]],
             [1 / 8, 3 / 8, 3 / 8, 1 / 8]),
}


def erk_step(params: OracleParams, W, m, a, b, hin=None, nthreads: int = 1) -> np.ndarray:
    W = _f64(W)
    N = W.shape[0]
    m = _f64(m, (3, N)).copy()
    s = len(b)
    A = _f64(a, (s, s))
    B = _f64(b, (s,))
    hin_a = _f64(hin, (N,)) if hin is not None else np.zeros(N)
    c = params._c()
    _load().orc_erk_step(N, ctypes.byref(c), _d(W), _d(hin_a), _d(m), s, _d(A), _d(B), nthreads)
    return m


def run_erk(params: OracleParams, W, w_in, m0, u, a, b, T: int | None = None, nthreads: int = 1):
    """`run` with an explicit Runge-Kutta tableau in place of classic RK4."""
    W = _f64(W)
    N = W.shape[0]
    u = _f64(u)
    if u.ndim == 1:
        u = u.reshape(-1, 1)
    if T is None:
        T = u.shape[0]
    u = np.ascontiguousarray(u[:T].reshape(T, params.n_in)) if T > 0 else np.zeros((1, params.n_in))
    w_in = _f64(w_in).reshape(N, params.n_in)
    m = _f64(m0, (3, N)).copy()
    s = len(b)
    A = _f64(a, (s, s))
    B = _f64(b, (s,))
    states = np.zeros((max(T, 1), N))
    c = params._c()
    rc = _load().orc_run_erk(N, ctypes.byref(c), _d(W), _d(w_in), _d(m), _d(u), T, _d(states),
                             s, _d(A), _d(B), nthreads)
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return m, states[:T]
