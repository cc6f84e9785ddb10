"""Shared test utilities: seeded systems, GPU runs through the C ABI, oracle runs."""
from __future__ import annotations

import os

import numpy as np

import oracle
from paper_2312_01121_b300 import inputs

NTHREADS = max(1, min(16, os.cpu_count() or 1))


def make_system(N: int, kind: str = "gauss", seed: int = 0, T: int = 10, n_in: int = 1):
    """float32-rounded W, w_in, m0 (3, N), u (T, n_in) of the given structure."""
    if kind == "paper":
        W = inputs.coupling_paper(N, seed=seed)
    elif kind == "gauss":
        W = inputs.coupling_gaussian(N, seed=seed)
    else:
        raise ValueError(kind)
    return (inputs.f32(W), inputs.f32(inputs.input_weights(N, n_in, seed=seed)),
            inputs.f32(inputs.random_unit_states(N, seed=seed)),
            inputs.f32(inputs.input_series(T, n_in, seed=seed)))


def oracle_params(P) -> oracle.OracleParams:
    """The oracle's parameter record with the same values as a sto.Params."""
    return oracle.OracleParams(
        gamma=P.gamma, alpha=P.alpha, M=P.Ms, H_K=P.Hk, H_appl=P.Happl, eta=P.eta,
        lambda_=P.lambda_, I=P.current, V=P.volume, e=P.e_charge, hbar=P.hbar, p=tuple(P.p),
        A_cp=P.A_cp, A_in=P.A_in, g=P.input_gain, dt=P.dt, substeps=P.substeps, n_in=P.n_in,
        component=P.sample_component)


def run_oracle(P, W, w_in, m0, u, T=None, m0_f64=None):
    m_start = m0_f64 if m0_f64 is not None else np.asarray(m0, dtype=np.float64)
    return oracle.run(oracle_params(P), np.asarray(W, np.float64), np.asarray(w_in, np.float64),
                      m_start, np.asarray(u, np.float64), T=T, nthreads=NTHREADS)


def run_gpu(P, W, w_in, m0, u, T=None, grid=0, device=True, timeout_ms=0):
    """Run through libsto; returns (final FP64 state (3, N), states (T, N) float32)."""
    import torch

    from paper_2312_01121_b300 import sto
    N = W.shape[0]
    T = u.shape[0] if T is None else T
    if device:
        dev = torch.device("cuda")
        Wt, wt, mt = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (W, w_in, m0))
        ut = torch.from_numpy(np.ascontiguousarray(u)).to(dev)
        st = torch.zeros((max(T, 1), N), dtype=torch.float32, device=dev)
        with sto.Reservoir(Wt, wt, P, m0=mt, stream=torch.cuda.current_stream(), grid=grid,
                           timeout_ms=timeout_ms) as r:
            r.run(ut, st, T=T)
            m = r.state()
        return m, st[:T].cpu().numpy()
    st = np.zeros((max(T, 1), N), dtype=np.float32)
    with sto.Reservoir(W, w_in, P, m0=m0, grid=grid, timeout_ms=timeout_ms) as r:
        r.run(u, st, T=T)
        m = r.state()
    return m, st[:T]
