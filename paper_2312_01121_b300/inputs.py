"""Seeded synthetic inputs for the coupled-STO reservoir (arXiv 2312.01121).

This module only draws random numbers; it holds none of the simulator's
arithmetic.  Both the CUDA library's callers and the CPU oracle's tests take
their inputs from here, so both sides see identical bytes.

Every generator takes a seed and a stream id and draws from
``numpy.random.default_rng([seed, stream])``, so each array is reproducible
on its own.

Structures (Sec. 3.1, the paragraph after Eq. (in)):
  * paper coupling matrix: zero diagonal, off-diagonal entries i.i.d.
    uniform on [-1, 1], rescaled so that its spectral radius is 1;
  * input weights: i.i.d. uniform on [-1, 1].
Workload structures used by the benchmarks (not fixed by the paper):
  * Gaussian coupling matrix: zero diagonal, i.i.d. N(0, std^2) with
    std = 0.1 / sqrt(N) by default;
  * input series: i.i.d. uniform on [0, 1];
  * random initial magnetisations: normalised i.i.d. N(0, 1) 3-vectors.
"""
from __future__ import annotations

import numpy as np

STREAM_W, STREAM_WIN, STREAM_U, STREAM_M0, STREAM_SWEEP = 1, 2, 3, 4, 5


def rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


def coupling_paper(N: int, seed: int = 0) -> np.ndarray:
    """N x N float64: zero diagonal, U[-1,1] off-diagonal, spectral radius 1.

    The spectral radius comes from LAPACK geev (numpy.linalg.eigvals); for
    N = 1 the matrix is [0] and is not rescaled."""
    g = rng(seed, STREAM_W)
    W = g.uniform(-1.0, 1.0, size=(N, N))
    np.fill_diagonal(W, 0.0)
    if N > 1:
        rho = float(np.max(np.abs(np.linalg.eigvals(W))))
        if rho > 0:
            W = W / rho
    return W


def coupling_paper_circular(N: int, seed: int = 0) -> np.ndarray:
    """The paper's structure (zero diagonal, U[-1,1] off-diagonal) scaled by
    the circular law's spectral radius sqrt(N/3) instead of an eigensolve
    (which takes minutes at N = 10^4); for timing runs, where the radius
    only needs to be about 1.  Same random draws as coupling_paper."""
    g = rng(seed, STREAM_W)
    W = g.uniform(-1.0, 1.0, size=(N, N))
    np.fill_diagonal(W, 0.0)
    if N > 1:
        W /= np.sqrt(N / 3.0)
    return W


def coupling_gaussian(N: int, seed: int = 0, std: float | None = None,
                      dtype=np.float64) -> np.ndarray:
    """N x N: zero diagonal, i.i.d. normal entries of std 0.1/sqrt(N)."""
    g = rng(seed, STREAM_W)
    s = (0.1 / np.sqrt(N)) if std is None else std
    if dtype == np.float32:
        W = g.standard_normal(size=(N, N), dtype=np.float32)
        W *= np.float32(s)
    else:
        W = g.standard_normal(size=(N, N)) * s
    np.fill_diagonal(W, 0.0)
    return W


def input_weights(N: int, n_in: int = 1, seed: int = 0) -> np.ndarray:
    """N x n_in, i.i.d. U[-1, 1]."""
    return rng(seed, STREAM_WIN).uniform(-1.0, 1.0, size=(N, n_in))


def input_series(T: int, n_in: int = 1, seed: int = 0) -> np.ndarray:
    """T x n_in, i.i.d. U[0, 1]."""
    return rng(seed, STREAM_U).uniform(0.0, 1.0, size=(T, n_in))


def random_unit_states(N: int, seed: int = 0) -> np.ndarray:
    """(3, N): columns are normalised i.i.d. standard-normal 3-vectors."""
    v = rng(seed, STREAM_M0).standard_normal(size=(3, N))
    return v / np.linalg.norm(v, axis=0, keepdims=True)


def f32(a) -> np.ndarray:
    """Round to float32 (the values the CUDA path stores)."""
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def f32_exact64(a) -> np.ndarray:
    """The float32-rounded values, exactly widened back to float64."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def unit_f32(m) -> np.ndarray:
    """Round unit vectors to float32 (3, N) as stored by the CUDA path."""
    return f32(m)
