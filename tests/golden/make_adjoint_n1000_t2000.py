"""Writes adjoint_n1000_t2000.txt next to this file: the FP64 oracle's
discrete adjoint (exact gradients of L = sum_{t,k} G[t,k] states[t,k]) for
the benchmark's adjoint configuration — N = 1000 oscillators, Gaussian W
(std 0.1/sqrt(N), zero diagonal), 2000 input samples of 100 RK4 steps, the
Table defaults (Sec. 3.1) — with G ~ N(0, 1) i.i.d., everything seeded with
21.  Calls only the oracle and the seeded input generators; about 30 minutes
on 8 host cores (the oracle keeps the 2e5-step trajectory, 4.8 GB).

    python tests/golden/make_adjoint_n1000_t2000.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2312_01121_b300 import inputs  # noqa: E402  (seeded random numbers only)

N, T, SEED, S = 1000, 2000, 21, 100


def main():
    W = inputs.f32(inputs.coupling_gaussian(N, seed=SEED)).astype(np.float64)
    w_in = inputs.f32(inputs.input_weights(N, 1, seed=SEED)).astype(np.float64)
    m0 = inputs.f32(inputs.random_unit_states(N, seed=SEED)).astype(np.float64)
    u = inputs.f32(inputs.input_series(T, 1, seed=SEED)).astype(np.float64)
    G = np.random.default_rng(SEED).standard_normal((T, N)).astype(np.float32).astype(np.float64)
    t0 = time.time()
    g = oracle.adjoint(oracle.OracleParams(substeps=S), W, w_in, m0, u, G, nthreads=os.cpu_count() or 1)
    with open(os.path.join(HERE, "adjoint_n1000_t2000.txt"), "w") as fh:
        fh.write("# FP64 oracle discrete adjoint, N=1000, T=2000 samples x 100 RK4 steps, Gaussian W,\n")
        fh.write("# seed 21, L = sum G * states with G ~ N(0,1) (written by make_adjoint_n1000_t2000.py,\n")
        fh.write(f"# {time.time() - t0:.0f} s)\n")
        fh.write(f"dA_cp {float(g['A_cp'])!r}\n")
        fh.write(f"dcurrent {float(g['current'])!r}\n")
        for k in (0, 1, 499, 998):
            fh.write(f"dw_in_{k} {float(g['w_in'][k, 0])!r}\n")


if __name__ == "__main__":
    main()
