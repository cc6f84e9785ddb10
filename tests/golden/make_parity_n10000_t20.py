"""Writes parity_n10000_t20.txt next to this file: the FP64 oracle's sampled
states of the largest single-reservoir workload over its first 20 input
samples — N = 10^4 oscillators, Gaussian W (std 0.1/sqrt(N), zero diagonal),
w_in ~ U[-1, 1], random unit initial state, u ~ U[0, 1], 100 RK4 steps of
1e-11 s per sample, the Table defaults (Sec. 3.1) otherwise, seed 0; every
array rounded to float32 first, as the library stores it.

Stored: states[t, k] (the m^x sample after input sample t, Sec. 3.1) for
every t < 20 and every 37th oscillator k, and the FP64 end state of the same
oscillators.  Calls only the oracle and the seeded input generators; about
10 to 20 minutes on 8 host cores (8000 stages of a 10^4 x 10^4 FP64 matvec).

    python tests/golden/make_parity_n10000_t20.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2312_01121_b300 import inputs  # noqa: E402  (seeded random numbers only)

N, T, SEED, S, STRIDE = 10000, 20, 0, 100, 37
OUT = os.path.join(HERE, "parity_n10000_t20.txt")


def system():
    """float32-rounded W, w_in, m0 (3, N), u (T, 1), widened to float64."""
    W = inputs.f32(inputs.coupling_gaussian(N, seed=SEED)).astype(np.float64)
    w_in = inputs.f32(inputs.input_weights(N, 1, seed=SEED)).astype(np.float64)
    m0 = inputs.f32(inputs.random_unit_states(N, seed=SEED)).astype(np.float64)
    u = inputs.f32(inputs.input_series(T, 1, seed=SEED)).astype(np.float64)
    return W, w_in, m0, u


def main():
    W, w_in, m0, u = system()
    t0 = time.time()
    m, states = oracle.run(oracle.OracleParams(substeps=S), W, w_in, m0, u,
                           nthreads=os.cpu_count() or 1)
    ks = np.arange(0, N, STRIDE)
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle, N=10000, first 20 input samples x 100 RK4 steps, Gaussian W "
                 "(std 0.1/sqrt(N)),\n")
        fh.write(f"# seed {SEED}, Table defaults; oscillators k = 0, {STRIDE}, ... "
                 f"(written by make_parity_n10000_t20.py, {time.time() - t0:.0f} s)\n")
        fh.write("# states t k value\n")
        for t in range(T):
            for k in ks:
                fh.write(f"s {t} {k} {float(states[t, k])!r}\n")
        fh.write("# end state: component k value\n")
        for c in range(3):
            for k in ks:
                fh.write(f"m {c} {k} {float(m[c, k])!r}\n")


if __name__ == "__main__":
    main()
