"""Writes readout_n1000_t10000.txt next to this file: the FP64 oracle on the
plain-method readout workload — one reservoir of N = 1000 oscillators,
Gaussian W (std 0.1/sqrt(N), zero diagonal), w_in ~ U[-1, 1], random unit
initial state, 10^4 input samples u ~ U[0, 1] of 100 RK4 steps each, input
amplitude A_in = 30 Oe, the x component sampled after every input sample,
the Table defaults (Sec. 3.1) otherwise, seed 0 — and a ridge readout
(oracle/readout.py) of the delay-5 recall target y_t = u_{t-5}: washout 100,
trained on the first half of the remaining samples, scored (NMSE) on the
second half.

Over 10^4 samples the reservoir is chaotic (an initial difference of 1e-7
reaches O(1) within a few thousand samples), so the readout NMSE is a property
of the ensemble of equally valid trajectories, not of one of them.  The script
therefore runs the oracle K = 6 times: from the float32-rounded initial state
(run 0) and from five copies of it multiplied element-wise by
1 + 1e-7 xi, xi ~ N(0, 1) (runs 1-5, the size of FP32 rounding), and stores
every run's NMSE for beta_rel in {0.01, 0.1, 1}; plus run 0's states of every
50th oscillator over the first 200 input samples (the pointwise horizon).
Calls only the oracle and the seeded input generators; about 50 minutes on
8 host cores.

    python tests/golden/make_readout_n1000_t10000.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import readout  # noqa: E402
from paper_2312_01121_b300 import inputs  # noqa: E402  (seeded random numbers only)

N, T, SEED, S, A_IN, COMP = 1000, 10000, 0, 100, 30.0, 0
DELAY, WASHOUT, BETAS, RUNS, EPS = 5, 100, (0.01, 0.1, 1.0), 6, 1e-7
STRIDE, T_POINT = 50, 200
OUT = os.path.join(HERE, "readout_n1000_t10000.txt")


def system():
    """float32-rounded W, w_in, m0 (3, N), u (T, 1), widened to float64."""
    W = inputs.f32(inputs.coupling_gaussian(N, seed=SEED)).astype(np.float64)
    w_in = inputs.f32(inputs.input_weights(N, 1, seed=SEED)).astype(np.float64)
    m0 = inputs.f32(inputs.random_unit_states(N, seed=SEED)).astype(np.float64)
    u = inputs.f32(inputs.input_series(T, 1, seed=SEED)).astype(np.float64)
    return W, w_in, m0, u


def start_state(m0, k):
    if k == 0:
        return m0.copy()
    xi = np.random.default_rng([7, k]).standard_normal(m0.shape)
    return m0 * (1.0 + EPS * xi)


def main():
    W, w_in, m0, u = system()
    P = oracle.OracleParams(substeps=S, A_in=A_IN, component=COMP)
    t_start = time.time()
    lines = []
    for k in range(RUNS):
        _, states = oracle.run(P, W, w_in, start_state(m0, k), u, nthreads=os.cpu_count() or 1)
        for b in BETAS:
            _, n = readout.evaluate(states, u, washout=WASHOUT, delay=DELAY, beta_rel=b)
            lines.append(f"nmse {k} {b!r} {float(n)!r}\n")
        if k == 0:
            for t in range(T_POINT):
                for i in range(0, N, STRIDE):
                    lines.append(f"s {t} {i} {float(states[t, i])!r}\n")
        print(f"run {k} done at {time.time() - t_start:.0f} s", flush=True)
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle, N=1000, T=10000 input samples x 100 RK4 steps, Gaussian W (std 0.1/sqrt(N)),\n")
        fh.write(f"# A_in={A_IN} Oe, component x, seed {SEED}; delay-{DELAY} recall, washout {WASHOUT}, "
                 "first half trains, second half scores\n")
        fh.write(f"# runs 1-{RUNS - 1}: m0 * (1 + {EPS} xi); (written by make_readout_n1000_t10000.py, "
                 f"{time.time() - t_start:.0f} s)\n")
        fh.write("# nmse run beta_rel value | s t k value (run 0, states of every 50th oscillator)\n")
        fh.writelines(lines)


if __name__ == "__main__":
    main()
