"""The largest reservoirs the automatic plan accepts, against the oracle.

On a B300 (148 SMs, 232448 bytes of shared memory a CTA may have) the
stepper's rows per CTA are bounded by its shared-memory ring: at least two
slots of R_max x 512-byte panel rows, beside the stage values of all N
oscillators.
- FP32 coupling: the largest N is 21164, with 143 rows per CTA, 2 slots and
  232048 bytes; its rows per warp (10) run in the 16-row instantiation.
- FP64-class couplings (8-byte elements, 64 per panel row): the largest N
  is 15488, with 105 rows per CTA and 232336 bytes.
One more oscillator returns STO_ENOTSUP at create.  These sizes come from
the library's planner; the tests check that the plan really sits at the
limit, and then every output of a short run against the oracle.
"""
import numpy as np
import pytest

import oracle
from helpers import NTHREADS, make_system, oracle_params, run_gpu, run_oracle
from paper_2312_01121_b300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_F32_MAX = 21164
N_F64_MAX = 15488


@pytest.fixture(scope="module")
def sto():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    props = torch.cuda.get_device_properties(0)
    if props.multi_processor_count != 148:
        pytest.skip("the limits are those of a 148-SM part")
    from paper_2312_01121_b300 import build, sto as _sto
    build.build()
    _sto.load_library()
    return _sto


def test_largest_fp32_reservoir(sto):
    """N = 21164: the plan uses 148 CTAs of 143 rows and 2 ring slots; one
    input sample of 2 RK4 steps matches the oracle to 1e-5 in every state;
    N = 21165 is refused."""
    N = N_F32_MAX
    W, w_in, m0, u = make_system(N, "gauss", seed=21, T=1)
    P = sto.Params(substeps=2, A_cp=50.0)
    dev = torch.device("cuda")
    Wt = torch.from_numpy(W).to(dev)
    with sto.Reservoir(Wt, torch.from_numpy(w_in).to(dev), P, m0=torch.from_numpy(m0).to(dev)) as r:
        info = r.info()
    assert (info["grid"], info["rows_max"], info["ring_slots"], info["resident"]) == (148, 143, 2, 0)
    assert info["smem_bytes"] == 232048
    del Wt
    m_gpu, st_gpu = run_gpu(P, W, w_in, m0, u)
    m_orc, st_orc = run_oracle(P, W, w_in, m0, u)
    assert np.max(np.abs(st_gpu - st_orc)) <= 1e-5
    assert np.max(np.abs(m_gpu - m_orc)) <= 1e-5
    del W
    Z = torch.zeros((N + 1, N + 1), dtype=torch.float32, device=dev)
    zin = torch.zeros((N + 1, 1), dtype=torch.float32, device=dev)
    with pytest.raises(sto.StoError) as e:
        sto.Reservoir(Z, zin, P)
    assert e.value.code == sto.STO_ENOTSUP


@pytest.mark.parametrize("coupling", ["df64", "f64"])
def test_largest_fp64_reservoir(sto, coupling):
    """N = 15488 with the FP64-class couplings: 148 CTAs of 105 rows, 2 ring
    slots; one input sample of 2 RK4 steps from float64 inputs matches the
    FP64 oracle to 1e-11 (the FP64 replica's one-step bar); N = 15489 is
    refused."""
    N = N_F64_MAX
    W = np.ascontiguousarray(inputs.coupling_gaussian(N, seed=22))
    w_in = inputs.f32(inputs.input_weights(N, 1, seed=22))
    m0 = np.ascontiguousarray(inputs.random_unit_states(N, seed=22))
    u = inputs.f32(inputs.input_series(1, 1, seed=22))
    P = sto.Params(substeps=2, A_cp=50.0)
    st = np.zeros((1, N), np.float32)
    with sto.Reservoir(W, w_in, P, m0=m0, coupling=coupling) as r:
        info = r.info()
        r.run(u, st)
        m = r.state()
    assert (info["grid"], info["rows_max"], info["ring_slots"], info["resident"]) == (148, 105, 2, 0)
    m_orc, st_orc = oracle.run(oracle_params(P), W, w_in.astype(np.float64), m0, u.astype(np.float64),
                               nthreads=NTHREADS)
    assert np.max(np.abs(m - m_orc)) <= 1e-11
    assert np.max(np.abs(st - st_orc)) <= 1e-6  # the sampled states are FP32
    del W
    Z = np.zeros((N + 1, N + 1), np.float64)
    with pytest.raises(sto.StoError) as e:
        sto.Reservoir(Z, np.zeros((N + 1, 1), np.float32), P, coupling=coupling)
    assert e.value.code == sto.STO_ENOTSUP


def test_largest_sweep(sto):
    """R N = 2^29 (R = 32768 reservoirs sharing one N = 16384 W), the largest
    batch the sweep's 32-bit per-pair offsets allow: its state is 38.6 GB,
    formed on the device.  One RK4 step with BN = 40 (a ragged last tile of
    8 reservoirs); three sampled reservoirs against the oracle on the
    BF16-rounded W (1e-5).  One reservoir more is refused."""
    N, R = 16384, 32768
    W, w_in, _, u = make_system(N, "gauss", seed=23, T=1)
    rng = np.random.default_rng(23)
    cur = rng.uniform(1e-3, 3e-3, R)
    gain = rng.uniform(0.5, 2.0, R)
    P = sto.Params(substeps=1, A_cp=50.0, A_in=20.0)
    dev = torch.device("cuda")
    st = torch.zeros((1, R, N), dtype=torch.float32, device=dev)
    sw = sto.Sweep(W, w_in, P, currents=cur, gains=gain)
    try:
        sw.set_plan(40, 3, 2, 1, 512)
        sw.run(u, st)
        picks = (0, R // 2 - 1, R - 1)
        got = {r: st[0, r].cpu().numpy() for r in picks}
    finally:
        sw.close()
    del st
    Wb = torch.from_numpy(W).to(torch.bfloat16).float().numpy().astype(np.float64)
    m0 = np.asarray(oracle.initial_state(N), np.float64)
    for r in picks:
        OP = oracle_params(P.replace(current=float(cur[r]), input_gain=float(gain[r])))
        _, ref = oracle.run(OP, Wb, w_in.astype(np.float64), m0, u.astype(np.float64), nthreads=NTHREADS)
        assert np.max(np.abs(got[r] - ref[0])) <= 1e-5, r
    del Wb
    with pytest.raises(sto.StoError) as e:
        sto.Sweep(W, w_in, P, currents=np.full(R + 1, 2e-3))
    assert e.value.code == sto.STO_ENOTSUP
