"""FP64 coupling (sto_create_f64): the precision of the paper's own benchmark
(Sec. 3.3, Table 1), against the FP64 oracle on the same float64 inputs.

Tolerances.  Double-float carries about 2^-47 ~ 7e-15 relative per
operation; W in the double-float product is the FP64 value rounded to 48
significand bits (relative 2^-48 ~ 3.6e-15).  One RK4 step of the torque
chains a few dozen such operations, so the increment m_{n+1} - m_n agrees to
about 1e-13 of its size: the test allows 1e-11.  Over 200 input samples of
100 RK4 steps (20000 steps, each adding ~1e-15 absolute) on a non-chaotic
Gaussian reservoir the error grows roughly linearly to ~1e-11: the test
allows 1e-9.  FP64 FMA (STO_PRODUCT_F64) differs from the oracle only in
the order of the row sums and in the double-float torque, so the same bars
apply.
"""
import numpy as np
import pytest

import oracle
from helpers import NTHREADS, oracle_params
from paper_2312_01121_b300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PRODUCTS = ["df64", "f64"]


@pytest.fixture(scope="module")
def sto():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2312_01121_b300 import build, sto as _sto
    build.build()
    _sto.load_library()
    return _sto


def system64(N, kind="paper", seed=0, T=4):
    """float64 W and m0 (used as given), float32 w_in and u."""
    W = inputs.coupling_paper(N, seed=seed) if kind == "paper" else inputs.coupling_gaussian(N, seed=seed)
    w_in = inputs.f32(inputs.input_weights(N, 1, seed=seed))
    m0 = inputs.random_unit_states(N, seed=seed)
    u = inputs.f32(inputs.input_series(T, 1, seed=seed))
    return np.ascontiguousarray(W), w_in, np.ascontiguousarray(m0), u


def gpu64(sto, P, W, w_in, m0, u, coupling, grid=0, T=None):
    N = W.shape[0]
    T = u.shape[0] if T is None else T
    st = np.zeros((max(T, 1), N), np.float32)
    with sto.Reservoir(W, w_in, P, m0=m0, coupling=coupling, grid=grid) as r:
        r.run(u, st, T=T)
        m = r.state()
        info = r.info()
    return m, st[:T], info


def orc64(P, W, w_in, m0, u):
    m_start = oracle.initial_state(W.shape[0]) if m0 is None else m0
    return oracle.run(oracle_params(P), W, w_in.astype(np.float64), np.array(m_start, np.float64),
                      u.astype(np.float64), nthreads=NTHREADS)


@pytest.mark.parametrize("coupling", PRODUCTS)
@pytest.mark.parametrize("N", [1, 8, 100, 333, 1000])
def test_one_rk4_step_matches_oracle(sto, coupling, N):
    W, w_in, m0, u = system64(N, "paper", seed=N, T=1)
    P = sto.Params(substeps=1, A_cp=50.0, A_in=20.0)
    m_gpu, _, info = gpu64(sto, P, W, w_in, m0, u, coupling)
    m_orc, _ = orc64(P, W, w_in, m0, u)
    inc_g, inc_o = m_gpu - m0, m_orc - m0
    scale = np.max(np.abs(inc_o))
    assert scale > 1e-4
    assert np.max(np.abs(inc_g - inc_o)) <= 1e-11 * scale, np.max(np.abs(inc_g - inc_o)) / scale
    assert info["panel_cols"] == 64 and info["w_bytes"] == 8 * N * N


@pytest.mark.parametrize("coupling", PRODUCTS)
def test_paper_benchmark_configuration(sto, coupling):
    """Sec. 3.3: u = 0, paper W (spectral radius 1), Eq. (initial) for every
    oscillator, dt = 1e-11 s; N = 1000, 100 RK4 steps."""
    N, T = 1000, 2
    W = inputs.coupling_paper(N, seed=3)
    w_in = inputs.f32(inputs.input_weights(N, 1, seed=3))
    u = np.zeros((T, 1), np.float32)
    P = sto.Params(substeps=50)
    m_gpu, st_gpu, _ = gpu64(sto, P, W, w_in, None, u, coupling)
    m_orc, st_orc = orc64(P, W, w_in, None, u)
    assert np.max(np.abs(m_gpu - m_orc)) <= 1e-11
    assert np.max(np.abs(st_gpu - st_orc.astype(np.float32))) <= 1e-7  # float32 samples


@pytest.mark.parametrize("coupling", PRODUCTS)
def test_first_200_input_samples(sto, coupling):
    N, T = 100, 200
    W, w_in, m0, u = system64(N, "gauss", seed=11, T=T)
    P = sto.Params(substeps=100, A_cp=1.0, A_in=1.0)
    m_gpu, _, _ = gpu64(sto, P, W, w_in, m0, u, coupling)
    m_orc, _ = orc64(P, W, w_in, m0, u)
    assert np.max(np.abs(m_gpu - m_orc)) <= 1e-9, np.max(np.abs(m_gpu - m_orc))


@pytest.mark.parametrize("coupling", PRODUCTS)
@pytest.mark.parametrize("N,grid", [(700, 4), (4099, 0), (130, 1)])
def test_streamed_ring_and_ragged_sizes(sto, coupling, N, grid):
    """Streamed W ring (grid 4: 175 rows x 700 x 8 B per CTA exceed shared
    memory), a ragged N past the on-chip limit, and one CTA."""
    W, w_in, m0, u = system64(N, "gauss", seed=N + grid, T=2)
    P = sto.Params(substeps=3, A_cp=80.0, A_in=10.0)
    m_gpu, st_gpu, info = gpu64(sto, P, W, w_in, m0, u, coupling, grid=grid)
    m_orc, st_orc = orc64(P, W, w_in, m0, u)
    if grid:
        assert info["grid"] == grid
    if N == 700:
        assert info["resident"] == 0
    assert np.max(np.abs(m_gpu - m_orc)) <= 1e-11
    assert np.max(np.abs(st_gpu - st_orc.astype(np.float32))) <= 1e-7


@pytest.mark.parametrize("coupling", PRODUCTS)
def test_full_size_n10000_launch_config(sto, coupling):
    """The benchmark's N = 10^4 launch (148 CTAs, streamed ring, part of W
    kept in L2): two RK4 steps against the oracle on the whole state."""
    N = 10000
    W = inputs.coupling_gaussian(N, seed=2)
    w_in = inputs.f32(inputs.input_weights(N, 1, seed=2))
    m0 = inputs.random_unit_states(N, seed=2)
    u = inputs.f32(inputs.input_series(1, 1, seed=2))
    P = sto.Params(substeps=2, A_cp=30.0)
    m_gpu, _, info = gpu64(sto, P, W, w_in, m0, u, coupling)
    assert info["resident"] == 0 and info["grid"] == info["sm_count"]
    m_orc, _ = orc64(P, W, w_in, m0, u)
    assert np.max(np.abs((m_gpu - m0) - (m_orc - m0))) <= 1e-11 * np.max(np.abs(m_orc - m0))


@pytest.mark.parametrize("coupling", PRODUCTS)
def test_resume_is_bitwise(sto, coupling):
    W, w_in, m0, u = system64(300, "gauss", seed=5, T=4)
    P = sto.Params(substeps=4, A_cp=40.0)
    a = np.zeros((4, 300), np.float32)
    with sto.Reservoir(W, w_in, P, m0=m0, coupling=coupling) as r:
        r.run(u, a)
        ma = r.state()
    b = np.zeros((4, 300), np.float32)
    with sto.Reservoir(W, w_in, P, m0=m0, coupling=coupling) as r:
        r.run(u[:2], b[:2])
        r.run(u[2:], b[2:])
        mb = r.state()
    assert np.array_equal(a, b) and np.array_equal(ma, mb)


def test_products_agree_and_differ_from_fp32(sto):
    """The two FP64 products agree far below the FP32 coupling's rounding."""
    W, w_in, m0, u = system64(500, "gauss", seed=6, T=3)
    P = sto.Params(substeps=20, A_cp=100.0)
    m_df, _, _ = gpu64(sto, P, W, w_in, m0, u, "df64")
    m_64, _, _ = gpu64(sto, P, W, w_in, m0, u, "f64")
    st = np.zeros((3, 500), np.float32)
    with sto.Reservoir(inputs.f32(W), w_in, P, m0=inputs.f32(m0)) as r:
        r.run(u, st)
    assert np.max(np.abs(m_df - m_64)) <= 1e-11
    assert np.max(np.abs(m_df - m_64)) < 1e-3 * np.max(np.abs(st[-1] - m_64[0]))


def test_group_with_fp64_handles(sto):
    """sto_run_group drives FP64 and FP32 handles alike, bit-equal to sto_run."""
    T = 2
    u = inputs.f32(inputs.input_series(T, 1, seed=9))
    specs = [(200, "df64"), (513, "f64"), (300, "f32")]
    P = sto.Params(substeps=3, A_cp=20.0)
    def make(N, c):
        W, w_in, m0, _ = system64(N, "gauss", seed=N, T=1)
        if c == "f32":
            W, m0 = inputs.f32(W), inputs.f32(m0)
        return sto.Reservoir(W, w_in, P, m0=m0, coupling=c)
    grp = [make(N, c) for N, c in specs]
    outs = [np.zeros((T, N), np.float32) for N, _ in specs]
    sto.sto_run_group(grp, u, T, outs)
    ends = [r.state() for r in grp]
    for r in grp:
        r.close()
    for (N, c), o, e in zip(specs, outs, ends):
        r = make(N, c)
        ref = np.zeros_like(o)
        r.run(u, ref)
        assert np.array_equal(o, ref) and np.array_equal(r.state(), e)
        r.close()


@pytest.mark.parametrize("coupling", PRODUCTS)
def test_adjoint_and_tableau_not_supported(sto, coupling):
    W, w_in, m0, u = system64(64, "gauss", seed=1, T=2)
    with sto.Reservoir(W, w_in, sto.Params(substeps=2), m0=m0, coupling=coupling) as r:
        with pytest.raises(sto.StoError) as e:
            r.adjoint(u, np.zeros((2, 64), np.float32), ckpt_every=1)
        assert e.value.code == sto.STO_ENOTSUP
        with pytest.raises(sto.StoError) as e:
            r.set_tableau([[0.0]], [1.0])
        assert e.value.code == sto.STO_ENOTSUP


def test_nonfinite_fp64_w_rejected(sto):
    W, w_in, m0, _ = system64(16, "gauss", seed=1, T=1)
    W[3, 5] = np.nan
    with pytest.raises(sto.StoError) as e:
        sto.Reservoir(W, w_in, sto.Params(), m0=m0, coupling="df64")
    assert e.value.code == sto.STO_ENONFINITE
