"""The CUDA row block (sto_shard_*, through the C ABI and
paper_2312_01121_b300/shard.py) against the FP64 oracle: one block holding
every row (a single rank, no collective), and several blocks on one GPU whose
stage values this test gathers between stages (each stage is one kernel per
block; no kernel waits on another).  Tolerance 1e-5 over a few input samples,
as for the single-reservoir stepper; the block and the stepper share the
double-float arithmetic and differ only in the order of the FP32 row sums."""
import numpy as np
import pytest

from helpers import make_system, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sto():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2312_01121_b300 import build, sto as _sto
    build.build()
    _sto.load_library()
    return _sto


def dev_arrays(*arrays):
    d = torch.device("cuda")
    return [torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in arrays]


@pytest.mark.parametrize("N,kind", [(1, "paper"), (7, "paper"), (100, "gauss"), (1000, "gauss"),
                                    (2501, "gauss")])
def test_single_block_equals_oracle(sto, N, kind):
    from paper_2312_01121_b300.shard import ShardedReservoir
    T = 3
    W, w_in, m0, u = make_system(N, kind, seed=N + 3, T=T)
    P = sto.Params(substeps=5, A_cp=100.0, A_in=20.0)
    Wd, wd, md, ud = dev_arrays(W, w_in, m0, u)
    res = ShardedReservoir(N, P, W_rows=Wd, w_in_rows=wd, m0_rows=md)
    assert (res.world, res.row0, res.rows) == (1, 0, N)
    st = torch.zeros((T, N), dtype=torch.float32, device="cuda")
    res.run(ud, st)
    torch.cuda.synchronize()
    m_orc, st_orc = run_oracle(P, W, w_in, m0, u)
    assert np.max(np.abs(st.cpu().numpy() - st_orc)) <= 1e-5
    assert np.max(np.abs(res.state() - m_orc)) <= 1e-5


def run_blocks_on_one_gpu(P, W, w_in, m0, u, world):
    """`world` row blocks on this GPU; the stage values are gathered by a
    device copy between stages (what the all-gather does across GPUs)."""
    from paper_2312_01121_b300.shard import SAMPLE_END, SAMPLE_START, CudaBlock, partition
    N, T, S = W.shape[0], u.shape[0], P.substeps
    parts = partition(N, world)
    chunk = -(-N // world)
    blocks = []
    for r0, n in parts:
        Wr, wr, mr = dev_arrays(W[r0:r0 + n], w_in[r0:r0 + n], m0[:, r0:r0 + n])
        blocks.append(CudaBlock(N, r0, n, P, Wr, wr, mr))
    x = torch.zeros(world * chunk + 4, dtype=torch.float32, device="cuda")
    own = [torch.zeros(chunk, dtype=torch.float32, device="cuda") for _ in parts]
    outs = [torch.zeros((T, n), dtype=torch.float32, device="cuda") for _, n in parts]
    ud = dev_arrays(u)[0]

    def gather():
        x[:world * chunk] = torch.cat(own)

    for b, o in zip(blocks, own):
        b.publish(o)
    gather()
    for t in range(T):
        for j in range(S):
            for stg in range(4):
                flags = (SAMPLE_START if (j == 0 and stg == 0) else 0) | (SAMPLE_END if (j == S - 1 and stg == 3) else 0)
                for b, o, so in zip(blocks, own, outs):
                    b.stage(x, stg, ud[t] if flags & SAMPLE_START else None, flags, o,
                            so[t] if flags & SAMPLE_END else None)
                gather()
    torch.cuda.synchronize()
    states = np.hstack([so.cpu().numpy() for so in outs])
    m = np.hstack([b.state() for b in blocks])
    return states, m


@pytest.mark.parametrize("N,world", [(1001, 3), (256, 2), (10, 4)])
def test_blocks_on_one_gpu_equal_oracle(sto, N, world):
    T = 3
    W, w_in, m0, u = make_system(N, "gauss", seed=N, T=T, n_in=2)
    P = sto.Params(substeps=4, A_cp=120.0, A_in=15.0, n_in=2, sample_component=1)
    st, m = run_blocks_on_one_gpu(P, W, w_in, m0, u, world)
    m_orc, st_orc = run_oracle(P, W, w_in, m0, u)
    assert np.max(np.abs(st - st_orc)) <= 1e-5
    assert np.max(np.abs(m - m_orc)) <= 1e-5


def test_full_size_n10000_two_blocks(sto):
    """N = 10^4 as two row blocks of 5000 rows: one input sample of 2 RK4 steps."""
    N = 10000
    W, w_in, m0, u = make_system(N, "gauss", seed=0, T=1)
    P = sto.Params(substeps=2)
    st, m = run_blocks_on_one_gpu(P, W, w_in, m0, u, 2)
    m_orc, st_orc = run_oracle(P, W, w_in, m0, u)
    assert np.max(np.abs(st - st_orc)) <= 1e-5
    assert np.max(np.abs(m - m_orc)) <= 1e-5


def test_blocks_track_the_persistent_stepper(sto):
    """30 input samples at N = 1000: the block path and sto_run (one persistent
    launch) agree to 1e-5; both carry the same double-float state and differ
    only in the order of the FP32 row sums."""
    from paper_2312_01121_b300.shard import ShardedReservoir
    N, T = 1000, 30
    W, w_in, m0, u = make_system(N, "gauss", seed=1, T=T)
    P = sto.Params(substeps=20, A_cp=80.0, A_in=20.0)
    m_ref, st_ref = run_gpu(P, W, w_in, m0, u)
    Wd, wd, md, ud = dev_arrays(W, w_in, m0, u)
    res = ShardedReservoir(N, P, W_rows=Wd, w_in_rows=wd, m0_rows=md)
    st = torch.zeros((T, N), dtype=torch.float32, device="cuda")
    res.run(ud, st)
    torch.cuda.synchronize()
    assert np.max(np.abs(st.cpu().numpy() - st_ref)) <= 1e-5
    assert np.max(np.abs(res.state() - m_ref)) <= 1e-5


def test_shard_argument_errors(sto):
    import ctypes
    from paper_2312_01121_b300.shard import CudaBlock
    lib = sto.load_library()
    N = 12
    W, w_in, m0, u = make_system(N, "gauss", seed=2, T=1)
    Wd, wd, md, ud = dev_arrays(W, w_in, m0, u)
    cp = sto.Params().to_c()
    h = ctypes.c_void_p()
    for row0, rows in ((-1, 3), (0, 0), (10, 3)):
        assert lib.sto_shard_create(N, row0, rows, ctypes.byref(cp), Wd.data_ptr(), wd.data_ptr(), None, None,
                                    ctypes.byref(h)) == sto.STO_EINVAL
    Wbad = W.copy()
    Wbad[1, 2] = np.inf
    with pytest.raises(sto.StoError) as e:
        CudaBlock(N, 0, N, sto.Params(), dev_arrays(Wbad)[0], wd, md)
    assert e.value.code == sto.STO_ENONFINITE
    b = CudaBlock(N, 0, N, sto.Params(), Wd, wd, md)
    x = torch.zeros(N + 8, dtype=torch.float32, device="cuda")
    o = torch.zeros(N, dtype=torch.float32, device="cuda")
    xh = torch.zeros(N + 8, dtype=torch.float32)
    cases = [(x, 4, None, 0),          # no stage 4
             (x[1:], 0, None, 0),      # x not 16-byte aligned
             (xh, 0, None, 0),         # x in host memory
             (x, 1, ud[0], 1),         # the input is taken at stage 0 only
             (x, 2, None, 2)]          # sampling after stage 3 only
    for xx, stg, ut, fl in cases:
        rc = lib.sto_shard_stage(b.handle, xx.data_ptr(), stg, ut.data_ptr() if ut is not None else None, fl,
                                 o.data_ptr(), None)
        assert rc == sto.STO_EINVAL, (stg, fl)
    b.close()


@pytest.mark.parametrize("N,T,S", [(1000, 4, 10), (10000, 1, 2)])
def test_graph_replay_equals_the_launch_loop(sto, N, T, S):
    """run(graph=True) captures one input sample (4 S stage launches and
    exchanges) as a CUDA graph and replays it per sample: the same bits as
    the launch loop, and the oracle's states."""
    from paper_2312_01121_b300.shard import ShardedReservoir
    W, w_in, m0, u = make_system(N, "gauss", seed=N + 7, T=T)
    P = sto.Params(substeps=S, A_cp=90.0, A_in=20.0)
    Wd, wd, md, ud = dev_arrays(W, w_in, m0, u)
    outs = []
    for graph in (False, True):
        res = ShardedReservoir(N, P, W_rows=Wd, w_in_rows=wd, m0_rows=md)
        st = torch.zeros((T, N), dtype=torch.float32, device="cuda")
        res.run(ud, st, graph=graph)
        torch.cuda.synchronize()
        outs.append((st.cpu().numpy(), res.state()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    m_orc, st_orc = run_oracle(P, W, w_in, m0, u)
    assert np.max(np.abs(outs[1][0] - st_orc)) <= 1e-5
    assert np.max(np.abs(outs[1][1] - m_orc)) <= 1e-5
