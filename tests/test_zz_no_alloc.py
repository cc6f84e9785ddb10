"""sto_run_noalloc: the allocation-free entry point for callers that must not
allocate device memory (a framework's pool allocator owns the device, a
real-time loop cannot afford cudaMalloc's implicit synchronisation, or a
plug-in may only use the buffers it is given).

It is checked through the C ABI against the handle-based sto_run and against
the FP64 oracle on the same inputs, over two consecutive calls that continue
from the state the first one left, with the tolerance the other parity tests
use (1e-5), and a call after the first must leave the device's free memory
unchanged.  The file is named to be collected last, and it passes alone in a
fresh process as well as after the other tests.
"""
import numpy as np
import pytest

from helpers import make_system, run_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sto():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2312_01121_b300 import build, sto as _sto
    build.build()
    _sto.load_library()
    return _sto


@pytest.mark.parametrize("N", [1000, 4100])   # W resident on chip / streamed through the ring
def test_noalloc_matches_sto_run_on_two_calls(sto, N):
    T1, T2 = 3, 2
    W, w_in, m0, u = make_system(N, "gauss", seed=21, T=T1 + T2)
    P = sto.Params(substeps=4, A_cp=80.0, A_in=20.0)
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    Wd, wd = torch.from_numpy(W).to(dev), torch.from_numpy(w_in).to(dev)
    ud = torch.from_numpy(u).to(dev)

    # reference: the handle-based entry point
    ref1 = torch.zeros((T1, N), dtype=torch.float32, device=dev)
    ref2 = torch.zeros((T2, N), dtype=torch.float32, device=dev)
    with sto.Reservoir(Wd, wd, P, m0=torch.from_numpy(m0).to(dev), stream=stream) as r:
        r.run(ud[:T1], ref1)
        r.run(ud[T1:], ref2)
        m_ref = r.state()

    # the allocation-free entry point on caller-owned buffers
    state = torch.from_numpy(m0.astype(np.float64)).to(dev)
    out1 = torch.zeros((T1, N), dtype=torch.float32, device=dev)
    out2 = torch.zeros((T2, N), dtype=torch.float32, device=dev)
    sto.sto_run_noalloc(N, P, Wd, wd, state, ud[:T1], T1, out1, stream)
    sto.sto_run_noalloc(N, P, Wd, wd, state, ud[T1:], T2, out2, stream)
    torch.cuda.synchronize()

    assert torch.max(torch.abs(out1 - ref1)).item() <= 1e-5
    assert torch.max(torch.abs(out2 - ref2)).item() <= 1e-5
    assert np.max(np.abs(state.cpu().numpy() - m_ref)) <= 1e-5

    # and against the FP64 oracle over the same five samples
    m_orc, st_orc = run_oracle(P, W, w_in, m0, u)
    got = np.vstack([out1.cpu().numpy(), out2.cpu().numpy()])
    assert np.max(np.abs(got - st_orc)) <= 1e-5
    assert np.max(np.abs(state.cpu().numpy() - m_orc)) <= 1e-5


def test_noalloc_call_allocates_no_device_memory(sto):
    """After the first call on the device (which looks up the static array),
    a call leaves the device's free memory exactly as it was."""
    N, T = 1000, 2
    W, w_in, m0, u = make_system(N, "gauss", seed=22, T=T)
    P = sto.Params(substeps=3, A_cp=50.0)
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    Wd, wd, ud = torch.from_numpy(W).to(dev), torch.from_numpy(w_in).to(dev), torch.from_numpy(u).to(dev)
    state = torch.from_numpy(m0.astype(np.float64)).to(dev)
    out = torch.zeros((T, N), dtype=torch.float32, device=dev)
    sto.sto_run_noalloc(N, P, Wd, wd, state, ud, T, out, stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        sto.sto_run_noalloc(N, P, Wd, wd, state, ud, T, out, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_sizes_beyond_its_scratch(sto):
    """The library's own checks, called through the C ABI directly (the Python
    binding would already refuse these arrays for their extents)."""
    import ctypes
    lib = sto.load_library()
    cp = sto.Params().to_c()
    dev = torch.device("cuda")
    tiny = torch.zeros(16, dtype=torch.float32, device=dev)
    st = torch.zeros(3 * 16, dtype=torch.float64, device=dev)
    p = tiny.data_ptr()
    assert lib.sto_run_noalloc(16388, ctypes.byref(cp), p, p, st.data_ptr(), p, 1, None,
                               None) == sto.STO_ETOOBIG
    # N must be a multiple of 4
    assert lib.sto_run_noalloc(6, ctypes.byref(cp), p, p, st.data_ptr(), p, 1, None,
                               None) == sto.STO_EINVAL
