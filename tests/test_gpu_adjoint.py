"""The hand-written adjoint (sto_adjoint) on the GPU: against the FP64
oracle's adjoint, against finite differences of the GPU forward, invariance
under the checkpoint interval, and the torch.autograd wrapper."""
import os

import numpy as np
import pytest

import oracle
from helpers import make_system, oracle_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sto():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2312_01121_b300 import build, sto as _sto
    build.build()
    _sto.load_library()
    return _sto


def _rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("N,kind,comp,n_in", [(16, "paper", 0, 1), (40, "gauss", 2, 2),
                                             (300, "gauss", 0, 1)])
def test_adjoint_matches_oracle_adjoint(sto, N, kind, comp, n_in):
    T = 6
    W, w_in, m0, u = make_system(N, kind, seed=N, T=T, n_in=n_in)
    P = sto.Params(substeps=10, A_cp=80.0, A_in=40.0, alpha=0.02, sample_component=comp, n_in=n_in)
    G = np.random.default_rng(N).standard_normal((T, N)).astype(np.float32)
    with sto.Reservoir(W, w_in, P, m0=m0) as r:
        g = r.adjoint(u, G, ckpt_every=2)
    ref = oracle.adjoint(oracle_params(P), W.astype(np.float64), w_in.astype(np.float64),
                         m0.astype(np.float64), u.astype(np.float64), G.astype(np.float64),
                         nthreads=8)
    assert abs(g["A_cp"] - ref["A_cp"]) <= 1e-3 * abs(ref["A_cp"])
    assert abs(g["current"] - ref["current"]) <= 1e-3 * abs(ref["current"])
    assert _rel(g["w_in"], ref["w_in"]) <= 1e-3
    assert _rel(g["m0"], ref["m0"]) <= 1e-3


def test_checkpoint_interval_does_not_change_gradients(sto):
    N, T = 200, 7
    W, w_in, m0, u = make_system(N, "gauss", seed=5, T=T)
    P = sto.Params(substeps=8, A_cp=50.0)
    G = np.random.default_rng(1).standard_normal((T, N)).astype(np.float32)
    out = []
    for K in (1, 3, 7, 100):
        with sto.Reservoir(W, w_in, P, m0=m0) as r:
            out.append(r.adjoint(u, G, ckpt_every=K))
            m_end = r.state()
    with sto.Reservoir(W, w_in, P, m0=m0) as r:
        r.run(u)
        assert np.array_equal(r.state(), m_end)      # adjoint leaves the state like run
    for g in out[1:]:
        assert np.array_equal(g["m0"], out[0]["m0"]) and np.array_equal(g["w_in"], out[0]["w_in"])
        assert abs(g["A_cp"] - out[0]["A_cp"]) <= 1e-9 * abs(out[0]["A_cp"])
        assert abs(g["current"] - out[0]["current"]) <= 1e-9 * abs(out[0]["current"])


def test_overlapped_reverse_sweep_gives_the_sequential_bits(sto):
    """N = 1000 (W on chip, 63 CTAs, a pool of exchange-buffer placements):
    with several checkpoint segments the recomputation of segment g - 1 runs
    on a second stream beside the reverse pass of segment g; with one
    segment the sweep is sequential.  The checkpoint interval changes no
    arithmetic (test above), so every interval gives the same gradients."""
    N, T = 1000, 8
    W, w_in, m0, u = make_system(N, "gauss", seed=6, T=T)
    P = sto.Params(substeps=10, A_cp=50.0)
    G = np.random.default_rng(2).standard_normal((T, N)).astype(np.float32)
    out = []
    for K in (8, 1, 2, 3):  # 8: one segment, in sequence; the others overlapped
        with sto.Reservoir(W, w_in, P, m0=m0) as r:
            assert r.info()["grid"] > 1 and r.info()["resident"] == 1
            out.append((r.adjoint(u, G, ckpt_every=K), r.state()))
    for g, m in out[1:]:
        assert np.array_equal(m, out[0][1])
        assert np.array_equal(g["m0"], out[0][0]["m0"]) and np.array_equal(g["w_in"], out[0][0]["w_in"])
        assert abs(g["A_cp"] - out[0][0]["A_cp"]) <= 1e-9 * abs(out[0][0]["A_cp"])
        assert abs(g["current"] - out[0][0]["current"]) <= 1e-9 * abs(out[0][0]["current"])


def test_adjoint_matches_finite_differences_n1000(sto):
    """N = 1000, A_cp = 300: L = G . m^x after the last sample.
    (a) central differences (h = 1e-4 relative) of the FP64 oracle's forward;
    (b) central differences of the GPU forward itself, read as the exact FP64
        state, with h = 3e-3 relative: the FP32 coupling sums round at ~1e-7 of
        |W||x| per stage (~6e-5 Oe here), which is comparable to the field change
        of an h = 1e-4 step and would dominate such a difference quotient."""
    N, T = 1000, 5
    W, w_in, m0, u = make_system(N, "gauss", seed=7, T=T)
    P = sto.Params(substeps=20, A_cp=300.0, A_in=50.0)
    Gl = np.random.default_rng(7).standard_normal(N)
    G = np.zeros((T, N), np.float32)
    G[-1] = Gl
    with sto.Reservoir(W, w_in, P, m0=m0) as r:
        g = r.adjoint(u, G, ckpt_every=2)

        def L_gpu(params=P, win=w_in):
            r.set_params(params)
            r.set_input_weights(win)
            r.set_state(m0)
            r.run(u)
            return float(np.dot(Gl, r.state()[0]))

        OP = oracle_params(P)
        W64, w64, m64, u64 = (a.astype(np.float64) for a in (W, w_in, m0, u))

        def L_orc(op=OP, win=w64):
            m, _ = oracle.run(op, W64, win, m64, u64, nthreads=16)
            return float(np.dot(Gl, m[0]))

        for name, ofield, gfield in [("A_cp", "A_cp", "A_cp"), ("current", "I", "current")]:
            h = 1e-4 * getattr(OP, ofield)
            fd = (L_orc(OP.replace(**{ofield: getattr(OP, ofield) + h})) -
                  L_orc(OP.replace(**{ofield: getattr(OP, ofield) - h}))) / (2 * h)
            assert abs(g[name] - fd) <= 1e-3 * abs(fd), ("oracle", name, g[name], fd)
            h = 3e-3 * getattr(P, gfield)
            fd = (L_gpu(P.replace(**{gfield: getattr(P, gfield) + h})) -
                  L_gpu(P.replace(**{gfield: getattr(P, gfield) - h}))) / (2 * h)
            assert abs(g[name] - fd) <= 1e-3 * abs(fd), ("gpu", name, g[name], fd)
        for k in (0, 499):
            wp, wm = w64.copy(), w64.copy()
            wp[k, 0] += 1e-4
            wm[k, 0] -= 1e-4
            fd = (L_orc(win=wp) - L_orc(win=wm)) / 2e-4
            assert abs(g["w_in"][k, 0] - fd) <= 1e-3 * abs(fd) + 1e-6 * np.max(np.abs(g["w_in"]))


def test_autograd_function_gives_readout_loss_gradients(sto):
    from paper_2312_01121_b300 import autograd as ag
    N, T, washout = 100, 120, 20
    W, w_in, m0, u = make_system(N, "gauss", seed=9, T=T)
    dev = torch.device("cuda")
    P = sto.Params(substeps=10, A_in=60.0)
    y = torch.zeros(T, dtype=torch.float64, device=dev)
    y[5:] = torch.from_numpy(u[:-5, 0]).to(dev, torch.float64)
    ud = torch.from_numpy(u).to(dev)
    with sto.Reservoir(W, w_in, P, m0=m0) as r:
        A = torch.tensor(P.A_cp, dtype=torch.float64, requires_grad=True)
        I = torch.tensor(P.current, dtype=torch.float64, requires_grad=True)
        wt = torch.from_numpy(w_in.astype(np.float64)).to(dev).requires_grad_(True)
        st = ag.sto_states(r, A, I, wt, ud, ckpt_every=40)
        loss = ag.ridge_objective(st, y, washout, 1e-4)
        loss.backward()
        # the same number through the oracle adjoint of dLoss/dstates
        r.set_state(m0)
        st2 = torch.empty((T, N), device=dev)
        r.run(ud, st2)
        st2 = st2.detach().requires_grad_(True)
        ag.ridge_objective(st2, y, washout, 1e-4).backward()
        Gs = st2.grad.cpu().numpy()
    ref = oracle.adjoint(oracle_params(P), W.astype(np.float64), w_in.astype(np.float64),
                         m0.astype(np.float64), u.astype(np.float64), Gs, nthreads=8)
    assert abs(A.grad.item() - ref["A_cp"]) <= 1e-3 * abs(ref["A_cp"])
    assert abs(I.grad.item() - ref["current"]) <= 1e-3 * abs(ref["current"])
    assert _rel(wt.grad.cpu().numpy(), ref["w_in"]) <= 1e-3


def _golden(name):
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_adjoint_full_configuration_n1000_t2000(sto):
    """The benchmark's adjoint configuration: N = 1000, FP32, 2000 input
    samples of 100 RK4 steps (2e5 RK4 steps), checkpoint every 100 samples.
    (a) L = sum G * states with G ~ N(0, 1) over all samples: dA_cp, dI and
        dw_in against the FP64 oracle's adjoint of the same run, stored in
        tests/golden/adjoint_n1000_t2000.txt by make_adjoint_n1000_t2000.py
        (30 minutes of host time), within 1e-3;
    (b) the refitted ridge readout objective on y_t = u_{t-5} (washout 100)
        gives the same gradients with another checkpoint interval;
    (c) for G restricted to the first 1000 samples (the adjoint still sweeps
        all 20 checkpoint segments), central differences of the GPU forward
        within 1e-3: h = 1e-5 relative for A_cp, 1e-7 for I.
    Over 2e5 steps the reservoir is weakly chaotic: sensitivities grow ~47x
    from 1000 to 2000 samples, and differences of the FP32 forward over all
    2000 samples do not settle below ~2e-3 at any step (the truncation error
    needs h <= 1e-6, where the two perturbed runs' FP32 rounding, amplified
    by the dynamics, takes over), hence the oracle for the full horizon and
    differences over the first half."""
    from paper_2312_01121_b300 import autograd as ag
    N, T, washout, beta = 1000, 2000, 100, 1e-4
    W, w_in, m0, u = make_system(N, "gauss", seed=21, T=T)
    dev = torch.device("cuda")
    P = sto.Params(substeps=100)
    ud = torch.from_numpy(u).to(dev)
    G = np.random.default_rng(21).standard_normal((T, N)).astype(np.float32)
    gold = _golden("adjoint_n1000_t2000.txt")
    with sto.Reservoir(W, w_in, P, m0=m0) as r:
        g = r.adjoint(ud, torch.from_numpy(G).to(dev), ckpt_every=100, want_m0=False)
        for name, key in (("A_cp", "dA_cp"), ("current", "dcurrent")):
            assert abs(g[name] - gold[key]) <= 1e-3 * abs(gold[key]), (name, g[name], gold[key])
        scale = np.max(np.abs(g["w_in"]))
        for k in (0, 1, 499, 998):
            assert abs(g["w_in"][k, 0] - gold[f"dw_in_{k}"]) <= 1e-3 * scale, k

        y = torch.zeros(T, dtype=torch.float64, device=dev)
        y[5:] = torch.from_numpy(u[:-5, 0]).to(dev, torch.float64)
        grads = []
        for K in (100, 250):
            r.set_params(P)
            r.set_input_weights(w_in)
            r.set_state(m0)
            A = torch.tensor(P.A_cp, dtype=torch.float64, requires_grad=True)
            I = torch.tensor(P.current, dtype=torch.float64, requires_grad=True)
            wt = torch.from_numpy(w_in.astype(np.float64)).to(dev).requires_grad_(True)
            st = ag.sto_states(r, A, I, wt, ud, ckpt_every=K)
            ag.ridge_objective(st, y, washout, beta).backward()
            grads.append((A.grad.item(), I.grad.item(), wt.grad.cpu().numpy()))
        assert abs(grads[0][0] - grads[1][0]) <= 1e-9 * abs(grads[0][0])
        assert abs(grads[0][1] - grads[1][1]) <= 1e-9 * abs(grads[0][1])
        assert np.max(np.abs(grads[0][2] - grads[1][2])) <= 1e-9 * np.max(np.abs(grads[0][2]))

        G[1000:] = 0.0
        Gd = torch.from_numpy(G).to(dev)
        r.set_params(P)
        r.set_input_weights(w_in)
        r.set_state(m0)
        g_half = r.adjoint(ud, Gd, ckpt_every=100, want_w_in=False, want_m0=False)

        def L(params):
            r.set_params(params)
            r.set_input_weights(w_in)
            r.set_state(m0)
            st = torch.empty((T, N), dtype=torch.float32, device=dev)
            r.run(ud, st)
            return float((st.double() * Gd.double()).sum())

        for name, rel in (("A_cp", 1e-5), ("current", 1e-7)):
            h = rel * getattr(P, name)
            fd = (L(P.replace(**{name: getattr(P, name) + h})) - L(P.replace(**{name: getattr(P, name) - h}))) / (2 * h)
            assert abs(g_half[name] - fd) <= 1e-3 * abs(fd), (name, g_half[name], fd)
