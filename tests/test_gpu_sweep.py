"""The batched sweep (sto_run_batched): every reservoir against the FP64
oracle run with the same BF16-rounded W and that reservoir's current and
input gain; the sweep against the single-reservoir stepper."""
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


def bf16_round(W):
    return torch.from_numpy(np.ascontiguousarray(W, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def _sweep_vs_oracle(sto, N, R, T, S, A_cp, tol, seed=0, n_in=1, A_in=30.0):
    W, w_in, _, u = make_system(N, "gauss", seed=seed, T=T, n_in=n_in)
    rng = np.random.default_rng(seed)
    cur = rng.uniform(1e-3, 3e-3, R)
    gain = rng.uniform(0.5, 2.0, R)
    m0 = np.stack([make_system(N, "gauss", seed=seed + 100 + r, T=1, n_in=n_in)[2] for r in range(R)])
    P = sto.Params(substeps=S, A_cp=A_cp, A_in=A_in, n_in=n_in)
    st = np.zeros((T, R, N), np.float32)
    with sto.Sweep(W, w_in, P, currents=cur, gains=gain, m0=m0) as sw:
        sw.run(u, st)
        m_end = sw.state()
    Wb = bf16_round(W).astype(np.float64)
    for r in range(R):
        OP = oracle_params(P.replace(current=float(cur[r]), input_gain=float(gain[r])))
        m, ref = oracle.run(OP, Wb, w_in.astype(np.float64), m0[r].astype(np.float64),
                            u.astype(np.float64), nthreads=8)
        assert np.max(np.abs(st[:, r] - ref)) <= tol, r
        assert np.max(np.abs(m_end[r] - m)) <= tol, r


def test_sweep_matches_oracle_per_reservoir(sto):
    _sweep_vs_oracle(sto, N=200, R=6, T=3, S=10, A_cp=50.0, tol=1e-5)


def test_sweep_ragged_tiles(sto):
    """N not a multiple of the 128 x 64 tile, R not a multiple of 64."""
    _sweep_vs_oracle(sto, N=300, R=70, T=2, S=4, A_cp=100.0, tol=1e-5, seed=3)
    _sweep_vs_oracle(sto, N=1000, R=65, T=1, S=3, A_cp=100.0, tol=1e-5, seed=4)


@pytest.mark.parametrize("N,R", [(1, 3), (8, 5), (64, 9), (129, 17), (256, 40)])
def test_sweep_small_and_k_padded_sizes(sto, N, R):
    """N below one 128-row tile and around the 128-wide K padding of a ring
    slot (two 64-wide K slices): one slot per tile for N <= 128, two for
    129 <= N <= 256; N = 1 has W = [0] (Sec. 3.1: no self-coupling)."""
    _sweep_vs_oracle(sto, N=N, R=R, T=2, S=4, A_cp=60.0, tol=1e-5, seed=30 + N)


def test_sweep_first_200_input_samples(sto):
    """The paper's A_in = 1 Oe: outside the chaotic regime (with A_in = 30 Oe
    the FP64 oracle perturbed by 1e-7 in W itself drifts by 1e-4..5e-2 within
    200 samples, where only the readout NMSE can be compared)."""
    _sweep_vs_oracle(sto, N=100, R=3, T=200, S=100, A_cp=1.0, tol=1e-4, seed=5, A_in=1.0)


def test_sweep_equals_single_reservoir_stepper(sto):
    """R = 1 sweep vs the plain stepper given the BF16-rounded W."""
    N, T = 500, 3
    W, w_in, m0, u = make_system(N, "gauss", seed=8, T=T)
    P = sto.Params(substeps=5, A_cp=80.0)
    st = np.zeros((T, 1, N), np.float32)
    with sto.Sweep(W, w_in, P, currents=[P.current], m0=m0[None]) as sw:
        sw.run(u, st)
    ref = np.zeros((T, N), np.float32)
    with sto.Reservoir(bf16_round(W), w_in, P, m0=m0) as r:
        r.run(u, ref)
    assert np.max(np.abs(st[:, 0] - ref)) <= 1e-5


def test_sweep_resumes_across_calls(sto):
    N, R, T = 128, 5, 4
    W, w_in, m0, u = make_system(N, "gauss", seed=9, T=T)
    P = sto.Params(substeps=3, A_cp=20.0)
    cur = np.linspace(1e-3, 3e-3, R)
    a = np.zeros((T, R, N), np.float32)
    with sto.Sweep(W, w_in, P, currents=cur) as sw:
        sw.run(u, a)
    b1 = np.zeros((2, R, N), np.float32)
    b2 = np.zeros((2, R, N), np.float32)
    with sto.Sweep(W, w_in, P, currents=cur) as sw:
        sw.run(u[:2], b1)
        sw.run(u[2:], b2)
    assert np.array_equal(np.concatenate([b1, b2]), a)


def test_group_of_own_w_reservoirs_matches_separate_runs(sto):
    """Reservoirs with their own W and uneven N in one graph-captured call
    give the same bits as separate sto_run calls, and match the oracle."""
    Ns = [100, 333, 1000, 2049, 4000]
    T = 2
    u = make_system(4, "gauss", seed=1, T=T)[3]
    systems = [make_system(N, "gauss", seed=20 + i, T=T) for i, N in enumerate(Ns)]
    params = [sto.Params(substeps=4, current=1e-3 + 4e-4 * i, A_cp=30.0) for i in range(len(Ns))]
    grp = [sto.Reservoir(W, w_in, P, m0=m0) for (W, w_in, m0, _), P in zip(systems, params)]
    outs = [np.zeros((T, N), np.float32) for N in Ns]
    sto.sto_run_group(grp, u, T, outs)
    ends = [r.state() for r in grp]
    for r in grp:
        r.close()
    for (W, w_in, m0, _), P, o, e in zip(systems, params, outs, ends):
        ref = np.zeros_like(o)
        with sto.Reservoir(W, w_in, P, m0=m0) as r:
            r.run(u, ref)
            assert np.array_equal(r.state(), e)
        assert np.array_equal(o, ref)
    W, w_in, m0, _ = systems[0]
    _, orc = oracle.run(oracle_params(params[0]), W.astype(np.float64), w_in.astype(np.float64),
                        m0.astype(np.float64), u.astype(np.float64))
    assert np.max(np.abs(outs[0] - orc)) <= 1e-5


@pytest.mark.parametrize("tile_n,slots,groups", [(16, 3, 1), (32, 4, 1), (48, 3, 1), (80, 2, 1), (80, 3, 1),
                                                 (64, 3, 1), (16, 5, 1), (112, 2, 1), (128, 2, 1), (16, 4, 2),
                                                 (24, 3, 2), (40, 2, 2), (48, 3, 2), (32, 4, 2), (24, 3, 1),
                                                 (56, 3, 2), (8 * 7, 2, 1)])
def test_sweep_forced_plans_match_oracle(sto, tile_n, slots, groups):
    """Every tile width, ring depth (also depths that are not a multiple of
    the three copy warps, which then own unequal numbers of slots) and group
    count gives the oracle's states (ragged N and R; with 2 groups of unequal
    size for 16, 24 and 48)."""
    N, R, T = 300, 70, 2
    W, w_in, _, u = make_system(N, "gauss", seed=11, T=T)
    rng = np.random.default_rng(11)
    cur = rng.uniform(1e-3, 3e-3, R)
    gain = rng.uniform(0.5, 2.0, R)
    P = sto.Params(substeps=3, A_cp=100.0, A_in=30.0)
    st = np.zeros((T, R, N), np.float32)
    with sto.Sweep(W, w_in, P, currents=cur, gains=gain) as sw:
        sw.set_plan(tile_n, slots, groups)
        plan = sw.plan()
        assert (plan["tile_n"], plan["slots"], plan["tuned"], plan["groups"]) == (tile_n, slots, 0, groups)
        assert plan["staged"] in (0, 1)
        assert plan["tiles"] == -(-N // 128) * -(-R // tile_n)
        sw.run(u, st)
    Wb = bf16_round(W).astype(np.float64)
    m0 = np.asarray(oracle.initial_state(N), np.float64)
    for r in (0, 17, 33, 64, 69):
        OP = oracle_params(P.replace(current=float(cur[r]), input_gain=float(gain[r])))
        _, ref = oracle.run(OP, Wb, w_in.astype(np.float64), m0, u.astype(np.float64), nthreads=8)
        assert np.max(np.abs(st[:, r] - ref)) <= 1e-5, r


def test_sweep_several_tiles_per_cta(sto):
    """More tiles than SMs: each CTA finishes several tiles per stage,
    alternating between its two tensor-memory accumulators."""
    N, R, T = 256, 2400, 2
    W, w_in, _, u = make_system(N, "gauss", seed=12, T=T)
    rng = np.random.default_rng(12)
    cur = rng.uniform(1e-3, 3e-3, R)
    P = sto.Params(substeps=2, A_cp=100.0, A_in=30.0)
    st = np.zeros((T, R, N), np.float32)
    with sto.Sweep(W, w_in, P, currents=cur) as sw:
        sw.set_plan(16, 3)
        plan = sw.plan()
        assert plan["tiles"] == 2 * 150 and plan["tiles"] > plan["grid"]
        sw.run(u, st)
    Wb = bf16_round(W).astype(np.float64)
    m0 = np.asarray(oracle.initial_state(N), np.float64)
    for r in (0, 1, 799, 1500, 2399):
        OP = oracle_params(P.replace(current=float(cur[r])))
        _, ref = oracle.run(OP, Wb, w_in.astype(np.float64), m0, u.astype(np.float64), nthreads=8)
        assert np.max(np.abs(st[:, r] - ref)) <= 1e-5, r


def test_sweep_autotuner_and_invalid_plans(sto):
    N, R, T = 500, 130, 1
    W, w_in, _, u = make_system(N, "gauss", seed=13, T=T)
    P = sto.Params(substeps=2)
    with sto.Sweep(W, w_in, P, currents=np.full(64, 2e-3)) as sw:
        with pytest.raises(sto.StoError):
            sw.set_plan(64, 3, 2)  # R = 64 is one tile column: nothing to split into groups
    with sto.Sweep(W, w_in, P, currents=np.full(R, 2e-3)) as sw:
        assert sw.plan()["tile_n"] == 0  # no plan before the first run
        with pytest.raises(sto.StoError):
            sw.set_plan(36, 3)  # not a multiple of 8
        with pytest.raises(sto.StoError):
            sw.set_plan(64, 3, 3)  # at most two reservoir groups
        with pytest.raises(sto.StoError):
            sw.set_plan(64, 9)  # ring deeper than shared memory allows
        with pytest.raises(sto.StoError):
            sw.set_plan(64, 1)  # at least two ring slots
        st = np.zeros((T, R, N), np.float32)
        sw.run(u, st)
        plan = sw.plan()
        assert plan["tuned"] == 1 and plan["candidates"] >= 1 and plan["tuned_us_per_stage"] > 0
        assert plan["tile_n"] % 8 == 0 and plan["grid"] <= torch.cuda.get_device_properties(0).multi_processor_count
        assert plan["groups"] in (1, 2) and plan["threads"] in (512, 1024)
        # the tuner restored the state it ran from: same samples as a forced plan
        ref = np.zeros_like(st)
        with sto.Sweep(W, w_in, P, currents=np.full(R, 2e-3)) as sw2:
            sw2.set_plan(plan["tile_n"], plan["slots"], plan["groups"], plan["staged"], plan["threads"])
            sw2.run(u, ref)
        assert np.array_equal(st, ref)
    with sto.Sweep(W, w_in, P, currents=np.full(R, 2e-3)) as sw:
        with pytest.raises(sto.StoError) as e:
            sw.set_plan(40, 2, 1, 1, threads=1024)  # 64 registers leave no room to load ahead
        assert e.value.code == sto.STO_ENOTSUP
        with pytest.raises(sto.StoError) as e:
            sw.set_plan(40, 2, 1, 0, threads=768)  # 512 or 1024 threads
        assert e.value.code == sto.STO_EINVAL
        with pytest.raises(sto.StoError):
            sw.set_plan(64, 3, 1, 2)  # staging mode outside -1..1
        for staged, threads in ((0, 512), (1, 512), (0, 1024)):
            sw.set_plan(40, 2, 1, staged, threads)
            assert (sw.plan()["staged"], sw.plan()["threads"]) == (staged, threads)


@pytest.mark.parametrize("N,R,tile_n,slots,groups", [(300, 70, 16, 3, 1), (300, 70, 40, 2, 2),
                                                     (2500, 512, 40, 3, 2)])
def test_sweep_threads_and_staging_bitwise_equal(sto, N, R, tile_n, slots, groups):
    """512 threads with the next pair loaded ahead, 512 without, and 1024
    threads run the same per-pair arithmetic on the same products: the
    samples and the end state are the same bits, and they match the oracle."""
    T = 2
    W, w_in, _, u = make_system(N, "gauss", seed=17, T=T)
    rng = np.random.default_rng(17)
    cur = rng.uniform(1e-3, 3e-3, R)
    P = sto.Params(substeps=3, A_cp=100.0, A_in=30.0)
    outs = []
    for staged, threads in ((1, 512), (0, 512), (0, 1024)):
        st = np.zeros((T, R, N), np.float32)
        with sto.Sweep(W, w_in, P, currents=cur) as sw:
            sw.set_plan(tile_n, slots, groups, staged, threads)
            sw.run(u, st)
            outs.append((st, sw.state()))
    for st, m in outs[1:]:
        assert np.array_equal(st, outs[0][0]) and np.array_equal(m, outs[0][1])
    Wb = bf16_round(W).astype(np.float64)
    m0 = np.asarray(oracle.initial_state(N), np.float64)
    for r in (0, R // 2, R - 1):
        OP = oracle_params(P.replace(current=float(cur[r])))
        _, ref = oracle.run(OP, Wb, w_in.astype(np.float64), m0, u.astype(np.float64), nthreads=8)
        assert np.max(np.abs(outs[0][0][:, r] - ref)) <= 1e-5, r


@pytest.mark.parametrize("N,R,tile_n,slots", [(300, 70, 16, 3), (256, 2400, 16, 3), (2500, 512, 40, 3), (2500, 512, 24, 3),
                                              (1000, 65, 32, 4), (2500, 512, 40, 2)])
def test_sweep_two_groups_bitwise_equal_to_one(sto, N, R, tile_n, slots):
    """Two reservoir groups with their own barriers only reorder independent
    work: every tile's product and every pair's update are the same
    arithmetic, so the samples and the final state are the same bits as with
    one grid-wide barrier (including several tiles per CTA per group, and a
    second group with fewer tiles than the first)."""
    T = 2
    W, w_in, _, u = make_system(N, "gauss", seed=N + R, T=T)
    rng = np.random.default_rng(N + R)
    cur = rng.uniform(1e-3, 3e-3, R)
    gain = rng.uniform(0.5, 2.0, R)
    P = sto.Params(substeps=3, A_cp=60.0, A_in=20.0)
    out = []
    for groups in (1, 2):
        st = np.zeros((T, R, N), np.float32)
        with sto.Sweep(W, w_in, P, currents=cur, gains=gain) as sw:
            sw.set_plan(tile_n, slots, groups)
            assert sw.plan()["groups"] == groups
            sw.run(u, st)
            out.append((st, sw.state()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def _own_w_members(sto, Ns, T, seed0=40):
    systems = [make_system(N, "gauss", seed=seed0 + i, T=T) for i, N in enumerate(Ns)]
    params = [sto.Params(substeps=3 + (i % 3), current=1e-3 + 3e-4 * i, A_cp=30.0) for i in range(len(Ns))]
    return systems, params


@pytest.mark.parametrize("lanes", [0, 1, 2, 4])
def test_group_single_launch_matches_separate_runs(sto, lanes):
    """One persistent launch for reservoirs of uneven N and their own W and
    substeps: every member's samples and final state are the bits that
    sto_run gives on the same (re-planned) member handle from the same start,
    over two consecutive calls, whatever the lane count; every member also
    against the oracle."""
    Ns = [100, 333, 1000, 2049, 4000, 150, 777]
    T = 2
    u = make_system(4, "gauss", seed=1, T=2 * T)[3]
    systems, params = _own_w_members(sto, Ns, 2 * T)
    if lanes == 1:  # one lane of 148 CTAs: every member needs N >= 148
        Ns, systems, params = Ns[1:5], systems[1:5], params[1:5]
    grp_res = [sto.Reservoir(W, w_in, P, m0=m0) for (W, w_in, m0, _), P in zip(systems, params)]
    outs = [np.zeros((2 * T, N), np.float32) for N in Ns]
    with sto.Group(grp_res, lanes=lanes) as grp:
        info = grp.info()
        if lanes:
            assert info["lanes"] == lanes
        assert info["lanes"] * info["lane_width"] <= torch.cuda.get_device_properties(0).multi_processor_count
        assert sorted(set(info["lane_of"])) == list(range(info["lanes"]))
        grp.run(u[:T], T, [o[:T] for o in outs])
        grp.run(u[T:], T, [o[T:] for o in outs])
        ends = [r.state() for r in grp_res]
    for (W, w_in, m0, _), P, o, e, r in zip(systems, params, outs, ends, grp_res):
        assert r.info()["grid"] == info["lane_width"]
        ref = np.zeros_like(o)
        r.set_state(m0)
        r.run(u[:T], ref[:T])
        r.run(u[T:], ref[T:])
        assert np.array_equal(r.state(), e)
        assert np.array_equal(o, ref)
        r.close()
        _, orc = oracle.run(oracle_params(P), W.astype(np.float64), w_in.astype(np.float64),
                            m0.astype(np.float64), u.astype(np.float64), nthreads=8)
        assert np.max(np.abs(o - orc)) <= 1e-5


def test_group_device_buffers_and_rejections(sto):
    Ns = [200, 300]
    T = 2
    u = make_system(4, "gauss", seed=2, T=T)[3]
    systems, params = _own_w_members(sto, Ns, T, seed0=60)
    res = [sto.Reservoir(W, w_in, P, m0=m0) for (W, w_in, m0, _), P in zip(systems, params)]
    dev = torch.device("cuda")
    outs = [torch.zeros((T, N), dtype=torch.float32, device=dev) for N in Ns]
    with sto.Group(res) as grp:
        grp.run(torch.from_numpy(u).to(dev), T, outs)
        torch.cuda.synchronize()
        for (W, w_in, m0, _), o, r in zip(systems, outs, res):
            ref = np.zeros((T, W.shape[0]), np.float32)
            r.set_state(m0)
            r.run(u, ref)  # the same member handle, run alone
            assert np.array_equal(o.cpu().numpy(), ref)
        res[1].set_tableau([[0.0, 0.0], [1.0, 0.0]], [0.5, 0.5])  # not classic RK4 any more
        with pytest.raises(sto.StoError) as e:
            grp.run(u, T)
        assert e.value.code == sto.STO_ENOTSUP
    with pytest.raises(sto.StoError) as e:
        sto.Group([res[0], res[0]])
    assert e.value.code == sto.STO_EINVAL
    W64 = systems[0][0].astype(np.float64)
    with sto.Reservoir(W64, systems[0][1], params[0], coupling="df64") as r64:
        with pytest.raises(sto.StoError) as e:
            sto.Group([res[0], r64])
        assert e.value.code == sto.STO_ENOTSUP
    for r in res:
        r.close()


def test_sweep_full_configuration_sampled_reservoirs(sto):
    """The benchmark's sweep: 512 reservoirs sharing one N = 2500 Gaussian W,
    I ~ U[1, 3] mA, g ~ U[0.5, 2], autotuned plan; reservoirs sampled across
    the tile columns against the oracle run with the BF16-rounded W."""
    N, R, T = 2500, 512, 2
    W, w_in, _, u = make_system(N, "gauss", seed=30, T=T)
    rng = np.random.default_rng(30)
    cur = rng.uniform(1e-3, 3e-3, R)
    gain = rng.uniform(0.5, 2.0, R)
    P = sto.Params(substeps=3, A_cp=50.0, A_in=20.0)
    st = np.zeros((T, R, N), np.float32)
    with sto.Sweep(W, w_in, P, currents=cur, gains=gain) as sw:
        sw.run(u, st)
        assert sw.plan()["tuned"] == 1
    Wb = bf16_round(W).astype(np.float64)
    m0 = np.asarray(oracle.initial_state(N), np.float64)
    for r in (0, 79, 80, 255, 256, 400, 511):
        OP = oracle_params(P.replace(current=float(cur[r]), input_gain=float(gain[r])))
        _, ref = oracle.run(OP, Wb, w_in.astype(np.float64), m0, u.astype(np.float64), nthreads=16)
        assert np.max(np.abs(st[:, r] - ref)) <= 1e-5, r


def test_sweep_replan_after_a_run_continues_exactly(sto):
    """A plan set between two calls (other group count and thread count)
    continues from m_n: the samples equal one call under the first plan."""
    N, R, T = 300, 70, 4
    W, w_in, _, u = make_system(N, "gauss", seed=19, T=T)
    cur = np.random.default_rng(19).uniform(1e-3, 3e-3, R)
    P = sto.Params(substeps=3, A_cp=100.0, A_in=30.0)
    s1, s2 = np.zeros((2, R, N), np.float32), np.zeros((2, R, N), np.float32)
    with sto.Sweep(W, w_in, P, currents=cur) as sw:
        sw.set_plan(40, 2, 1, 1, 512)
        sw.run(u[:2], s1)
        sw.set_plan(40, 3, 2, 0, 1024)
        sw.run(u[2:], s2)
    ref = np.zeros((T, R, N), np.float32)
    with sto.Sweep(W, w_in, P, currents=cur) as sw:
        sw.set_plan(40, 2, 1, 1, 512)
        sw.run(u, ref)
    assert np.array_equal(np.concatenate([s1, s2]), ref)


def test_sweep_and_group_in_one_launch_equal_their_own_calls(sto):
    """One cooperative launch (sto_run_sweep_group): the shared-W sweep on the
    SMs the own-W group leaves free, the group's lanes on the others.  Each
    part gives the same bits as its own call (sto_run_batched with the same
    tile width, sto_group_run of a group made for the same CTAs), and the
    oracle's states; the sweep's own plan is left as it was."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    N, R, T = 300, 70, 2
    W, w_in, _, u = make_system(N, "gauss", seed=31, T=T)
    rng = np.random.default_rng(31)
    cur = rng.uniform(1e-3, 3e-3, R)
    gain = rng.uniform(0.5, 2.0, R)
    P = sto.Params(substeps=3, A_cp=100.0, A_in=30.0)
    Ns = [100, 257, 513, 1000, 130]
    systems = [make_system(n, "gauss", seed=40 + i, T=1) for i, n in enumerate(Ns)]

    def make():
        sw = sto.Sweep(W, w_in, P, currents=cur, gains=gain)
        sw.set_plan(40, 2, 2, 1, 512)
        res = [sto.Reservoir(Wi, wi, P, m0=mi) for (Wi, wi, mi, _) in systems]
        grp = sto.Group(res, lanes=2, ctas=sms - 24)
        return sw, res, grp

    sw, res, grp = make()
    plan_before = sw.plan()
    st_sw = np.zeros((T, R, N), np.float32)
    st_g = [np.zeros((T, n), np.float32) for n in Ns]
    sto.run_sweep_group(sw, grp, u, sweep_states=st_sw, group_states=st_g)
    assert sw.plan() == plan_before
    info = grp.info()
    assert info["lanes"] * info["lane_width"] <= sms - 24
    sw2, res2, grp2 = make()
    ref_sw = np.zeros_like(st_sw)
    sw2.run(u, ref_sw)
    ref_g = [np.zeros((T, n), np.float32) for n in Ns]
    grp2.run(u, states_out=ref_g)
    assert np.array_equal(st_sw, ref_sw)
    assert np.array_equal(sw.state(), sw2.state())
    for a, b_, r1, r2 in zip(st_g, ref_g, res, res2):
        assert np.array_equal(a, b_)
        assert np.array_equal(r1.state(), r2.state())
    Wb = bf16_round(W).astype(np.float64)
    m0 = np.asarray(oracle.initial_state(N), np.float64)
    for r in (0, 41, 69):
        OP = oracle_params(P.replace(current=float(cur[r]), input_gain=float(gain[r])))
        _, ref = oracle.run(OP, Wb, w_in.astype(np.float64), m0, u.astype(np.float64), nthreads=8)
        assert np.max(np.abs(st_sw[:, r] - ref)) <= 1e-5, r
    for (Wi, wi, mi, _), st in zip(systems, st_g):
        _, ref = oracle.run(oracle_params(P), Wi.astype(np.float64), wi.astype(np.float64),
                            mi.astype(np.float64), u.astype(np.float64), nthreads=8)
        assert np.max(np.abs(st - ref)) <= 1e-5
    for obj in [grp, grp2, sw, sw2] + res + res2:
        obj.close()


def test_whole_sweep_configuration_in_one_launch(sto):
    """The benchmark's whole sweep in one cooperative launch
    (sto_run_sweep_group, the split it times): 512 reservoirs sharing one
    N = 2500 Gaussian W (I ~ U[1, 3] mA, g ~ U[0.5, 2]) beside 64 reservoirs
    with their own Gaussian W and N ~ U[100, 4000] on 3 lanes of the other
    SMs; sampled reservoirs of both kinds against the oracle (1e-5)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    N, R, T = 2500, 512, 1
    W, w_in, _, u = make_system(N, "gauss", seed=33, T=T)
    rng = np.random.default_rng(33)
    cur = rng.uniform(1e-3, 3e-3, R)
    gain = rng.uniform(0.5, 2.0, R)
    P = sto.Params(substeps=3, A_cp=50.0, A_in=20.0)
    Ns = np.random.default_rng([33, 11]).integers(100, 4001, 64)
    systems = [make_system(int(n), "gauss", seed=500 + i, T=1) for i, n in enumerate(Ns)]
    sw = sto.Sweep(W, w_in, P, currents=cur, gains=gain)
    res = [sto.Reservoir(Wi, wi, P, m0=mi) for (Wi, wi, mi, _) in systems]
    grp = sto.Group(res, lanes=0, ctas=sms - 28)
    st_sw = np.zeros((T, R, N), np.float32)
    st_g = [np.zeros((T, int(n)), np.float32) for n in Ns]
    sto.run_sweep_group(sw, grp, u, sweep_states=st_sw, group_states=st_g)
    Wb = bf16_round(W).astype(np.float64)
    m0 = np.asarray(oracle.initial_state(N), np.float64)
    for r in (0, 255, 511):
        OP = oracle_params(P.replace(current=float(cur[r]), input_gain=float(gain[r])))
        _, ref = oracle.run(OP, Wb, w_in.astype(np.float64), m0, u.astype(np.float64), nthreads=16)
        assert np.max(np.abs(st_sw[:, r] - ref)) <= 1e-5, r
    for i in (0, int(np.argmax(Ns)), int(np.argmin(Ns)), 63):
        Wi, wi, mi, _ = systems[i]
        _, ref = oracle.run(oracle_params(P), Wi.astype(np.float64), wi.astype(np.float64),
                            mi.astype(np.float64), u.astype(np.float64), nthreads=16)
        assert np.max(np.abs(st_g[i] - ref)) <= 1e-5, i
    for obj in [grp, sw] + res:
        obj.close()


def test_sweep_initial_state_from_device_or_host_and_nonfinite(sto):
    """The batch's initial state is formed on the device from m0 ([R][3][N]
    float32): a device m0 gives the same state as the same host m0, the
    default is Eq. (initial) for every oscillator, and a NaN anywhere in m0
    is refused with STO_ENONFINITE."""
    N, R = 130, 7
    W, w_in, _, u = make_system(N, "gauss", seed=41, T=1)
    m0 = np.stack([make_system(N, "gauss", seed=141 + r, T=1)[2] for r in range(R)]).astype(np.float32)
    P = sto.Params(substeps=2)
    with sto.Sweep(W, w_in, P, currents=np.full(R, 2e-3), m0=m0) as a:
        s_host = a.state()
    with sto.Sweep(W, w_in, P, currents=np.full(R, 2e-3), m0=torch.from_numpy(m0).cuda()) as b:
        s_dev = b.state()
    assert np.array_equal(s_host, s_dev)
    assert np.array_equal(s_host, m0.astype(np.float64))
    with sto.Sweep(W, w_in, P, currents=np.full(R, 2e-3)) as c:
        s_ic = c.state()
    ic = np.asarray(oracle.initial_state(N), np.float64)
    for r in range(R):
        assert np.max(np.abs(s_ic[r] - ic)) <= 1e-7
    bad = m0.copy()
    bad[3, 1, 17] = np.nan
    with pytest.raises(sto.StoError) as e:
        sto.Sweep(W, w_in, P, currents=np.full(R, 2e-3), m0=bad)
    assert e.value.code == sto.STO_ENONFINITE
