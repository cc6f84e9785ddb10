"""Benchmark: RK4 stepping of N coupled spin-torque oscillators on one B300.

Workload (default): one reservoir of N = 10^4 oscillators, dense FP32
Gaussian coupling W (std 0.1/sqrt(N), zero diagonal, 400 MB, larger than the
126 MB L2 so it is re-read from HBM every stage), w_in ~ U[-1, 1],
u ~ U[0, 1], random unit initial state, 100 RK4 substeps of 1e-11 s per input
sample, states sampled every input sample; seed 0.  A "step" is one sto_run
call over --ips input samples (one persistent kernel launch).  A second,
smaller workload (N = 10^3, the same structure) is measured beside it.

Metric: node-updates/s = N * RK4 steps / s (one node-update = one oscillator
advanced by one full RK4 step, four stages).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores instead (the
comparison arm; it runs a bounded sample of the same workload per step).
Under torchrun with N > 1 processes every rank runs its own independent
reservoir (replicas, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 126 * 2 ** 20
FALLBACK_HBM_GBS = 6400.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=10000, help="oscillators of the main workload")
    ap.add_argument("--ips", type=int, default=2, help="input samples per step")
    ap.add_argument("--substeps", type=int, default=100)
    ap.add_argument("--n-small", type=int, default=1000)
    ap.add_argument("--ips-small", type=int, default=20)
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--grid", type=int, default=0)
    ap.add_argument("--l2-keep-mb", type=int, default=0)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--sweep-n", type=int, default=2500)
    ap.add_argument("--sweep-r", type=int, default=512)
    ap.add_argument("--sweep-t", type=int, default=2, help="input samples per timed sweep call")
    ap.add_argument("--sweep-plan", default="",
                    help="tile_n,slots[,groups[,staged[,threads]]] of the sweep kernel (default: autotuned)")
    ap.add_argument("--no-group", action="store_true")
    ap.add_argument("--no-fused", action="store_true")
    ap.add_argument("--no-readout", action="store_true")
    ap.add_argument("--no-shard", action="store_true")
    ap.add_argument("--group-r", type=int, default=64)
    ap.add_argument("--group-t", type=int, default=1, help="input samples per timed group call")
    ap.add_argument("--group-lanes", type=int, default=0, help="lanes of the group launch (0 = auto)")
    ap.add_argument("--adj-n", type=int, default=1000)
    ap.add_argument("--adj-t", type=int, default=2000, help="input samples per adjoint call")
    ap.add_argument("--adj-k", type=int, default=100, help="checkpoint interval (samples)")
    ap.add_argument("--adj-reps", type=int, default=1, help="timed adjoint calls")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--fp64-ns", default="1000,10000",
                    help="N of the FP64 replica of the paper's benchmark (comma separated)")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed launches per FP64 case")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seed(rank: int) -> int:
    """Each rank simulates its own independent reservoir (weak scaling)."""
    return rank


def combine_ranks(total_ms, e2e_s, updates, world, all_reduce_max=None):
    """Whole-job throughput over `world` replicas: the slowest rank's time
    (max over ranks of the timed region) and the sum of node-updates."""
    if world > 1:
        total_ms, e2e_s = all_reduce_max([total_ms, e2e_s or 0.0])
        updates *= world
    value = updates / (total_ms / 1e3)
    e2e_value = updates / e2e_s if e2e_s else None
    return value, e2e_value, total_ms, updates


def workload(N, T, seed):
    from paper_2312_01121_b300 import inputs
    W = inputs.coupling_gaussian(N, seed=seed, dtype=np.float32)
    w_in = inputs.f32(inputs.input_weights(N, 1, seed=seed))
    m0 = inputs.f32(inputs.random_unit_states(N, seed=seed))
    u = inputs.f32(inputs.input_series(T, 1, seed=seed))
    return np.ascontiguousarray(W, dtype=np.float32), w_in, m0, u


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def measured_bf16():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return {"bf16": float(d["bf16_tflops"]), "bf16_sustained": float(d["bf16_tflops_sustained"]),
                "source": "measured"}
    except Exception:
        return {"bf16": 1800.0, "bf16_sustained": 1400.0, "source": "fallback"}


# Sources whose change invalidates a recorded DRAM-traffic figure of the
# stepper kernel (device code and the host code that plans its launch).
STEPPER_SOURCES = ("paper_2312_01121_b300/csrc/sto_kernel.cuh", "paper_2312_01121_b300/csrc/dfloat.cuh",
                   "paper_2312_01121_b300/csrc/stepper_plan.h", "paper_2312_01121_b300/csrc/sto.cu",
                   "include/sto.h")
TRAFFIC_FILE = os.path.join("profiles", "dram_traffic.txt")


def stepper_source_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in STEPPER_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(N: int, stages: int):
    """DRAM bytes (read + write) of one stepper launch of `stages` stages at N,
    from the steady per-stage figure an ncu capture recorded, or None when no
    capture of the current kernel sources at this N exists."""
    try:
        digest = stepper_source_digest()
        with open(os.path.join(ROOT, TRAFFIC_FILE)) as fh:
            for line in fh:
                f = line.split()
                if len(f) >= 4 and not f[0].startswith("#") and f[0] == "sto_persistent_kernel" \
                        and int(f[1]) == N and f[2] == digest:
                    return float(f[3]) * stages
    except (OSError, ValueError):
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms; only the
    samples taken between mark_start() and mark_end() are summarised."""
    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.t0 = self.t1 = None
        self.out = ""

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)  # let the sampler start before the timed region
        except Exception:
            self.proc = None
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()
        time.sleep(0.1)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.out = out

    def summary(self):
        import datetime
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if self.t0 is not None and not (self.t0 - 0.05 <= ts <= (self.t1 or ts) + 0.05):
                    continue
                sm.append(float(f[2]))
                mx.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[6:10]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def time_device(N, args, ips, seed, torch, sto, dev):
    """Device-resident timing of K steps; returns a dict of measurements."""
    K, Wm = args.steps, args.warmup
    T_all = (K + Wm) * ips
    W, w_in, m0, u = workload(N, T_all, seed)
    P = sto.Params(substeps=args.substeps)
    stream = torch.cuda.current_stream()
    Wd = torch.from_numpy(W).to(dev)
    res = sto.Reservoir(Wd, torch.from_numpy(w_in).to(dev), P,
                        m0=torch.from_numpy(m0).to(dev), stream=stream, grid=args.grid,
                        l2_keep_mb=args.l2_keep_mb)
    del Wd
    torch.cuda.empty_cache()
    u_d = torch.from_numpy(u).to(dev)
    st_d = torch.empty((ips, N), dtype=torch.float32, device=dev)
    for i in range(Wm):  # the first run also times the exchange-buffer placements (on-chip W)
        res.run(u_d[i * ips:(i + 1) * ips], st_d)
    torch.cuda.synchronize()
    info = res.info()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    rank, world, _ = dist_env()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        clk.mark_start()
        ev[0].record(stream)
        for i in range(K):
            j = Wm + i
            res.run(u_d[j * ips:(j + 1) * ips], st_d)
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        clk.mark_end()
    if world > 1:
        torch.distributed.barrier()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(K)]
    total_ms = ev[0].elapsed_time(ev[K])
    m = res.state()
    finite = bool(np.all(np.isfinite(m)))
    norm_err = float(np.max(np.abs(np.linalg.norm(m, axis=0) - 1.0)))
    out = {"N": N, "ips": ips, "total_ms": total_ms, "per_launch_ms": per, "info": info,
           "clocks": clk.summary(), "finite": finite, "norm_err": norm_err,
           "node_updates": N * ips * args.substeps * K}
    # end-to-end through the C ABI with host buffers (pinned), copies inside
    if not args.no_e2e:
        u_h = torch.from_numpy(u).pin_memory()
        st_h = torch.empty((ips, N), dtype=torch.float32).pin_memory()
        res.set_state(m0)
        for i in range(Wm):
            res.run(u_h[i * ips:(i + 1) * ips], st_h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(K):
            j = Wm + i
            res.run(u_h[j * ips:(j + 1) * ips], st_h)
        torch.cuda.synchronize()
        out["e2e_s"] = time.perf_counter() - t0
        out["h2d_bytes_per_step"] = ips * 1 * 4
        out["d2h_bytes_per_step"] = ips * N * 4 + 16
    res.close()
    return out


def time_adjoint(args, seed, torch, sto, dev):
    """sto_adjoint on the N = 10^3 reservoir (readout-loss gradients): node-updates of
    the differentiated run per second of the whole adjoint call (checkpoint pass,
    recomputation with recording, reverse pass)."""
    N, T, K = args.adj_n, args.adj_t, args.adj_k
    W, w_in, m0, u = workload(N, T, seed)
    P = sto.Params(substeps=args.substeps)
    stream = torch.cuda.current_stream()
    res = sto.Reservoir(torch.from_numpy(W).to(dev), torch.from_numpy(w_in).to(dev), P,
                        m0=torch.from_numpy(m0).to(dev), stream=stream)
    u_d = torch.from_numpy(u).to(dev)
    g = torch.from_numpy(np.random.default_rng(seed).standard_normal((T, N)).astype(np.float32)).to(dev)
    # warm-up on one checkpoint segment: builds W^T, allocates the recording
    # (K samples), times the exchange-buffer placements
    res.adjoint(u_d[:K], g[:K], K)
    reps = max(1, args.adj_reps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        res.set_state(m0)
        res.adjoint(u_d, g, K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    res.close()
    return {"N": N, "input_samples": T, "ckpt_every": K, "ms_per_call": ms,
            "value": N * T * args.substeps / (ms / 1e3), "unit": "node-updates/s",
            "note": "gradients of a loss on the sampled states w.r.t. A_cp, I, w_in, m0; "
                    "one call = checkpoint pass, then per segment the recomputation with recording "
                    "(beside the reverse pass of the segment after it) and the reverse pass"}


def time_sweep(args, seed, torch, sto, dev, peaks):
    """sto_run_batched: R reservoirs sharing one N x N Gaussian W, currents
    I ~ U[1, 3] mA and input gains g ~ U[0.5, 2] (one per reservoir), the same
    u ~ U[0, 1] for all; states of every reservoir sampled every input sample."""
    N, R, T = args.sweep_n, args.sweep_r, args.sweep_t
    W, w_in, _, u = workload(N, T * 4, seed)
    rng = np.random.default_rng([seed, 7])
    cur = rng.uniform(1e-3, 3e-3, R)
    gain = rng.uniform(0.5, 2.0, R)
    m0 = np.ascontiguousarray(np.stack([workload(N, 1, seed + 1000 + r)[2] for r in range(min(R, 8))]
                                       * ((R + 7) // 8))[:R])
    P = sto.Params(substeps=args.substeps)
    sw = sto.Sweep(torch.from_numpy(W).to(dev), torch.from_numpy(w_in).to(dev), P, currents=cur,
                   gains=gain, m0=torch.from_numpy(m0).to(dev), stream=torch.cuda.current_stream())
    if args.sweep_plan:
        sw.set_plan(*(int(x) for x in args.sweep_plan.split(",")))
    u_d = torch.from_numpy(u).to(dev)
    st = torch.empty((T, R, N), dtype=torch.float32, device=dev)
    sw.run(u_d[:T], st)  # warm-up (and the autotuner, unless a plan was given)
    torch.cuda.synchronize()
    reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    for i in range(reps):
        sw.run(u_d[T * (i + 1):T * (i + 2)], st)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    finite = bool(torch.isfinite(st).all().item())
    plan = sw.plan()
    sw.close()
    stages = 4 * args.substeps * T
    us_stage = ms * 1e3 / stages
    Mpad, Kpad = -(-N // 128) * 128, -(-N // 128) * 128  # K is padded to whole ring slots of 2 x 64
    Rpad = -(-R // plan["tile_n"]) * plan["tile_n"]
    alg_flop = 2.0 * N * N * R            # the coupling product W X of one stage
    exe_flop = 2.0 * Mpad * (2 * Kpad) * Rpad  # executed: hi/lo split, padded tiles
    return {"workload": f"{R} reservoirs sharing one N={N} Gaussian W (BF16), I~U[1,3] mA, "
                        f"g~U[0.5,2], u~U[0,1]; {T} input samples x {args.substeps} RK4 steps per call",
            "value": R * N * args.substeps * T / (ms / 1e3), "unit": "node-updates/s",
            "ms_per_call": ms, "us_per_stage": us_stage,
            "coupling_tflops_algorithmic": alg_flop / (us_stage * 1e-6) / 1e12,
            "coupling_tflops_executed": exe_flop / (us_stage * 1e-6) / 1e12,
            "tensor_peak_tflops": peaks.get("bf16"),
            "tensor_peak_tflops_sustained": peaks.get("bf16_sustained"),
            "frac_of_bf16_peak_whole_stage": (exe_flop / (us_stage * 1e-6) / 1e12) / peaks["bf16"]
            if peaks.get("bf16") else None,
            # the per-pair RK4 state (mn, ms, ksum as double-float triples) is read and written
            # every stage: on average 60 B read + 42 B written per pair and stage (stage 0 reads
            # mn only, stage 3 writes mn only), the other roofline of this kernel
            "state_bytes_per_stage": 102.0 * R * N,
            "state_gbs": 102.0 * R * N / (us_stage * 1e-6) / 1e9,
            "frac_of_hbm_state": (102.0 * R * N / (us_stage * 1e-6) / 1e9) / measured_peaks()[0],
            "finite": finite, "plan": plan,
            "launches_per_call": 1}


def time_group(args, seed, torch, sto, dev, hbm_peak):
    """R reservoirs with their own Gaussian W and N ~ U[100, 4000] (the own-W
    half of the sweep), one persistent launch per call of T samples
    (sto_group_run, lanes of CTAs running members side by side); the same
    members as a graph of one launch per member (sto_run_group) beside it."""
    rng = np.random.default_rng([seed, 11])
    Ns = rng.integers(100, 4001, args.group_r)
    T = args.group_t
    u = workload(4, T * 4, seed)[3]
    stream = torch.cuda.current_stream()
    P = sto.Params(substeps=args.substeps)
    res = []
    for i, N in enumerate(Ns):
        W, w_in, m0, _ = workload(int(N), 1, seed + 5000 + i)
        res.append(sto.Reservoir(torch.from_numpy(W).to(dev), torch.from_numpy(w_in).to(dev), P,
                                 m0=torch.from_numpy(m0).to(dev), stream=stream))
    u_d = torch.from_numpy(u).to(dev)
    reps = 2

    def timed(call):
        call(u_d[:T])  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(reps):
            call(u_d[T * (i + 1):T * (i + 2)])
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_graph = timed(lambda uu: sto.sto_run_group(res, uu, T))
    grp = sto.Group(res, lanes=args.group_lanes)
    info = grp.info()
    ms = timed(lambda uu: grp.run(uu, T))
    grp.close()
    for r in res:
        r.close()
    stages = 4 * args.substeps * T
    wbytes = float(np.sum(4.0 * Ns.astype(np.float64) ** 2))
    return {"workload": f"{args.group_r} reservoirs, own Gaussian W each, N~U[100,4000] "
                        f"(sum N^2 * 4 B = {wbytes / 1e9:.2f} GB of W per stage); "
                        f"{T} input sample(s) x {args.substeps} RK4 steps per call",
            "value": float(np.sum(Ns)) * args.substeps * T / (ms / 1e3), "unit": "node-updates/s",
            "ms_per_call": ms, "us_per_stage": ms * 1e3 / stages,
            "w_gbs_algorithmic": wbytes * stages / (ms / 1e3) / 1e9,
            "frac_of_hbm": wbytes * stages / (ms / 1e3) / 1e9 / hbm_peak,
            "launches_per_call": 1, "lanes": info["lanes"], "lane_width": info["lane_width"],
            "graph_of_launches_us_per_stage": ms_graph * 1e3 / stages,
            "note": "one cooperative launch; members on different lanes run side by side"}


def time_fused(args, seed, torch, sto, dev):
    """The whole parameter sweep of the configuration in ONE persistent launch
    per call (sto_run_sweep_group): the 512 shared-W reservoirs (tensor-core
    product) on the SMs the 64 own-W reservoirs' lanes leave free.  The SM
    split is a choice of the caller: a few are timed, the fastest reported."""
    N, R, T = args.sweep_n, args.sweep_r, 1
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    W, w_in, _, u = workload(N, 4, seed)
    rng = np.random.default_rng([seed, 7])
    cur = rng.uniform(1e-3, 3e-3, R)
    gain = rng.uniform(0.5, 2.0, R)
    P = sto.Params(substeps=args.substeps)
    stream = torch.cuda.current_stream()
    sw = sto.Sweep(torch.from_numpy(W).to(dev), torch.from_numpy(w_in).to(dev), P, currents=cur, gains=gain,
                   stream=stream)
    grng = np.random.default_rng([seed, 11])
    Ns = grng.integers(100, 4001, args.group_r)
    res = []
    for i, Ni in enumerate(Ns):
        Wi, wi, mi, _ = workload(int(Ni), 1, seed + 5000 + i)
        res.append(sto.Reservoir(torch.from_numpy(Wi).to(dev), torch.from_numpy(wi).to(dev), P,
                                 m0=torch.from_numpy(mi).to(dev), stream=stream))
    u_d = torch.from_numpy(u).to(dev)
    splits = []
    for sweep_sms in (20, 28, 36, 48):
        try:
            grp = sto.Group(res, lanes=0, ctas=sms - sweep_sms)
        except sto.StoError as e:
            splits.append({"sweep_sms": sweep_sms, "error": str(e)})
            continue
        info = grp.info()
        sto.run_sweep_group(sw, grp, u_d[:T], T)  # warm-up (the sweep's autotuner on the first call)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2
        e0.record(stream)
        for i in range(reps):
            sto.run_sweep_group(sw, grp, u_d[T * (i + 1):T * (i + 2)], T)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        grp.close()
        splits.append({"sweep_sms": sweep_sms, "group_lanes": info["lanes"], "lane_width": info["lane_width"],
                       "ms_per_call": ms, "us_per_stage": ms * 1e3 / (4 * args.substeps * T)})
    plan = sw.plan()
    sw.close()
    for r in res:
        r.close()
    ok = [x for x in splits if "us_per_stage" in x]
    best = min(ok, key=lambda x: x["us_per_stage"]) if ok else None
    out = {"workload": f"{R} reservoirs sharing one N={N} Gaussian W (BF16), I~U[1,3] mA, g~U[0.5,2], plus "
                       f"{args.group_r} reservoirs with their own Gaussian W, N~U[100,4000]; one input sample x "
                       f"{args.substeps} RK4 steps per call, one cooperative launch per call",
           "launches_per_call": 1, "splits": splits, "sweep_plan": plan}
    if best:
        out.update({"us_per_stage": best["us_per_stage"], "ms_per_call": best["ms_per_call"],
                    "value": (R * N + float(np.sum(Ns))) * args.substeps * T / (best["ms_per_call"] / 1e3),
                    "unit": "node-updates/s", "best_split": best})
    return out


def time_shard(args, seed, torch, sto, dev, hbm_peak):
    """The row-sharded path (one row block per GPU, an all-gather of the
    stage values between stages) on this one GPU: a single block holding all
    N = 10^4 rows, one stage launch per RK4 stage, one input sample replayed
    as a CUDA graph.  What a rank's stage costs before any exchange."""
    from paper_2312_01121_b300.shard import ShardedReservoir
    N, S, T = args.n, args.substeps, 2
    W, w_in, m0, u = workload(N, T + 1, seed)
    res = ShardedReservoir(N, sto.Params(substeps=S), W_rows=torch.from_numpy(W).to(dev),
                           w_in_rows=torch.from_numpy(w_in).to(dev), m0_rows=torch.from_numpy(m0).to(dev))
    u_d = torch.from_numpy(u).to(dev)
    res.run(u_d[:1], graph=True)  # capture and warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    res.run(u_d[1:], graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / (4 * S * T)
    return {"workload": f"one row block holding all N={N} rows (world size 1), {T} input samples x {S} RK4 "
                        "steps, each sample one CUDA-graph replay of its 4 S stage launches and exchanges",
            "us_per_stage": us, "value": N * S * T / (us * 4 * S * T / 1e6), "unit": "node-updates/s",
            "w_gbs_algorithmic": 4.0 * N * N / (us * 1e-6) / 1e9,
            "frac_of_hbm": 4.0 * N * N / (us * 1e-6) / 1e9 / hbm_peak}


def time_readout(args, seed, torch, sto, dev):
    """The ridge readout on the GPU (fit on the first half after a washout of
    100, NMSE on the second half) for states of the readout workload's shape:
    10^4 samples x N = 1000 (synthetic FP32 states; the cost does not depend
    on their values).  Set-up work, outside every timed step."""
    T, N = 10000, args.adj_n
    g = torch.Generator(device=dev).manual_seed(seed)
    states = torch.rand((T, N), generator=g, device=dev, dtype=torch.float32) * 2 - 1
    y = torch.rand((T,), generator=g, device=dev, dtype=torch.float64)
    (a, b), (c, d) = sto.readout_split(T, 100)
    stream = torch.cuda.current_stream()
    w = torch.empty(N + 1, dtype=torch.float64, device=dev)
    sto.sto_readout_fit(states, y, a, b, 0.1, w_out=w, stream=stream)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sto.sto_readout_fit(states, y, a, b, 0.1, w_out=w, stream=stream)
    t1 = time.perf_counter()
    sto.sto_readout_nmse(states, w, y, c, d, stream=stream)
    t2 = time.perf_counter()
    return {"N": N, "samples": T, "train": b - a, "fit_ms": (t1 - t0) * 1e3, "nmse_ms": (t2 - t1) * 1e3,
            "note": "FP64 Gram matrix, blocked Cholesky and solves on the GPU; wall time of one call"}


def time_fp64(args, seed, torch, sto, dev, hbm_peak):
    """The paper's own benchmark in its precision (Sec. 3.3, Table 1): FP64
    coupling, u = 0, Eq. (initial) for every oscillator, W of the paper's
    structure (zero diagonal, U[-1, 1], spectral radius ~1 by the circular
    law), dt = 1e-11 s.  One launch = 100 RK4 steps; both products."""
    from paper_2312_01121_b300 import inputs
    out = []
    stream = torch.cuda.current_stream()
    for N in [int(x) for x in args.fp64_ns.split(",") if x]:
        W = inputs.coupling_paper_circular(N, seed=seed)
        w_in = inputs.f32(inputs.input_weights(N, 1, seed=seed))
        Wd = torch.from_numpy(W).to(dev)
        del W
        S, K = args.substeps, args.fp64_steps
        u_d = torch.zeros((1, 1), dtype=torch.float32, device=dev)
        for coupling in ("df64", "f64"):
            res = sto.Reservoir(Wd, torch.from_numpy(w_in).to(dev), sto.Params(substeps=S),
                                stream=stream, coupling=coupling)
            res.run(u_d, None)  # warm-up
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
            ev[0].record(stream)
            for i in range(K):
                res.run(u_d, None)
                ev[i + 1].record(stream)
            torch.cuda.synchronize()
            per = [ev[i].elapsed_time(ev[i + 1]) for i in range(K)]
            m = res.state()
            info = res.info()
            res.close()
            stages = 4 * S
            ms = statistics.mean(per)
            gbs = 8.0 * N * N * stages / (ms / 1e3) / 1e9
            out.append({"N": N, "coupling": coupling, "us_per_stage": ms * 1e3 / stages,
                        "value": N * S / (ms / 1e3), "unit": "node-updates/s",
                        "w_gbs_algorithmic": gbs, "frac_of_hbm": gbs / hbm_peak,
                        "seconds_per_5e3_rk4_steps": ms / 1e3 / S * 5e3,
                        "max_abs_norm_minus_1": float(np.max(np.abs(np.linalg.norm(m, axis=0) - 1.0))),
                        "grid": info["grid"], "resident": info["resident"]})
        del Wd
        torch.cuda.empty_cache()
    return {"workload": "paper benchmark replica (Sec. 3.3, Table 1): FP64 coupling, u=0, "
                        "Eq. (initial), paper-structured W, dt=1e-11 s; one launch = "
                        f"{args.substeps} RK4 steps",
            "products": {"df64": "W as exact FP32 pairs (48-bit), double-float products and sums",
                         "f64": "W in FP64, FP64 fused multiply-adds"},
            "cases": out}


def cpu_oracle_rate(N, substeps_total_budget_s, seed, nthreads, steps=None):
    """Node-updates/s of the FP64 oracle on a bounded sample of the workload
    (steps RK4 steps, or as many as fit the time budget)."""
    import oracle
    W, w_in, m0, u = workload(N, 1, seed)
    W64 = W.astype(np.float64)
    del W
    P = oracle.OracleParams(substeps=1)
    m = m0.astype(np.float64)
    t0 = time.perf_counter()
    m, _ = oracle.run(P, W64, w_in.astype(np.float64), m, u.astype(np.float64), nthreads=nthreads)
    one = time.perf_counter() - t0
    if steps is None:
        steps = max(1, int(substeps_total_budget_s / max(one, 1e-6)))
    t0 = time.perf_counter()
    uu = np.repeat(u.astype(np.float64), steps, axis=0)
    m, _ = oracle.run(P, W64, w_in.astype(np.float64), m, uu, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return {"value": N * steps / dt, "steps": steps, "seconds": dt, "cores": nthreads}


def workload_config(args, world):
    """The workload the line's metric is measured on (both arms)."""
    N, ips, S = args.n, args.ips, args.substeps
    return {
        "workload": f"plain single reservoir, N={N}, dense Gaussian FP32 W (std 0.1/sqrt(N), "
                    f"zero diagonal, {4 * N * N / 1e6:.0f} MB), u~U[0,1], RK4 dt=1e-11 s, "
                    f"{S} substeps per input sample, states sampled every sample",
        "N": N, "input_samples_per_step": ips, "rk4_steps_per_step": ips * S,
        "stages_per_step": 4 * S * ips, "parallelism": "replicas" if world > 1 else "single",
        "l2": f"inputs larger than L2: W ({4 * N * N / 1e6:.0f} MB) > L2 (126 MB), no flush; by design "
              "a 110 MB slice of W stays in L2 across stages and the panel order alternates, the "
              "rest is re-read from HBM every stage",
    }


def reference_arm(args):
    """The FP64 CPU oracle as the comparison arm, on this host's cores."""
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    import oracle
    N = args.n
    nthreads = os.cpu_count() or 1
    W, w_in, m0, u = workload(N, args.steps + args.warmup, 0)
    W64 = W.astype(np.float64)
    del W
    P = oracle.OracleParams(substeps=1)
    m = m0.astype(np.float64)
    w64 = w_in.astype(np.float64)
    u64 = u.astype(np.float64)
    for i in range(args.warmup):
        m, _ = oracle.run(P, W64, w64, m, u64[i:i + 1], nthreads=nthreads)
    t0 = time.perf_counter()
    for i in range(args.steps):
        j = args.warmup + i
        m, _ = oracle.run(P, W64, w64, m, u64[j:j + 1], nthreads=nthreads)
    dt = time.perf_counter() - t0
    value = N * args.steps / dt
    line = {"impl": "reference", "metric": "node-updates/s", "value": value,
            "unit": "node-updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(args, world),
            "cpu_baseline": {"value": value, "unit": "node-updates/s", "cores": nthreads,
                             "kind": "oracle",
                             "sample": f"each step is 1 RK4 step of the same N={N} workload (the "
                                       f"oracle's rate is per node-update, like the GPU arm's); "
                                       f"{args.steps} timed steps"},
            "e2e": {"value": value, "unit": "node-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def summary(line, hbm_peak):
    """The secondary workloads' headline numbers in one short object, printed
    last in the line so that a truncated tail of the output still holds them."""
    n = line["config"]["N"]
    tag = "n1e4" if n == 10000 else f"n{n}"  # the headline workload's size
    out = {f"{tag}_us_per_stage": line["roofline"]["us_per_stage"],
           f"{tag}_frac_hbm_alg": line["roofline"]["frac"],
           f"{tag}_frac_hbm_dram": line["roofline"].get("frac_dram")}
    also = line.get("also")
    if also:
        out.update({"n1e3_node_updates_per_s": also["value"], "n1e3_us_per_stage": also["us_per_stage"],
                    "n1e3_hbm_equiv_us_per_stage": also["hbm_roofline_us_per_stage"]})
    adj = line.get("adjoint")
    if adj:
        out.update({"adjoint_node_updates_per_s": adj["value"], "adjoint_s_per_call": adj["ms_per_call"] / 1e3,
                    "adjoint_config": f"N={adj['N']} T={adj['input_samples']} K={adj['ckpt_every']}"})
    sw = line.get("sweep")
    if sw:
        out.update({"sweep_us_per_stage": sw["us_per_stage"], "sweep_node_updates_per_s": sw["value"],
                    "sweep_frac_bf16_alg": sw["coupling_tflops_algorithmic"] / sw["tensor_peak_tflops"],
                    "sweep_frac_bf16_alg_sustained": sw["coupling_tflops_algorithmic"]
                    / sw["tensor_peak_tflops_sustained"],
                    "sweep_frac_bf16_exec": sw["frac_of_bf16_peak_whole_stage"]})
    grp = line.get("group")
    if grp:
        out.update({"group_us_per_stage": grp["us_per_stage"], "group_frac_hbm": grp["frac_of_hbm"]})
    sh = line.get("shard")
    if sh:
        out["shard_n1e4_us_per_stage"] = sh["us_per_stage"]
    ro = line.get("readout")
    if ro:
        out["readout_fit_ms_n1000_t1e4"] = ro["fit_ms"]
    fu = line.get("sweep_and_group_one_launch")
    if fu and "us_per_stage" in fu:
        out.update({"sweep_and_group_one_launch_us_per_stage": fu["us_per_stage"],
                    "sweep_and_group_separate_us_per_stage": fu.get("separate_launches_us_per_stage")})
    fp = line.get("fp64")
    if fp:
        for c in fp["cases"]:
            if c["N"] == 10000:
                out[f"fp64_{c['coupling']}_n1e4_us_per_stage"] = c["us_per_stage"]
    return out


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2312_01121_b300 import build, sto
    build.build()
    sto.load_library()

    main_r = time_device(args.n, args, args.ips, replica_seed(rank), torch, sto, dev)
    small = None
    if not args.no_small:
        small = time_device(args.n_small, args, args.ips_small, replica_seed(rank), torch, sto, dev)

    def reduce_max(vals):
        t = torch.tensor(vals, device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return [float(x) for x in t]

    adj = None
    if not args.no_adjoint:
        adj = time_adjoint(args, replica_seed(rank), torch, sto, dev)
    sweep = None
    if not args.no_sweep:
        sweep = time_sweep(args, replica_seed(rank), torch, sto, dev, measured_bf16())
    group = None
    if not args.no_group:
        group = time_group(args, replica_seed(rank), torch, sto, dev, measured_peaks()[0])
    shard = None
    if not args.no_shard:
        shard = time_shard(args, replica_seed(rank), torch, sto, dev, measured_peaks()[0])
    readout = None
    if not args.no_readout:
        readout = time_readout(args, replica_seed(rank), torch, sto, dev)
    fused = None
    if not args.no_fused:
        fused = time_fused(args, replica_seed(rank), torch, sto, dev)
    fp64 = None
    if not args.no_fp64:
        fp64 = time_fp64(args, replica_seed(rank), torch, sto, dev, measured_peaks()[0])

    value, e2e_value, tot_ms, updates = combine_ranks(
        main_r["total_ms"], main_r.get("e2e_s"), main_r["node_updates"], world, reduce_max)

    # roofline of the stepper: algorithmic bytes per launch / mean launch time
    N, ips, S = args.n, args.ips, args.substeps
    stages = 4 * S * ips
    alg_bytes = stages * 4.0 * N * N + ips * 4.0 * N
    mean_launch_s = statistics.mean(main_r["per_launch_ms"]) / 1e3
    achieved = alg_bytes / mean_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    traffic = recorded_traffic(N, stages)

    cpu = None
    if rank == 0 and not args.no_cpu:
        try:
            cpu = cpu_oracle_rate(N, args.cpu_seconds, 0, os.cpu_count() or 1)
            # the same oracle on one host thread, a shorter sample
            cpu["single_thread"] = cpu_oracle_rate(N, max(1.0, args.cpu_seconds / 4), 0, 1)
        except Exception as e:  # the baseline is informative, never fatal
            cpu = {"error": str(e)}
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    line = {
        "metric": "node-updates/s",
        "value": value,
        "unit": "node-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tot_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "dtype_detail": "FP32 W and coupling matvec (FP32 accumulate); double-float (two FP32, "
                        "~48-bit) per-oscillator torque and RK4 combine; FP64 state between calls",
        "data": "synthetic",
        "config": workload_config(args, world),
        "plan": main_r["info"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "frac_dram": (traffic / mean_launch_s / 1e9 / peak) if traffic else None,
                     "peak_source": peak_kind,
                     "kernel": "sto_persistent_kernel",
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "mean_launch_ms": mean_launch_s * 1e3,
                     "us_per_stage": mean_launch_s * 1e6 / stages},
        "clocks": main_r["clocks"],
        "gpu_launches": args.steps,
        "check": {"finite": main_r["finite"], "max_abs_norm_minus_1": main_r["norm_err"]},
    }
    if e2e_value:
        line["e2e"] = {"value": e2e_value, "unit": "node-updates/s",
                       "h2d_bytes_per_step": main_r["h2d_bytes_per_step"],
                       "d2h_bytes_per_step": main_r["d2h_bytes_per_step"]}
    if cpu is not None:
        if "value" in cpu:
            line["cpu_baseline"] = {"value": cpu["value"], "unit": "node-updates/s",
                                    "cores": cpu["cores"], "kind": "oracle",
                                    "sample": f"{cpu['steps']} RK4 steps of the same N={N} "
                                              f"workload in {cpu['seconds']:.1f} s "
                                              "(FP64 C oracle, OpenMP over matvec rows)"}
            one = cpu.get("single_thread")
            if one:
                line["cpu_baseline"]["single_thread"] = {
                    "value": one["value"], "cores": 1,
                    "sample": f"{one['steps']} RK4 steps in {one['seconds']:.1f} s"}
        else:
            line["cpu_baseline"] = cpu
    if small is not None:
        Ns, ipss = args.n_small, args.ips_small
        st = 4 * S * ipss
        ml = statistics.mean(small["per_launch_ms"]) / 1e3
        line["also"] = {
            "workload": f"plain single reservoir, N={Ns}, dense Gaussian FP32 W (4 MB, "
                        "on chip: latency-bound)",
            "value": small["node_updates"] / (small["total_ms"] / 1e3),
            "unit": "node-updates/s", "us_per_stage": ml * 1e6 / st,
            "hbm_roofline_us_per_stage": 4.0 * Ns * Ns / (peak * 1e9) * 1e6,
            "plan": small["info"], "clocks": small["clocks"],
            "e2e_value": (small["node_updates"] / small["e2e_s"]) if small.get("e2e_s") else None,
        }
        if not args.no_cpu:
            # the FP64 oracle at this size too, on all host cores (a bounded sample)
            try:
                c3 = cpu_oracle_rate(Ns, 0.0, 0, os.cpu_count() or 1, steps=2000)
                line["also"]["cpu_oracle"] = {"value": c3["value"], "unit": "node-updates/s", "cores": c3["cores"],
                                              "sample": f"{c3['steps']} RK4 steps of the N={Ns} workload "
                                                        f"in {c3['seconds']:.1f} s"}
            except Exception as e:  # informative, never fatal
                line["also"]["cpu_oracle"] = {"error": str(e)}
    if adj is not None:
        line["adjoint"] = adj
    if sweep is not None:
        line["sweep"] = sweep
    if group is not None:
        line["group"] = group
    if readout is not None:
        line["readout"] = readout
    if shard is not None:
        line["shard"] = shard
    if fused is not None:
        if sweep is not None and group is not None:
            fused["separate_launches_us_per_stage"] = sweep["us_per_stage"] + group["us_per_stage"]
        line["sweep_and_group_one_launch"] = fused
    if fp64 is not None:
        line["fp64"] = fp64
    line["summary"] = summary(line, peak)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
