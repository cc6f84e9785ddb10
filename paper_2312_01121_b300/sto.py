"""Thin ctypes binding of libsto (include/sto.h); argument marshalling only.

Every computation runs inside libsto's CUDA kernels.  There is no fallback:
if ``libsto.so`` is missing or no CUDA device is usable, the calls raise.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA);
they are passed to the library as raw pointers.  The Python functions carry
the C names (``sto_create``, ``sto_run`` ...); ``Reservoir`` wraps a handle.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsto.so")

STO_OK, STO_EINVAL, STO_ENOMEM, STO_ECUDA, STO_ETIMEOUT, STO_ENONFINITE, STO_ENOTSUP = (
    0, -1, -2, -3, -4, -5, -6)
STO_ETOOBIG = -7
STO_ESINGULAR = -8
STO_PRODUCT_DF, STO_PRODUCT_F64 = 1, 2
# coupling precision of a Reservoir -> product of sto_create_f64 (None: FP32 sto_create)
COUPLINGS = {"f32": None, "df64": STO_PRODUCT_DF, "f64": STO_PRODUCT_F64}


class StoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libsto error {code}: {msg}")
        self.code = code


class sto_params(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double), ("alpha", ctypes.c_double), ("Ms", ctypes.c_double),
        ("Hk", ctypes.c_double), ("Happl", ctypes.c_double), ("eta", ctypes.c_double),
        ("lambda_", ctypes.c_double), ("current", ctypes.c_double), ("volume", ctypes.c_double),
        ("e_charge", ctypes.c_double), ("hbar", ctypes.c_double), ("p", ctypes.c_double * 3),
        ("A_cp", ctypes.c_double), ("A_in", ctypes.c_double), ("input_gain", ctypes.c_double),
        ("dt", ctypes.c_double), ("substeps", ctypes.c_int32), ("n_in", ctypes.c_int32),
        ("sample_component", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class sto_config(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32), ("timeout_ms", ctypes.c_int32),
                ("l2_keep_mb", ctypes.c_int32), ("tmem_w", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class sto_batch_plan(ctypes.Structure):
    _fields_ = [("tile_n", ctypes.c_int32), ("slots", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("tiles", ctypes.c_int32), ("smem_bytes", ctypes.c_int32), ("tuned", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("tuned_us_per_stage", ctypes.c_float),
                ("staged", ctypes.c_int32), ("groups", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_ if f[0] != "reserved"}


class sto_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("grid", ctypes.c_int32), ("rows_max", ctypes.c_int32),
                ("panel_cols", ctypes.c_int32), ("panels", ctypes.c_int32),
                ("ring_slots", ctypes.c_int32), ("resident", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32), ("sm_count", ctypes.c_int32),
                ("w_bytes", ctypes.c_int64), ("xbuf_timed", ctypes.c_int32), ("xbuf_slot", ctypes.c_int32),
                ("tmem_panels", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class sto_grads(ctypes.Structure):
    _fields_ = [("dA_cp", ctypes.c_double), ("dcurrent", ctypes.c_double),
                ("dw_in", ctypes.c_void_p), ("dm0", ctypes.c_void_p)]


# name -> (restype, argtypes); the exported symbols of include/sto.h
_VP, _I64, _I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
SIGNATURES = {
    "sto_default_params": (None, [ctypes.POINTER(sto_params)]),
    "sto_create": (ctypes.c_int, [_I64, ctypes.POINTER(sto_params), _VP, _VP, _VP, _VP,
                                  ctypes.POINTER(_VP)]),
    "sto_create_ex": (ctypes.c_int, [_I64, ctypes.POINTER(sto_params), _VP, _VP, _VP, _VP,
                                     ctypes.POINTER(sto_config), ctypes.POINTER(_VP)]),
    "sto_create_f64": (ctypes.c_int, [_I64, ctypes.POINTER(sto_params), _VP, _VP, _VP, _VP,
                                      ctypes.POINTER(sto_config), _I32, ctypes.POINTER(_VP)]),
    "sto_set_params": (ctypes.c_int, [_VP, ctypes.POINTER(sto_params)]),
    "sto_set_state": (ctypes.c_int, [_VP, _VP]),
    "sto_get_state": (ctypes.c_int, [_VP, _VP]),
    "sto_set_state_f64": (ctypes.c_int, [_VP, _VP]),
    "sto_get_state_f64": (ctypes.c_int, [_VP, _VP]),
    "sto_run": (ctypes.c_int, [_VP, _VP, _I64, _VP]),
    "sto_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(sto_info)]),
    "sto_destroy": (None, [_VP]),
    "sto_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "sto_abi_version": (ctypes.c_int, []),
    "sto_debug_inject_stall": (ctypes.c_int, [_VP, _I32]),
    "sto_run_noalloc": (ctypes.c_int, [_I64, ctypes.POINTER(sto_params), _VP, _VP, _VP, _VP,
                                       _I64, _VP, _VP]),
    "sto_adjoint": (ctypes.c_int, [_VP, _VP, _I64, _VP, _I32, ctypes.POINTER(sto_grads)]),
    "sto_set_input_weights": (ctypes.c_int, [_VP, _VP]),
    "sto_batch_create": (ctypes.c_int, [_I64, _I32, ctypes.POINTER(sto_params), _VP, _VP, _VP,
                                        _VP, _VP, _VP, ctypes.POINTER(_VP)]),
    "sto_run_batched": (ctypes.c_int, [_VP, _VP, _I64, _VP]),
    "sto_batch_get_state": (ctypes.c_int, [_VP, _VP]),
    "sto_batch_destroy": (None, [_VP]),
    "sto_batch_set_plan": (ctypes.c_int, [_VP, _I32, _I32]),
    "sto_batch_set_plan_ex": (ctypes.c_int, [_VP, _I32, _I32, _I32]),
    "sto_batch_set_plan_staged": (ctypes.c_int, [_VP, _I32, _I32, _I32, _I32]),
    "sto_batch_set_plan_threads": (ctypes.c_int, [_VP, _I32, _I32, _I32, _I32, _I32]),
    "sto_batch_get_plan": (ctypes.c_int, [_VP, ctypes.POINTER(sto_batch_plan)]),
    "sto_run_group": (ctypes.c_int, [ctypes.POINTER(_VP), _I32, _VP, _I64, ctypes.POINTER(_VP)]),
    "sto_set_tableau": (ctypes.c_int, [_VP, _I32, _VP, _VP]),
    "sto_group_create": (ctypes.c_int, [ctypes.POINTER(_VP), _I32, _I32, ctypes.POINTER(_VP)]),
    "sto_group_create_ex": (ctypes.c_int, [ctypes.POINTER(_VP), _I32, _I32, _I32, ctypes.POINTER(_VP)]),
    "sto_run_sweep_group": (ctypes.c_int, [_VP, _VP, _VP, _I64, _VP, ctypes.POINTER(_VP)]),
    "sto_group_run": (ctypes.c_int, [_VP, _VP, _I64, ctypes.POINTER(_VP)]),
    "sto_group_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "sto_group_destroy": (None, [_VP]),
    "sto_readout_fit": (ctypes.c_int, [_VP, _I64, _I64, _VP, _I64, _I64, ctypes.c_double, _VP, _VP]),
    "sto_readout_predict": (ctypes.c_int, [_VP, _I64, _I64, _VP, _VP, _VP]),
    "sto_readout_nmse": (ctypes.c_int, [_VP, _I64, _I64, _VP, _VP, _I64, _I64,
                                        ctypes.POINTER(ctypes.c_double), _VP]),
    "sto_shard_create": (ctypes.c_int, [_I64, _I64, _I64, ctypes.POINTER(sto_params), _VP, _VP, _VP, _VP,
                                        ctypes.POINTER(_VP)]),
    "sto_shard_publish": (ctypes.c_int, [_VP, _VP]),
    "sto_shard_stage": (ctypes.c_int, [_VP, _VP, _I32, _VP, _I32, _VP, _VP]),
    "sto_shard_set_state_f64": (ctypes.c_int, [_VP, _VP]),
    "sto_shard_get_state_f64": (ctypes.c_int, [_VP, _VP]),
    "sto_shard_destroy": (None, [_VP]),
}

_lib = None


def load_library(path: str | None = None):
    """Load libsto.so (built in-tree by paper_2312_01121_b300.build)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libsto.so not built ({p}); run __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(rc: int):
    if rc != STO_OK:
        raise StoError(rc, load_library().sto_strerror(rc).decode())


@dataclasses.dataclass
class Params:
    """Python mirror of sto_params; defaults = Table "Summary of parameters"."""
    gamma: float = 1.764e7
    alpha: float = 0.005
    Ms: float = 1448.3
    Hk: float = 18616.0
    Happl: float = 200.0
    eta: float = 0.537
    lambda_: float = 0.288
    current: float = 2.5e-3
    volume: float = math.pi * 60.0 ** 2 * 2.0 * 1e-21
    e_charge: float = 1.60217733e-19
    hbar: float = 1.05457266e-34
    p: tuple = (1.0, 0.0, 6.123234e-17)
    A_cp: float = 1.0
    A_in: float = 1.0
    input_gain: float = 1.0
    dt: float = 1e-11
    substeps: int = 100
    n_in: int = 1
    sample_component: int = 0

    def replace(self, **kw) -> "Params":
        return dataclasses.replace(self, **kw)

    def to_c(self) -> sto_params:
        c = sto_params()
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            if f.name == "p":
                c.p = (ctypes.c_double * 3)(*[float(x) for x in v])
            else:
                setattr(c, f.name, v)
        c.reserved = 0
        return c


def sto_default_params() -> Params:
    c = sto_params()
    load_library().sto_default_params(ctypes.byref(c))
    kw = {f[0]: getattr(c, f[0]) for f in sto_params._fields_ if f[0] not in ("p", "reserved")}
    return Params(p=tuple(c.p), **kw)


def _ptr(a, dtype):
    """(pointer, keepalive) for a numpy array or torch tensor of `dtype`."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch
        want = {np.float32: torch.float32, np.float64: torch.float64}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return a.data_ptr(), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, arr


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def sto_create(N, params: Params, W, w_in, m0=None, stream=None, grid=0, timeout_ms=0,
               l2_keep_mb=0, tmem_w=0):
    """Returns an opaque handle (int).  W, w_in, m0: numpy or torch float32."""
    lib = load_library()
    pW, kW = _ptr(W, np.float32)
    pwin, kwin = _ptr(w_in, np.float32)
    pm0, km0 = _ptr(m0, np.float32)
    h = _VP()
    cp = params.to_c()
    if grid or timeout_ms or l2_keep_mb or tmem_w:
        cfg = sto_config(grid=grid, timeout_ms=timeout_ms, l2_keep_mb=l2_keep_mb, tmem_w=tmem_w)
        rc = lib.sto_create_ex(N, ctypes.byref(cp), pW, pwin, pm0, _stream_ptr(stream),
                               ctypes.byref(cfg), ctypes.byref(h))
    else:
        rc = lib.sto_create(N, ctypes.byref(cp), pW, pwin, pm0, _stream_ptr(stream),
                            ctypes.byref(h))
    _check(rc)
    del kW, kwin, km0
    return h.value


def sto_create_f64(N, params: Params, W, w_in, m0=None, stream=None, product=STO_PRODUCT_DF,
                   grid=0, timeout_ms=0, l2_keep_mb=0):
    """Handle with an FP64 coupling (the paper's benchmark precision).  W and
    m0: float64 (numpy or torch); w_in: float32.  product: STO_PRODUCT_DF
    (double-float on the FP32 pipes) or STO_PRODUCT_F64 (FP64 FMA)."""
    lib = load_library()
    pW, kW = _ptr(W, np.float64)
    pwin, kwin = _ptr(w_in, np.float32)
    pm0, km0 = _ptr(m0, np.float64)
    h = _VP()
    cp = params.to_c()
    cfg = sto_config(grid=grid, timeout_ms=timeout_ms, l2_keep_mb=l2_keep_mb)
    _check(lib.sto_create_f64(N, ctypes.byref(cp), pW, pwin, pm0, _stream_ptr(stream),
                              ctypes.byref(cfg), int(product), ctypes.byref(h)))
    del kW, kwin, km0
    return h.value


def sto_run(h, u, T, states_out=None):
    pu, ku = _ptr(u, np.float32)
    if states_out is not None and not hasattr(states_out, "data_ptr"):
        if not (isinstance(states_out, np.ndarray) and states_out.dtype == np.float32
                and states_out.flags.c_contiguous):
            raise TypeError("states_out must be a contiguous float32 array")
    ps, ks = _ptr(states_out, np.float32)
    _check(load_library().sto_run(h, pu, T, ps))


def sto_set_params(h, params: Params):
    cp = params.to_c()
    _check(load_library().sto_set_params(h, ctypes.byref(cp)))


def sto_set_state(h, m):
    p, k = _ptr(m, np.float32)
    _check(load_library().sto_set_state(h, p))


def sto_get_state(h, out):
    p, k = _ptr(out, np.float32)
    _check(load_library().sto_get_state(h, p))


def sto_set_state_f64(h, m):
    p, k = _ptr(m, np.float64)
    _check(load_library().sto_set_state_f64(h, p))


def sto_get_state_f64(h, out):
    p, k = _ptr(out, np.float64)
    _check(load_library().sto_get_state_f64(h, p))


def sto_adjoint(h, u, T, dL_dstates, ckpt_every=100, dw_in=None, dm0=None) -> dict:
    """Gradients of sum(dL_dstates * states) of the run from the current state
    (see include/sto.h).  dw_in (N x n_in) and dm0 (3 x N) are optional float64
    outputs (numpy or torch).  Returns {"A_cp", "current"} (and fills the rest)."""
    pu, ku = _ptr(u, np.float32)
    pg, kg = _ptr(dL_dstates, np.float32)
    pw, kw = _ptr(dw_in, np.float64) if dw_in is not None else (None, None)
    pm, km = _ptr(dm0, np.float64) if dm0 is not None else (None, None)
    if dw_in is not None and not hasattr(dw_in, "data_ptr") and kw is not dw_in:
        raise TypeError("dw_in must be a contiguous float64 array")
    if dm0 is not None and not hasattr(dm0, "data_ptr") and km is not dm0:
        raise TypeError("dm0 must be a contiguous float64 array")
    g = sto_grads(0.0, 0.0, pw, pm)
    _check(load_library().sto_adjoint(h, pu, T, pg, int(ckpt_every), ctypes.byref(g)))
    return {"A_cp": g.dA_cp, "current": g.dcurrent}


def sto_set_input_weights(h, w_in):
    p, k = _ptr(w_in, np.float32)
    _check(load_library().sto_set_input_weights(h, p))


def sto_run_group(reservoirs, u, T=None, states_out=None):
    """Advance several Reservoir objects (own W, uneven N) over the same u in
    one graph-captured sequence of persistent launches."""
    n = len(reservoirs)
    if T is None:
        T = int(u.shape[0])
    hs = (_VP * n)(*[r.handle for r in reservoirs])
    pu, ku = _ptr(u, np.float32)
    keep = []
    outs = None
    if states_out is not None:
        ptrs = []
        for so in states_out:
            p, k = _ptr(so, np.float32)
            ptrs.append(p)
            keep.append(k)
        outs = (_VP * n)(*ptrs)
    _check(load_library().sto_run_group(hs, n, pu, T, outs))


class Group:
    """Reservoirs with their own W advanced by one persistent launch per call
    (lanes of CTAs run members side by side; see sto_group_create)."""

    def __init__(self, reservoirs, lanes: int = 0, ctas: int = 0):
        """ctas: CTAs the lanes occupy (0 = one per SM); fewer leave SMs to a
        sweep run beside the group by run_sweep_group."""
        self.reservoirs = list(reservoirs)  # keeps the handles alive
        n = len(self.reservoirs)
        hs = (_VP * n)(*[r.handle for r in self.reservoirs])
        g = _VP()
        _check(load_library().sto_group_create_ex(hs, n, int(lanes), int(ctas), ctypes.byref(g)))
        self.handle = g.value

    def run(self, u, T=None, states_out=None):
        if T is None:
            T = int(u.shape[0])
        n = len(self.reservoirs)
        pu, ku = _ptr(u, np.float32)
        keep = []
        outs = None
        if states_out is not None:
            ptrs = []
            for so in states_out:
                p, k = _ptr(so, np.float32)
                ptrs.append(p)
                keep.append(k)
            outs = (_VP * n)(*ptrs)
        _check(load_library().sto_group_run(self.handle, pu, T, outs))

    def info(self) -> dict:
        n = len(self.reservoirs)
        lanes, width = ctypes.c_int32(), ctypes.c_int32()
        lane_of = (ctypes.c_int32 * n)()
        _check(load_library().sto_group_get_info(self.handle, ctypes.byref(lanes), ctypes.byref(width), lane_of))
        return {"lanes": lanes.value, "lane_width": width.value, "lane_of": list(lane_of)}

    def close(self):
        if self.handle:
            load_library().sto_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_sweep_group(sweep, group, u, T=None, sweep_states=None, group_states=None):
    """A Sweep (shared W) and a Group (own W) advanced over the same input
    series by one persistent launch (sto_run_sweep_group)."""
    if T is None:
        T = int(u.shape[0])
    n = len(group.reservoirs)
    pu, ku = _ptr(u, np.float32)
    ps, ks = _ptr(sweep_states, np.float32)
    keep, outs = [], None
    if group_states is not None:
        ptrs = []
        for so in group_states:
            p, k = _ptr(so, np.float32)
            ptrs.append(p)
            keep.append(k)
        outs = (_VP * n)(*ptrs)
    _check(load_library().sto_run_sweep_group(sweep.handle, group.handle, pu, int(T), ps, outs))


def sto_get_info(h) -> dict:
    info = sto_info()
    _check(load_library().sto_get_info(h, ctypes.byref(info)))
    return info.as_dict()


def sto_destroy(h):
    if h:
        load_library().sto_destroy(h)


def sto_debug_inject_stall(h, cta: int):
    _check(load_library().sto_debug_inject_stall(h, cta))


def sto_run_noalloc(N, params: Params, W, w_in, state, u, T, states_out=None, stream=None):
    """Allocation-free stepping for callers that must not allocate device
    memory (pool-owned devices, capture-free real-time loops, plug-ins).
    All arrays are caller-owned CUDA tensors: W (N x N float32), w_in, state
    (3 x N float64, advanced in place), u, states_out (or None)."""
    # the library reads and writes these arrays in place and cannot see their
    # extents: check them here, before any kernel touches them
    N, T = int(N), int(T)
    sizes = {"W": (W, N * N, N * N), "w_in": (w_in, N * params.n_in, N * params.n_in),
             "state": (state, 3 * N, 3 * N), "u": (u, T * params.n_in, None)}
    if states_out is not None:
        sizes["states_out"] = (states_out, T * N, None)
    for name, (a, need, exact) in sizes.items():
        n = int(np.prod(a.shape))
        if n < need or (exact is not None and n != exact):
            raise ValueError(f"{name} holds {n} values; sto_run_noalloc(N={N}, T={T}, "
                             f"n_in={params.n_in}) needs {'exactly ' if exact is not None else ''}{need}")
    cp = params.to_c()
    pW, kW = _ptr(W, np.float32)
    pwin, kwin = _ptr(w_in, np.float32)
    pst, kst = _ptr(state, np.float64)
    pu, ku = _ptr(u, np.float32)
    pso, kso = _ptr(states_out, np.float32)
    _check(load_library().sto_run_noalloc(N, ctypes.byref(cp), pW, pwin, pst, pu, T, pso,
                                          _stream_ptr(stream)))


def _states_2d(states):
    if len(states.shape) != 2:
        raise ValueError("states must be T x N")
    return int(states.shape[0]), int(states.shape[1])


def _out_f64(out, n):
    """(pointer, keepalive, array) of a float64 output of n elements: a given
    contiguous float64 numpy array or torch tensor, or a new numpy array."""
    if out is None:
        out = np.empty(n, dtype=np.float64)
    if hasattr(out, "data_ptr"):
        p, k = _ptr(out, np.float64)
    elif isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous:
        p, k = out.ctypes.data, out
    else:
        raise TypeError("outputs must be contiguous float64 arrays")
    if int(np.prod(out.shape)) != n:
        raise ValueError(f"output must hold {n} values")
    return p, k, out


def sto_readout_fit(states, y, t0, t1, beta_rel=1e-6, w_out=None, stream=None):
    """Ridge readout with bias fitted on rows [t0, t1) of states (T x N float32)
    against y (T float64); returns the N + 1 weights (bias last) in w_out
    (numpy or torch float64, host or device; a new numpy array if None)."""
    T, N = _states_2d(states)
    if int(np.prod(y.shape)) != T:
        raise ValueError("y must hold one target per state row")
    ps, ks = _ptr(states, np.float32)
    py, ky = _ptr(y, np.float64)
    pw, kw, w = _out_f64(w_out, N + 1)
    _check(load_library().sto_readout_fit(ps, T, N, py, int(t0), int(t1), float(beta_rel), pw,
                                          _stream_ptr(stream)))
    return w


def sto_readout_predict(states, w, y_hat=None, stream=None):
    """y_hat[t] = states[t] . w[:N] + w[N] in FP64 (a new numpy array if y_hat is None)."""
    T, N = _states_2d(states)
    if int(np.prod(w.shape)) != N + 1:
        raise ValueError("w must hold N + 1 weights")
    ps, ks = _ptr(states, np.float32)
    pw, kw = _ptr(w, np.float64)
    po, ko, out = _out_f64(y_hat, T)
    _check(load_library().sto_readout_predict(ps, T, N, pw, po, _stream_ptr(stream)))
    return out


def sto_readout_nmse(states, w, y, t0, t1, stream=None) -> float:
    """mean((y_hat - y)^2) / var(y) over rows [t0, t1)."""
    T, N = _states_2d(states)
    if int(np.prod(w.shape)) != N + 1 or int(np.prod(y.shape)) != T:
        raise ValueError("w must hold N + 1 weights and y one target per state row")
    ps, ks = _ptr(states, np.float32)
    pw, kw = _ptr(w, np.float64)
    py, ky = _ptr(y, np.float64)
    out = ctypes.c_double()
    _check(load_library().sto_readout_nmse(ps, T, N, pw, py, int(t0), int(t1), ctypes.byref(out),
                                           _stream_ptr(stream)))
    return out.value


def delay_target(u, delay: int = 5) -> np.ndarray:
    """The recall target y_t = u_{t - delay} of the first input channel (0 for
    t < delay), as float64 on the host: an index shift of the input series."""
    if hasattr(u, "detach"):
        u = u.detach().cpu().numpy()
    u = np.asarray(u, dtype=np.float64).reshape(len(u), -1)[:, 0]
    y = np.zeros_like(u)
    if delay > 0:
        y[delay:] = u[:-delay]
    else:
        y[:] = u
    return y


def readout_split(T: int, washout: int):
    """(train, test) sample ranges after the washout: the first half of the
    remaining samples trains the readout, the second half scores it."""
    n = T - washout
    if n < 4:
        raise ValueError("too few samples after the washout")
    half = washout + n // 2
    return (washout, half), (half, T)


def readout_evaluate(states, y, washout: int = 100, beta_rel: float = 1e-6, stream=None):
    """Fit on the first half after the washout, score on the second half:
    returns (w, nmse_test)."""
    (a, b), (c, d) = readout_split(int(states.shape[0]), washout)
    w = sto_readout_fit(states, y, a, b, beta_rel, stream=stream)
    return w, sto_readout_nmse(states, w, y, c, d, stream=stream)


def sto_strerror(code: int) -> str:
    return load_library().sto_strerror(code).decode()


class Reservoir:
    """One reservoir of N coupled STOs on the current CUDA device.

    coupling: "f32" (FP32 W and products, W and m0 float32), or the FP64
    coupling of the paper's benchmark, "df64" (double-float products) or
    "f64" (FP64 FMA), with W and m0 float64.  tmem_w: -1 streams every panel
    of a streamed FP32 W instead of keeping a few in tensor memory
    (sto_config.tmem_w; same bits)."""

    def __init__(self, W, w_in, params: Params | None = None, m0=None, stream=None,
                 grid: int = 0, timeout_ms: int = 0, l2_keep_mb: int = 0, coupling: str = "f32",
                 tmem_w: int = 0):
        self.params = params or Params()
        self.N = int(W.shape[0])
        self.handle = None
        if coupling not in COUPLINGS:
            raise ValueError(f"coupling must be one of {sorted(COUPLINGS)}")
        self.coupling = coupling
        if COUPLINGS[coupling] is None:
            self.handle = sto_create(self.N, self.params, W, w_in, m0, stream, grid, timeout_ms,
                                     l2_keep_mb, tmem_w)
        else:
            self.handle = sto_create_f64(self.N, self.params, W, w_in, m0, stream, COUPLINGS[coupling],
                                         grid, timeout_ms, l2_keep_mb)

    def run(self, u, states_out=None, T=None):
        """Advance over T = len(u) input samples; fills states_out (T x N) if given."""
        if T is None:
            T = int(u.shape[0])
        sto_run(self.handle, u, T, states_out)
        return states_out

    def adjoint(self, u, dL_dstates, ckpt_every=100, T=None, want_w_in=True, want_m0=True):
        """Gradients of sum(dL_dstates * states) for the run from the current
        state; the state advances as in run().  Returns a dict with A_cp,
        current, and (numpy float64) w_in (N x n_in) and m0 (3 x N)."""
        if T is None:
            T = int(u.shape[0])
        dw = np.zeros((self.N, self.params.n_in)) if want_w_in else None
        dm = np.zeros((3, self.N)) if want_m0 else None
        g = sto_adjoint(self.handle, u, T, dL_dstates, ckpt_every, dw, dm)
        if want_w_in:
            g["w_in"] = dw
        if want_m0:
            g["m0"] = dm
        return g

    def set_tableau(self, a=None, b=None):
        """Explicit Runge-Kutta tableau (a: s x s strictly lower, b: s); None = RK4."""
        if b is None:
            _check(load_library().sto_set_tableau(self.handle, 0, None, None))
            return
        A = np.ascontiguousarray(a, dtype=np.float64)
        B = np.ascontiguousarray(b, dtype=np.float64)
        _check(load_library().sto_set_tableau(self.handle, len(B), A.ctypes.data, B.ctypes.data))

    def set_input_weights(self, w_in):
        sto_set_input_weights(self.handle, w_in)

    def set_params(self, params: Params):
        sto_set_params(self.handle, params)
        self.params = params

    def state(self) -> np.ndarray:
        out = np.empty((3, self.N), dtype=np.float64)
        sto_get_state_f64(self.handle, out)
        return out

    def set_state(self, m):
        m = np.asarray(m)
        if m.dtype == np.float64:
            sto_set_state_f64(self.handle, np.ascontiguousarray(m))
        else:
            sto_set_state(self.handle, m)

    def info(self) -> dict:
        return sto_get_info(self.handle)

    def close(self):
        if self.handle:
            sto_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Sweep:
    """R reservoirs sharing W (rounded to BF16), with per-reservoir current and
    input gain, advanced together (tensor-core coupling product per stage)."""

    def __init__(self, W, w_in, params: Params, currents=None, gains=None, m0=None, stream=None):
        lib = load_library()
        self.N = int(W.shape[0])
        self.params = params
        self.R = int(len(currents)) if currents is not None else int(len(gains))
        cur = np.ascontiguousarray(currents, dtype=np.float64) if currents is not None else None
        gn = np.ascontiguousarray(gains, dtype=np.float64) if gains is not None else None
        pW, kW = _ptr(W, np.float32)
        pwin, kwin = _ptr(w_in, np.float32)
        pm0, km0 = _ptr(m0, np.float32)
        h = _VP()
        cp = params.to_c()
        _check(lib.sto_batch_create(self.N, self.R, ctypes.byref(cp),
                                    cur.ctypes.data if cur is not None else None,
                                    gn.ctypes.data if gn is not None else None,
                                    pW, pwin, pm0, _stream_ptr(stream), ctypes.byref(h)))
        self.handle = h.value

    def run(self, u, states_out=None, T=None):
        """states_out: T x R x N float32 (numpy or torch) or None."""
        if T is None:
            T = int(u.shape[0])
        pu, ku = _ptr(u, np.float32)
        ps, ks = _ptr(states_out, np.float32)
        _check(load_library().sto_run_batched(self.handle, pu, T, ps))
        return states_out

    def state(self) -> np.ndarray:
        out = np.empty((self.R, 3, self.N), dtype=np.float64)
        _check(load_library().sto_batch_get_state(self.handle, out.ctypes.data))
        return out

    def set_plan(self, tile_n: int = 0, slots: int = 0, groups: int = 1, staged: int = -1, threads: int = 512):
        """Force a tile width / ring depth / reservoir-group count, staging
        mode (1, 0, or -1 = choose) and threads per CTA (512 or 1024), or
        (0, 0) to run the autotuner."""
        _check(load_library().sto_batch_set_plan_threads(self.handle, int(tile_n), int(slots), int(groups),
                                                         int(staged), int(threads)))

    def plan(self) -> dict:
        p = sto_batch_plan()
        _check(load_library().sto_batch_get_plan(self.handle, ctypes.byref(p)))
        return p.as_dict()

    def close(self):
        if self.handle:
            load_library().sto_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
