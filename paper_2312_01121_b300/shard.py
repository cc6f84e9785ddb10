"""One reservoir split across GPUs by rows, one process per GPU.

The coupling of Eq. (coup) is the matrix-vector product W m^x (Sec. 3.3).
Rank r holds a contiguous block of rows of W and advances exactly those
oscillators (``sto_shard_*`` in include/sto.h); between RK4 stages the ranks
all-gather the N stage values m^x (``torch.distributed``: NCCL between GPUs,
gloo between host processes).  Every stage is one kernel launch per rank;
the collective is the only exchange.

``partition`` cuts N oscillators into ``world`` blocks of ``ceil(N / world)``
rows (the last one shorter), so the all-gather moves equal chunks;
``ShardedReservoir`` runs one rank's block over an input series.  The
per-block compute is pluggable (``block``): the library's CUDA shard by
default; tests substitute a host implementation to exercise the partition
and exchange logic on CPU ranks.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import sto as _sto

SAMPLE_START, SAMPLE_END = 1, 2


def partition(N: int, world: int):
    """[(row0, rows)] of each rank: blocks of ceil(N / world) rows in rank order."""
    if world < 1 or N < world:
        raise ValueError("need 1 <= world <= N")
    chunk = -(-N // world)
    out = []
    for r in range(world):
        a = min(N, r * chunk)
        out.append((a, min(N, a + chunk) - a))
    if any(rows < 1 for _, rows in out):
        raise ValueError(f"N = {N} leaves a rank without rows at world = {world}")
    return out


class CudaBlock:
    """The library's row block (sto_shard_*) on the current CUDA device."""

    dtype = "float32"

    def __init__(self, N, row0, rows, params, W_rows, w_in_rows, m0_rows=None, stream=None):
        import torch
        lib = _sto.load_library()
        # the block's launches and the exchange's copies share one stream
        stream = stream if stream is not None else torch.cuda.current_stream()
        self.stream = stream
        self.N, self.row0, self.rows, self.params = int(N), int(row0), int(rows), params
        self.stream = stream
        pW, kW = _sto._ptr(W_rows, np.float32)
        pwin, kwin = _sto._ptr(w_in_rows, np.float32)
        pm0, km0 = _sto._ptr(m0_rows, np.float32)
        if int(np.prod(W_rows.shape)) != self.rows * self.N:
            raise ValueError("W_rows must be rows x N")
        if int(np.prod(w_in_rows.shape)) != self.rows * params.n_in:
            raise ValueError("w_in_rows must be rows x n_in")
        if m0_rows is not None and int(np.prod(m0_rows.shape)) != 3 * self.rows:
            raise ValueError("m0_rows must be 3 x rows")
        h = _sto._VP()
        cp = params.to_c()
        _sto._check(lib.sto_shard_create(self.N, self.row0, self.rows, ctypes.byref(cp), pW, pwin, pm0,
                                         _sto._stream_ptr(stream), ctypes.byref(h)))
        self.handle = h.value

    def publish(self, x_rows):
        _sto._check(_sto.load_library().sto_shard_publish(self.handle, x_rows.data_ptr()))

    def stage(self, x, st, u_t, flags, x_next, states_row):
        _sto._check(_sto.load_library().sto_shard_stage(
            self.handle, x.data_ptr(), int(st), u_t.data_ptr() if u_t is not None else None, int(flags),
            x_next.data_ptr(), states_row.data_ptr() if states_row is not None else None))

    def state(self) -> np.ndarray:
        out = np.empty((3, self.rows), dtype=np.float64)
        _sto._check(_sto.load_library().sto_shard_get_state_f64(self.handle, out.ctypes.data))
        return out

    def set_state(self, m):
        m = np.ascontiguousarray(m, dtype=np.float64)
        if m.size != 3 * self.rows:
            raise ValueError("state must be 3 x rows")
        _sto._check(_sto.load_library().sto_shard_set_state_f64(self.handle, m.ctypes.data))

    def close(self):
        if getattr(self, "handle", None):
            _sto.load_library().sto_shard_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ShardedReservoir:
    """Rank `rank`'s block of an N-oscillator reservoir split over `world`
    ranks of a torch.distributed process group (or a single rank).

    block: an object with publish / stage / state (CudaBlock by default,
    built from W_rows, w_in_rows, m0_rows on the current CUDA device)."""

    def __init__(self, N, params, W_rows=None, w_in_rows=None, m0_rows=None, group=None, block=None,
                 device=None, stream=None):
        import torch
        import torch.distributed as dist
        self.N, self.params, self.group = int(N), params, group
        dist_on = dist.is_available() and dist.is_initialized()
        self.world = dist.get_world_size(group) if dist_on else 1
        self.rank = dist.get_rank(group) if dist_on else 0
        self.row0, self.rows = partition(self.N, self.world)[self.rank]
        self.chunk = -(-self.N // self.world)
        if block is None:
            # a stream of its own: the stage launches and the exchange are
            # ordered on it, and run(graph=True) captures both from it
            stream = stream if stream is not None else torch.cuda.Stream()
            block = CudaBlock(self.N, self.row0, self.rows, params, W_rows, w_in_rows, m0_rows, stream)
            device = device or torch.device("cuda", torch.cuda.current_device())
        self.block = block
        self.stream = getattr(block, "stream", None)
        self._graph = None
        self.device = device or torch.device("cpu")
        dt = getattr(torch, block.dtype)
        # the gathered stage values (world chunks; entries past N stay zero)
        # and this rank's chunk; both 16-byte aligned as whole tensors
        self.x = torch.zeros(self.world * self.chunk + 4, dtype=dt, device=self.device)
        self.x_own = torch.zeros(self.chunk, dtype=dt, device=self.device)

    def _exchange(self):
        if self.world == 1:
            self.x[:self.rows].copy_(self.x_own[:self.rows])
            return
        import torch.distributed as dist
        dist.all_gather_into_tensor(self.x[:self.world * self.chunk], self.x_own, group=self.group)

    def _sample(self, u_t, row):
        """One input sample: substeps x 4 stages, each followed by the exchange."""
        S = int(self.params.substeps)
        for j in range(S):
            for st in range(4):
                flags = (SAMPLE_START if (j == 0 and st == 0) else 0) | \
                        (SAMPLE_END if (j == S - 1 and st == 3) else 0)
                self.block.stage(self.x, st, u_t if flags & SAMPLE_START else None, flags, self.x_own,
                                 row if flags & SAMPLE_END else None)
                self._exchange()

    def run(self, u, states_out=None, graph: bool = False):
        """Advance over the input series u (T x n_in, a tensor on this rank's
        device); states_out (T x rows, same device) receives this block's
        samples.  Every rank calls run with the same u.

        graph=True (CUDA blocks): one input sample (its 4 x substeps stage
        launches and exchanges) is captured once as a CUDA graph and replayed
        per sample, with the sample's input and output rows copied through
        fixed buffers; the results are the same bits."""
        import contextlib

        import torch
        T = int(u.shape[0])
        caller = torch.cuda.current_stream() if self.stream is not None else None
        if caller is not None:
            self.stream.wait_stream(caller)  # the caller's inputs first
        ctx = torch.cuda.stream(self.stream) if self.stream is not None else contextlib.nullcontext()
        try:
            return self._run(u, states_out, graph, T, ctx)
        finally:
            if caller is not None:
                caller.wait_stream(self.stream)  # then the caller's later work

    def _run(self, u, states_out, graph, T, ctx):
        import torch
        with ctx:
            self.block.publish(self.x_own)
            self._exchange()
            if not graph:
                for t in range(T):
                    self._sample(u[t], states_out[t] if states_out is not None else None)
                return states_out
            if self.stream is None:
                raise ValueError("graph=True needs a CUDA block")
            if self._graph is None:
                self._u_buf = torch.zeros(int(self.params.n_in), dtype=torch.float32, device=self.device)
                self._row_buf = torch.zeros(self.rows, dtype=torch.float32, device=self.device)
                g = torch.cuda.CUDAGraph()
                # relaxed: the library checks its pointers (cudaPointerGetAttributes)
                with torch.cuda.graph(g, stream=self.stream, capture_error_mode="relaxed"):
                    self._sample(self._u_buf, self._row_buf)
                self._graph = g
            for t in range(T):
                self._u_buf.copy_(u[t])
                self._graph.replay()
                if states_out is not None:
                    states_out[t].copy_(self._row_buf)
        return states_out

    def state(self) -> np.ndarray:
        return self.block.state()
