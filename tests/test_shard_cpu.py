"""The row-sharded split of one reservoir (paper_2312_01121_b300/shard.py) on
CPU ranks over gloo: partition, stage schedule and the all-gather of the
stage values between stages.  Each rank's block is computed on the host from
the oracle's vector field (its rows of W times the gathered values, then
Eq. (gov) with that coupling field), so the sharded run must reproduce the
oracle's whole-reservoir run to rounding (1e-11).  The CUDA block is
checked against the oracle in tests/test_gpu_shard.py."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def test_partition_covers_every_row_once():
    from paper_2312_01121_b300.shard import partition
    for N in (1, 2, 7, 13, 100, 1001):
        for world in range(1, min(N, 9) + 1):
            try:
                blocks = partition(N, world)
            except ValueError:
                # only when equal chunks leave the last rank empty
                assert -(-N // world) * (world - 1) >= N
                continue
            rows = [r for r0, n in blocks for r in range(r0, r0 + n)]
            assert rows == list(range(N))
            assert all(n == -(-N // world) for _, n in blocks[:-1])
    with pytest.raises(ValueError):
        partition(3, 4)


class OracleBlock:
    """Rows [row0, row0 + rows) advanced on the host, in FP64, with the
    oracle's field: b_x gets A_cp (W_rows x) + H_in."""
    dtype = "float64"

    def __init__(self, OP, W, w_in, m0, row0, rows):
        self.OP, self.rows = OP, rows
        self.Wr = np.ascontiguousarray(W[row0:row0 + rows])
        self.win = np.ascontiguousarray(w_in[row0:row0 + rows])
        self.mn = np.ascontiguousarray(m0[:, row0:row0 + rows], dtype=np.float64)
        self.ms, self.ks, self.hin = self.mn.copy(), np.zeros_like(self.mn), np.zeros(rows)
        self.zero = np.zeros((rows, rows))

    def publish(self, x_rows):
        x_rows[:self.rows] = torch.from_numpy(self.mn[0].copy())

    def stage(self, x, st, u_t, flags, x_next, states_row):
        import oracle
        N = self.Wr.shape[1]
        if flags & 1:
            self.hin = oracle.input_field(self.OP, self.win, u_t.numpy())
        h = self.OP.A_cp * (self.Wr @ x.numpy()[:N])
        y = self.mn if st == 0 else self.ms
        d = self.OP.dt * oracle.field(self.OP.replace(A_cp=0.0), self.zero, y, self.hin + h)[0]
        w, c = (1.0, 2.0, 2.0, 1.0)[st], (0.5, 0.5, 1.0, 0.0)[st]
        self.ks = w * d if st == 0 else self.ks + w * d
        if st == 3:
            self.mn = self.mn + self.ks / 6.0
            self.ms = self.mn
        else:
            self.ms = self.mn + c * d
        x_next[:self.rows] = torch.from_numpy(self.ms[0].copy())
        if st == 3 and (flags & 2) and states_row is not None:
            states_row[:] = torch.from_numpy(self.mn[self.OP.component].copy())

    def state(self):
        return self.mn.copy()


def _system(N, T):
    import helpers
    return helpers.make_system(N, "gauss", seed=N, T=T, n_in=2)


def _worker(rank, world, port, N, T, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    import helpers
    from paper_2312_01121_b300 import sto
    from paper_2312_01121_b300.shard import ShardedReservoir, partition
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    W, w_in, m0, u = _system(N, T)
    P = sto.Params(substeps=4, A_cp=150.0, A_in=20.0, n_in=2)
    OP = helpers.oracle_params(P)
    row0, rows = partition(N, world)[rank]
    block = OracleBlock(OP, W.astype(np.float64), w_in.astype(np.float64), m0, row0, rows)
    res = ShardedReservoir(N, P, block=block)
    assert (res.row0, res.rows, res.world, res.rank) == (row0, rows, world, rank)
    st = torch.zeros((T, rows), dtype=torch.float64)
    res.run(torch.from_numpy(u.astype(np.float64)), st)
    out[rank] = (row0, rows, st.numpy().copy(), res.state())
    dist.destroy_process_group()


@pytest.mark.parametrize("N,world", [(13, 2), (13, 3), (40, 2)])
def test_sharded_run_over_gloo_equals_whole_reservoir(N, world):
    import helpers
    import oracle
    from paper_2312_01121_b300 import sto
    T = 3
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        s = socket.socket()
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
        s.close()
        procs = [ctx.Process(target=_worker, args=(r, world, port, N, T, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        res = dict(out)
    W, w_in, m0, u = _system(N, T)
    P = sto.Params(substeps=4, A_cp=150.0, A_in=20.0, n_in=2)
    m_ref, st_ref = oracle.run(helpers.oracle_params(P), W.astype(np.float64), w_in.astype(np.float64),
                               m0.astype(np.float64), u.astype(np.float64))
    seen = []
    for r in range(world):
        row0, rows, st, m = res[r]
        seen.extend(range(row0, row0 + rows))
        assert np.max(np.abs(st - st_ref[:, row0:row0 + rows])) <= 1e-11
        assert np.max(np.abs(m - m_ref[:, row0:row0 + rows])) <= 1e-11
    assert seen == list(range(N))
