"""torch.autograd integration of the simulator.

`sto_states(res, A_cp, current, w_in, u)` returns the sampled reservoir
states of `res.run(u)` as a differentiable function of the coupling
strength A_cp, the current I and the input weights w_in; backward calls the
hand-written discrete adjoint (`sto_adjoint`) with checkpointing.  The
forward advances the reservoir's state exactly like `Reservoir.run`.
"""
from __future__ import annotations

import numpy as np
import torch

from . import sto


class StoRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A_cp, current, w_in, u, res, ckpt_every):
        params = res.params.replace(A_cp=float(A_cp), current=float(current))
        res.set_params(params)
        res.set_input_weights(w_in.detach().to(torch.float32).contiguous())
        m0 = res.state()
        T = int(u.shape[0])
        states = torch.empty((T, res.N), dtype=torch.float32, device=u.device)
        res.run(u, states)
        ctx.res, ctx.m0, ctx.ckpt = res, m0, int(ckpt_every)
        ctx.save_for_backward(u, w_in)
        return states

    @staticmethod
    def backward(ctx, grad_states):
        u, w_in = ctx.saved_tensors
        res = ctx.res
        m_end = res.state()
        res.set_state(ctx.m0)
        g = res.adjoint(u, grad_states.detach().to(torch.float32).contiguous(), ctx.ckpt,
                        want_m0=False)
        res.set_state(m_end)
        dA = torch.tensor(g["A_cp"], dtype=torch.float64)
        dI = torch.tensor(g["current"], dtype=torch.float64)
        dw = torch.from_numpy(np.ascontiguousarray(g["w_in"])).to(w_in.device, w_in.dtype)
        return dA, dI, dw, None, None, None


def sto_states(res: "sto.Reservoir", A_cp, current, w_in, u, ckpt_every: int = 100):
    """Differentiable sampled states (T x N, float32) of res.run(u)."""
    return StoRun.apply(A_cp, current, w_in, u, res, ckpt_every)


def ridge_objective(states, y, washout: int, beta: float):
    """Ridge objective with bias at the fitted readout: the mean squared error
    on samples t >= washout plus beta * |w|^2 (bias not penalised), in FP64.
    Differentiating through the solve gives the envelope-theorem gradient."""
    X = states[washout:].to(torch.float64)
    n = X.shape[0]
    X = torch.cat([X, torch.ones((n, 1), dtype=X.dtype, device=X.device)], dim=1)
    yt = y[washout:].to(torch.float64)
    D = torch.eye(X.shape[1], dtype=X.dtype, device=X.device)
    D[-1, -1] = 0.0
    w = torch.linalg.solve(X.T @ X / n + beta * D, X.T @ yt / n)
    r = X @ w - yt
    return (r * r).mean() + beta * (w[:-1] * w[:-1]).sum()
