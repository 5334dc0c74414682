"""torch.autograd wrappers of the hand-written adjoints, and a checkpointed
rollout giving the gradient of the volume-averaged Nusselt number with respect
to the initial temperature.

All forward and backward arithmetic runs in libafid (afid_project,
afid_rk3_substep and their *_adjoint entry points); this module only
orchestrates calls and buffers. The time step is treated as a constant: the
CFL maximum (Listing 1) is not differentiated, a rollout records its dt
sequence forward and reuses it backward.

Nu = 1 + sqrt(Ra Pr) <w T>_V, the volume form of the Nusselt number (wall
temperatures fixed, so <-dT/dz>_V = 1), with <.>_V the sum over interior
z-faces weighted by dx dy dzf_k divided by the box volume; afid_nusselt forms
it and its derivatives with respect to w and T on the device.
"""
from __future__ import annotations

import math

import torch

from .afid import Context


def _zeros_like_state(S):
    return [torch.zeros_like(a) if a is not None else None for a in S]


def _clone(S):
    return [a.clone() if a is not None else None for a in S]


def _run_step(ctx: Context, dt: float, S, save_substeps: bool = False):
    """One RK3 step in place on S = [u, v, w, T, p]; returns the inputs of the
    three substeps when save_substeps."""
    H = [torch.zeros_like(S[0]), torch.zeros_like(S[1]), torch.zeros_like(S[2]),
         torch.zeros_like(S[3]) if S[3] is not None else None]
    saved = []
    for l in range(3):
        if save_substeps:
            saved.append(_clone(S[:4]))
        ctx.rk3_substep(l, dt, *S, *H)
    return saved


def _step_adjoint(ctx: Context, dt: float, substep_inputs, G):
    """Reverse the three substeps of one step: G = [gu, gv, gw, gT, gp] holds the
    cotangent of the step's output on entry and of its input on exit."""
    gH = [torch.zeros_like(G[0]), torch.zeros_like(G[1]), torch.zeros_like(G[2]),
          torch.zeros_like(G[3]) if G[3] is not None else None]
    for l in (2, 1, 0):
        u, v, w, T = substep_inputs[l]
        ctx.rk3_substep_adjoint(l, dt, u, v, w, T, G[0], G[1], G[2], G[3], G[4], *gH)
    return G


class ProjectFn(torch.autograd.Function):
    """(u, v, w, p) -> pressure-corrected (u, v, w, p) with scale s and the
    pressure-update coefficient beta (afid_project / afid_project_adjoint)."""

    @staticmethod
    def forward(fctx, ctx: Context, u, v, w, p, s: float = 1.0, beta: float = 0.0):
        out = [u.detach().clone(), v.detach().clone(), w.detach().clone(), p.detach().clone()]
        ctx.project(*out, s, beta)
        fctx.shapes = [(tuple(a.shape), a.device) for a in out]
        fctx.afid = ctx
        fctx.sb = (s, beta)
        return tuple(out)

    @staticmethod
    def backward(fctx, gu, gv, gw, gp):
        G = [g.contiguous().clone() if g is not None else torch.zeros(sh, dtype=torch.float64, device=dv)
             for g, (sh, dv) in zip((gu, gv, gw, gp), fctx.shapes)]
        fctx.afid.project_adjoint(*G, *fctx.sb)
        return (None, G[0], G[1], G[2], G[3], None, None)


class RK3StepFn(torch.autograd.Function):
    """One full RK3 step (three substeps, fixed dt) of (u, v, w, T, p)."""

    @staticmethod
    def forward(fctx, ctx: Context, dt: float, u, v, w, T, p):
        S = [u.detach().clone(), v.detach().clone(), w.detach().clone(), T.detach().clone(),
             p.detach().clone()]
        fctx.save_for_backward(u.detach(), v.detach(), w.detach(), T.detach(), p.detach())
        fctx.afid = ctx
        fctx.dt = dt
        _run_step(ctx, dt, S)
        return tuple(S)

    @staticmethod
    def backward(fctx, gu, gv, gw, gT, gp):
        u, v, w, T, p = fctx.saved_tensors
        S = [u.clone(), v.clone(), w.clone(), T.clone(), p.clone()]
        subs = _run_step(fctx.afid, fctx.dt, S, save_substeps=True)   # recompute
        G = [g.contiguous().clone() if g is not None else torch.zeros_like(r)
             for g, r in zip((gu, gv, gw, gT, gp), S)]
        _step_adjoint(fctx.afid, fctx.dt, subs, G)
        return (None, None, G[0], G[1], G[2], G[3], G[4])


def nusselt_gradient(ctx: Context, state0, dts, ra: float, pr: float, checkpoint_every: int = 5):
    """Nu after len(dts) RK3 steps from state0 = (u, v, w, T, p) (device tensors,
    unchanged) and dNu/dT0 (interior faces; walls are data and get zero). Nu and
    its seed cotangents come from afid_nusselt.

    Checkpointing: the forward keeps the state at every `checkpoint_every`-th
    step; the backward recomputes each segment from its checkpoint, keeping the
    segment's step inputs, and reverses the steps (and within each step its
    three substeps, whose inputs the segment recompute kept) with the
    hand-written substep adjoint. Memory: about n/c + 3c states instead of 3n."""
    n = len(dts)
    c = max(1, int(checkpoint_every))
    S = _clone(state0)
    ckpt = {}
    for s in range(n):
        if s % c == 0:
            ckpt[s] = _clone(S)
        _run_step(ctx, dts[s], S)
    G = _zeros_like_state(S)
    nu, G[2], G[3] = ctx.nusselt(S[2], S[3], math.sqrt(ra * pr), seeds=True)  # Nu, dNu/dw, dNu/dT
    starts = sorted(ckpt)
    for seg_start in reversed(starts):
        seg_end = min(seg_start + c, n)
        X = _clone(ckpt[seg_start])
        subs = [_run_step(ctx, dts[s], X, save_substeps=True) for s in range(seg_start, seg_end)]
        for s in reversed(range(seg_start, seg_end)):
            _step_adjoint(ctx, dts[s], subs[s - seg_start], G)
    return nu, G[3]   # the substep adjoint leaves the wall planes of gT at zero
