"""Reverse-time adjoint: gradient of a trace misfit with respect to squared slowness.

``Propagate.apply(m, geometry)`` maps the squared slowness m = 1/v^2 (a CUDA
tensor shaped like the grid) to the traces [nt][nrec] of one shot, running the
fused step kernels of libfd; its backward is the discrete adjoint of that time
step.  With w = (dt v / h)^2, damping a and g^n = dJ/dtrace^n, the adjoint
wavefield psi obeys the same damped leapfrog backwards in time,

    (1 + a) psi_k = 2 psi_{k+1} - (1 - a) psi_{k+2} + W L' psi_{k+1} + W R^T g^{k-1},

so it advances with ``fd_step`` on a second model with the same velocity and no
source, the receiver terms entering through ``fd_inject_receivers``; the
gradient is dJ/dm = -(1/m) sum_n psi_{n+1} L'P^n.  The sponge's damping is held
fixed.

Memory is bounded by checkpointing: the forward pass keeps (P, Pold) every
``checkpoint_every`` steps; the backward pass walks the segments last to first
and recomputes each segment from its checkpoint with ``fd_step_lp``, which
stores the stencil sums L'P^n the imaging condition needs (one field per step
of the segment) instead of the levels themselves.  The adjoint then runs through
the segment, each adjoint step adding psi_{n+1} L'P^n to the gradient as it
goes (``fd_step_image``, ``fd_inject_receivers_image``); one
``fd_adjoint_segment`` call issues a whole segment from native code.  The
forward work is therefore done twice, and no stencil is evaluated a third time.

With ``store_all`` the forward pass keeps every L'P^n instead (``fd_step_lp_n``;
nt fields, 100 GB for 256^3 x 1500 steps, which the B300's HBM holds) and the
backward pass runs the adjoint straight through them (``fd_adjoint_backward``)
without recomputing: the same gradient, bitwise, in less time.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fd


@dataclass
class Geometry:
    """One shot's fixed inputs (everything but the model)."""
    ndim: int
    shape: tuple
    h: float
    dt: float
    nt: int
    src: tuple
    wavelet: np.ndarray
    receivers: np.ndarray
    sponge_width: int = 0
    sponge_R: float = 1e-3
    sponge_vmax: float | None = None
    checkpoint_every: int = 50
    store_all: bool = False     # keep every L'P^n (nt fields) instead of checkpoints

    @classmethod
    def from_shot(cls, shot, checkpoint_every=50, sponge_vmax=None, store_all=False):
        return cls(shot.ndim, tuple(shot.shape), shot.h, shot.dt, shot.nt, shot.src, shot.wavelet, shot.receivers,
                   shot.sponge_width, shot.sponge_R, sponge_vmax, checkpoint_every, store_all)


def _model(torch, geo: Geometry, v, with_source: bool):
    stream = torch.cuda.current_stream()
    m = fd.Model(geo.ndim, geo.shape, geo.h, geo.dt, v.contiguous(), geo.sponge_width, geo.sponge_R, stream=stream)
    if geo.sponge_vmax is not None:
        fd.fd_set_sponge_vmax(m.handle, geo.sponge_vmax)
    if with_source:
        m.set_source(geo.src, geo.wavelet)
    m.set_receivers(geo.receivers)
    return m


class Propagate:
    """torch.autograd.Function: squared slowness -> traces, with the adjoint as backward."""

    _fn = None

    @classmethod
    def apply(cls, m, geo: Geometry):
        if cls._fn is None:
            cls._fn = _make_function()
        return cls._fn.apply(m, geo)


def _make_function():
    import torch

    class _Propagate(torch.autograd.Function):
        @staticmethod
        def forward(ctx, m, geo):
            if not m.is_cuda:
                raise ValueError("m must be a CUDA tensor")
            v = torch.rsqrt(m.detach().to(torch.float32)).contiguous()
            model = _model(torch, geo, v, with_source=True)
            nrec = len(geo.receivers)
            traces = torch.zeros((geo.nt, nrec), device=m.device, dtype=torch.float32)
            fd.fd_reset(model.handle)
            fd.fd_set_trace_buffer(model.handle, traces, geo.nt)
            ckpts = []
            lp_all = None
            if geo.store_all:
                lp_all = torch.empty((geo.nt,) + tuple(geo.shape), device=m.device, dtype=torch.float32)
                fd.fd_step_lp_n(model.handle, geo.nt, lp_all)           # lp_all[n] = L'P^n
            else:
                K = max(1, int(geo.checkpoint_every))
                for n0 in range(0, geo.nt, K):
                    P = torch.empty(geo.shape, device=m.device, dtype=torch.float32)
                    Po = torch.empty_like(P)
                    fd.fd_get_wavefield_dev(model.handle, P, Po)
                    ckpts.append((P, Po))
                    fd.fd_step(model.handle, min(K, geo.nt - n0))
            fd.fd_synchronize(model.handle)
            ctx.geo = geo
            ctx.model = model
            ctx.v = v
            ctx.ckpts = ckpts
            ctx.lp_all = lp_all
            ctx.save_for_backward(m)
            return traces

        @staticmethod
        def backward(ctx, grad_traces):
            (m,) = ctx.saved_tensors
            geo, model, v = ctx.geo, ctx.model, ctx.v
            g = grad_traces.detach().to(torch.float32).contiguous()
            K = max(1, int(geo.checkpoint_every))
            adj = _model(torch, geo, v, with_source=False)
            fd.fd_reset(adj.handle)
            acc = torch.zeros(geo.shape, device=m.device, dtype=torch.float32)
            if ctx.lp_all is not None:
                # every L'P^n is stored: the adjoint runs back through them at once
                fd.fd_adjoint_backward(adj.handle, 0, geo.nt, ctx.lp_all, g, acc)
                ctx.lp_all = None
            fd.fd_set_trace_buffer(model.handle, None, 0)       # recompute without recording
            seg = torch.empty((K,) + tuple(geo.shape), device=m.device, dtype=torch.float32) if ctx.ckpts else None
            for s in range(len(ctx.ckpts) - 1, -1, -1):
                n0 = s * K
                n1 = min(n0 + K, geo.nt)
                P, Po = ctx.ckpts[s]
                fd.fd_set_wavefield_dev(model.handle, P, Po, n0)
                # seg[j] = L'P^{n0+j}; then for k = n1 .. n0+1: psi_k from psi_{k+1},
                # psi_{k+2}, + w g^{k-1} / (1 + a) at the receivers, acc += psi_k L'P^{k-1}
                fd.fd_adjoint_segment(model.handle, adj.handle, n0, n1, seg, g, acc)
            fd.fd_synchronize(adj.handle)
            adj.close()
            model.close()
            ctx.model = None
            ctx.ckpts = None
            grad_m = -(acc / m.detach().to(torch.float32)).to(m.dtype)
            return grad_m, None

    return _Propagate


def misfit_and_gradient(m, geo: Geometry, observed):
    """J = 1/2 |traces(m) - observed|^2 (accumulated in FP64) and dJ/dm."""
    import torch
    mm = m.detach().clone().requires_grad_(True)
    tr = Propagate.apply(mm, geo)
    r = tr - observed
    J = 0.5 * (r.double() * r.double()).sum()
    J.backward()
    return float(J.detach()), mm.grad
