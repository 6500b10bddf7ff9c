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
            m32 = m.detach().to(torch.float32).contiguous()
            v = torch.empty_like(m32)
            fd.fd_velocity_from_slowness(m32, v, torch.cuda.current_stream())
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
            grad_m = torch.empty(geo.shape, device=m.device, dtype=torch.float32)
            fd.fd_gradient_from_image(acc, m.detach().to(torch.float32).contiguous(), grad_m,
                                      torch.cuda.current_stream())
            return grad_m.to(m.dtype), None

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


# ---------------------------------------------------------------- many shots at once

class ShotLanes:
    """The summed misfit J = 1/2 sum_shots |d_s(m) - observed_s|^2 and dJ/dm over
    many shots of one grid, with the shots spread over ``lanes`` CUDA streams
    that run at the same time.

    A single shot of a mid-sized grid does not fill the B300 (at 256^3 a step
    launch is under two waves of CTAs), so running shots side by side recovers
    the idle SMs.  Each lane owns a forward and an adjoint model, its
    checkpoint and segment buffers and a library stream, allocated once and
    reused for every shot and every call; a host thread per lane issues its
    shots' work (forward with checkpoints, residual, segment-wise adjoint), so a
    lane never waits on another lane's launches.  Each lane accumulates its
    shots' images psi_{n+1} L'P^n; ``fd_gradient_from_image`` sums the lanes and
    divides by -m.  The per-shot arithmetic is that of ``Propagate``.

    All shots must share the grid, h, dt, sponge and nt; sources, wavelets and
    receivers may differ.
    """

    def __init__(self, geos, lanes=4):
        import torch
        self.torch = torch
        self.geos = list(geos)
        g0 = self.geos[0]
        for g in self.geos:
            if (g.ndim, tuple(g.shape), g.h, g.dt, g.nt, g.sponge_width, g.sponge_R, g.sponge_vmax,
                    g.checkpoint_every) != (g0.ndim, tuple(g0.shape), g0.h, g0.dt, g0.nt, g0.sponge_width,
                                           g0.sponge_R, g0.sponge_vmax, g0.checkpoint_every):
                raise ValueError("all shots of a ShotLanes must share grid, time step, sponge and nt")
        self.shape = tuple(g0.shape)
        self.nt = g0.nt
        self.K = max(1, int(g0.checkpoint_every))
        self.nseg = (self.nt + self.K - 1) // self.K
        nrec = max(len(g.receivers) for g in self.geos)
        L = max(1, min(int(lanes), len(self.geos)))
        dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.acc = torch.zeros((L,) + self.shape, device=dev, dtype=torch.float32)
        self.lanes = []
        placeholder = 1e-3 * g0.h / g0.dt      # a velocity far inside the Courant limit
        for _ in range(L):
            handle, _ = fd.fd_stream_create(0)
            ext = torch.cuda.ExternalStream(handle)
            with torch.cuda.stream(ext):
                v0 = torch.full(self.shape, placeholder, device=dev, dtype=torch.float32)
                models = []
                for _k in range(2):
                    md = fd.Model(g0.ndim, self.shape, g0.h, g0.dt, v0, g0.sponge_width, g0.sponge_R, stream=handle)
                    if g0.sponge_vmax is not None:
                        fd.fd_set_sponge_vmax(md.handle, g0.sponge_vmax)
                    models.append(md)
                lane = {
                    "stream": handle, "ext": ext, "fwd": models[0], "adj": models[1], "geo": None,
                    "ckpts": torch.empty((self.nseg, 2) + self.shape, device=dev, dtype=torch.float32),
                    "seg": torch.empty((self.K,) + self.shape, device=dev, dtype=torch.float32),
                    "traces": torch.empty((self.nt, nrec), device=dev, dtype=torch.float32),
                    "J": torch.zeros((), device=dev, dtype=torch.float64),
                }
            ext.synchronize()
            self.lanes.append(lane)

    def _shot(self, lane, geo, obs, backward, acc):
        torch = self.torch
        fwd, adj = lane["fwd"], lane["adj"]
        if lane["geo"] is not geo:
            fwd.set_source(geo.src, geo.wavelet)
            fwd.set_receivers(geo.receivers)
            adj.set_receivers(geo.receivers)
            lane["geo"] = geo
        nrec = len(geo.receivers)
        traces = lane["traces"][:, :nrec] if nrec == lane["traces"].shape[1] else \
            lane["traces"].view(-1)[:self.nt * nrec].view(self.nt, nrec)
        fd.fd_reset(fwd.handle)
        fd.fd_set_trace_buffer(fwd.handle, traces, self.nt)
        ck = lane["ckpts"]
        for s in range(self.nseg):
            fd.fd_get_wavefield_dev(fwd.handle, ck[s, 0], ck[s, 1])
            fd.fd_step(fwd.handle, min(self.K, self.nt - s * self.K))
        r = (traces - obs).contiguous()
        lane["J"] += (r.double() * r.double()).sum()
        if not backward:
            return
        fd.fd_reset(adj.handle)
        fd.fd_set_trace_buffer(fwd.handle, None, 0)       # the recompute records nothing
        for s in range(self.nseg - 1, -1, -1):
            n0 = s * self.K
            n1 = min(n0 + self.K, self.nt)
            fd.fd_set_wavefield_dev(fwd.handle, ck[s, 0], ck[s, 1], n0)
            fd.fd_adjoint_segment(fwd.handle, adj.handle, n0, n1, lane["seg"], r, acc)

    def _lane(self, li, v, observed, backward):
        torch = self.torch
        torch.cuda.set_device(self.device)
        lane = self.lanes[li]
        with torch.cuda.stream(lane["ext"]):
            fd.fd_set_velocity_dev(lane["fwd"].handle, v)
            fd.fd_set_velocity_dev(lane["adj"].handle, v)
            acc = self.acc[li]
            acc.zero_()
            lane["J"].zero_()
            for j in range(li, len(self.geos), len(self.lanes)):
                self._shot(lane, self.geos[j], observed[j], backward, acc)
            fd.fd_synchronize(lane["fwd"].handle)
            fd.fd_synchronize(lane["adj"].handle)

    def run(self, m, observed, backward=True):
        """(J, dJ/dm) for squared slowness m (FP32 CUDA tensor shaped like the grid)
        and one observed trace array [nt][nrec] per shot; dJ/dm is None without
        ``backward``."""
        import concurrent.futures as cf
        torch = self.torch
        if len(observed) != len(self.geos):
            raise ValueError("one observed trace array per shot")
        m32 = m.detach().to(torch.float32).contiguous()
        v = torch.empty_like(m32)
        cur = torch.cuda.current_stream()
        fd.fd_velocity_from_slowness(m32, v, cur)
        obs = [o.detach().to(torch.float32).contiguous() for o in observed]
        cur.synchronize()                       # v, m and the observed data are ready for every lane
        with cf.ThreadPoolExecutor(len(self.lanes)) as ex:
            for f in [ex.submit(self._lane, li, v, obs, backward) for li in range(len(self.lanes))]:
                f.result()
        J = 0.5 * float(sum(float(lane["J"]) for lane in self.lanes))
        if not backward:
            return J, None
        grad = torch.empty_like(m32)
        fd.fd_gradient_from_image(self.acc, m32, grad, cur)
        return J, grad

    def close(self):
        for lane in self.lanes:
            lane["fwd"].close()
            lane["adj"].close()
            fd.fd_stream_destroy(lane["stream"])
        self.lanes = []


class ShotsMisfit:
    """torch.autograd.Function: squared slowness -> the summed misfit of a
    ShotLanes' shots (an FP64 scalar), whose backward is their adjoint gradient."""

    _fn = None

    @classmethod
    def apply(cls, m, lanes: ShotLanes, observed):
        if cls._fn is None:
            import torch

            class _ShotsMisfit(torch.autograd.Function):
                @staticmethod
                def forward(ctx, m, lanes, observed):
                    J, grad = lanes.run(m, observed, backward=True)
                    ctx.save_for_backward(grad)
                    return torch.tensor(J, dtype=torch.float64, device=m.device)

                @staticmethod
                def backward(ctx, gJ):
                    (grad,) = ctx.saved_tensors
                    return (gJ.to(grad.dtype) * grad).to(grad.dtype), None, None

            cls._fn = _ShotsMisfit
        return cls._fn.apply(m, lanes, tuple(observed))
