"""Differentiable TTI, elastic and isotropic acoustic modelling for PyTorch.

``TTIModelling.apply(m, wavelet, spec)`` maps squared slowness m = 1/vp^2
[s^2/m^2] (physical grid) and the source wavelets to receiver traces.  Its
backward pass is the library's adjoint-state gradient (Sec. III: zero-lag
cross-correlation of the forward wavefield with the adjoint wavefield driven
by the incoming trace gradient), returning dL/dm and dL/dwavelet.  Forward
wavefields are kept inside the library according to ``spec.snap_mode``:
full FP32 storage, or checkpoints (FP32, BF16 or FP16 with one scale per
field) with FP32 recomputation of each segment during the adjoint sweep.

``ElasticModelling.apply(lam, mu, b, wavelet, spec)`` does the same for the
elastic system with respect to the Lame parameters and buoyancy, and
``AcousticModelling.apply(m, wavelet, spec)`` for the isotropic acoustic
equation of Sec. II-A (Eq. acou).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import (PROP_ACOUSTIC, PROP_ELASTIC, PROP_TTI, SNAP_FULL_FP32, Propagator)


@dataclass
class Spec:
    """Static part of a modelling problem (everything except the model
    parameters being differentiated and the wavelet)."""
    shape: tuple            # physical (nx, ny, nz)
    nbl: int
    h: float
    space_order: int
    nt: int
    dt: float
    src: torch.Tensor       # [nsrc, 3]
    rec: torch.Tensor       # [nrec, 3]
    eps: torch.Tensor = None      # TTI
    delta: torch.Tensor = None
    theta: torch.Tensor = None
    phi: torch.Tensor = None
    vdamp: float = 0.0
    snap_mode: int = SNAP_FULL_FP32
    ckpt_interval: int = 0


def _stream(t):
    return torch.cuda.current_stream(t.device).cuda_stream if t.is_cuda else None


class TTIModelling(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, wavelet, spec: Spec):
        vp = torch.rsqrt(m.detach().to(torch.float32)) / 1000.0          # km/s
        model = [vp.contiguous(), spec.eps, spec.delta, spec.theta, spec.phi]
        prop = Propagator(PROP_TTI, spec.shape, spec.nbl, spec.h, spec.space_order, spec.nt,
                          model, dt=spec.dt, vdamp=spec.vdamp, snap_mode=spec.snap_mode,
                          ckpt_interval=spec.ckpt_interval, stream=_stream(m))
        traces = prop.forward(wavelet.detach().contiguous(), spec.src, spec.rec, save=True)
        ctx.prop = prop
        ctx.nsrc = spec.src.shape[0]
        return traces

    @staticmethod
    def backward(ctx, gtr):
        prop = ctx.prop
        gm, gw = prop.backward(gtr.contiguous(), nsrc=ctx.nsrc)
        prop.close()
        ctx.prop = None
        return gm, gw, None


class AcousticModelling(torch.autograd.Function):
    """m = 1/vp^2 [s^2/m^2] on the physical grid and the wavelets -> traces."""

    @staticmethod
    def forward(ctx, m, wavelet, spec: Spec):
        vp = torch.rsqrt(m.detach().to(torch.float32)) / 1000.0          # km/s
        prop = Propagator(PROP_ACOUSTIC, spec.shape, spec.nbl, spec.h, spec.space_order, spec.nt,
                          [vp.contiguous()], dt=spec.dt, vdamp=spec.vdamp, snap_mode=spec.snap_mode,
                          ckpt_interval=spec.ckpt_interval, stream=_stream(m))
        traces = prop.forward(wavelet.detach().contiguous(), spec.src, spec.rec, save=True)
        ctx.prop = prop
        ctx.nsrc = spec.src.shape[0]
        return traces

    @staticmethod
    def backward(ctx, gtr):
        prop = ctx.prop
        gm, gw = prop.backward(gtr.contiguous(), nsrc=ctx.nsrc)
        prop.close()
        ctx.prop = None
        return gm, gw, None


class ElasticModelling(torch.autograd.Function):
    """Parameters on the physical grid: lam [Pa], mu [Pa], b = 1/rho [m^3/kg]."""

    @staticmethod
    def forward(ctx, lam, mu, b, wavelet, spec: Spec):
        rho = 1.0 / b.detach()
        vp = torch.sqrt((lam.detach() + 2 * mu.detach()) * b.detach()) / 1000.0
        vs = torch.sqrt(torch.clamp(mu.detach(), min=0) * b.detach()) / 1000.0
        model = [vp.float().contiguous(), vs.float().contiguous(), (rho / 1000.0).float().contiguous()]
        prop = Propagator(PROP_ELASTIC, spec.shape, spec.nbl, spec.h, spec.space_order, spec.nt,
                          model, dt=spec.dt, snap_mode=spec.snap_mode,
                          ckpt_interval=spec.ckpt_interval, stream=_stream(lam))
        traces = prop.forward(wavelet.detach().contiguous(), spec.src, spec.rec, save=True)
        ctx.prop = prop
        ctx.nsrc = spec.src.shape[0]
        return traces

    @staticmethod
    def backward(ctx, gtr):
        g, gw = ctx.prop.backward(gtr.contiguous(), nsrc=ctx.nsrc)
        ctx.prop.close()
        ctx.prop = None
        return g[0], g[1], g[2], gw, None


def tti_spec_from_problem(prob, device, **kw) -> Spec:
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
    return Spec((prob.nx, prob.ny, prob.nz), prob.nbl, prob.h, prob.so, prob.nt, prob.dt,
                t(prob.src), t(prob.rec), t(prob.model["eps"]), t(prob.model["delta"]),
                t(prob.model["theta"]), t(prob.model["phi"]),
                vdamp=getattr(prob, "vdamp", 0.0) or 0.0, **kw)


def acoustic_spec_from_problem(prob, device, **kw) -> Spec:
    """Spec of an acoustic ``synth.Problem`` (model given to
    ``AcousticModelling.apply`` as m = 1/vp^2)."""
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
    return Spec((prob.nx, prob.ny, prob.nz), prob.nbl, prob.h, prob.so, prob.nt, prob.dt,
                t(prob.src), t(prob.rec), vdamp=getattr(prob, "vdamp", 0.0) or 0.0, **kw)
