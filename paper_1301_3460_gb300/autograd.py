"""torch.autograd glue for differentiating gauge-fixed observables.

GaugeFixUnroll: K Fourier-accelerated steepest-descent steps (FP64), links in,
links out, with checkpoints every `every` steps; the backward recomputes each
segment forward from its checkpoint and applies the hand-written step
vector-Jacobian product (lgf_step_bwd) in reverse.  GluonPmin: the Landau-gauge
gluon propagator at the smallest momenta and its derivative (lgf_gluon_pmin,
lgf_gluon_pmin_bwd).  Tensors are complex128 CUDA tensors (4, V, 3, 3); the
gradient convention is torch's (dL = Re sum conj(grad) dU).
"""
from __future__ import annotations

import torch

from . import lgf


class GaugeFixUnroll(torch.autograd.Function):
    """Checkpoints and the states replayed in the backward are snapshots of the
    library's own link layout (save_links / load_links): device-to-device copies,
    without the conversion and SU(3) check of set_links."""

    @staticmethod
    def forward(ctx, U0, lat, K: int, alpha: float, every: int):
        U0 = U0.detach().contiguous()
        lat.set_links(U0)
        ckpts = [lat.save_links()]
        done = 0
        while done < K:
            n = min(every, K - done)
            lat.fix(alpha, 0.0, n)
            done += n
            if done < K:
                ckpts.append(lat.save_links())
        UK = lat.get_links(device=U0.device)
        ctx.lat, ctx.K, ctx.alpha, ctx.every, ctx.ckpts = lat, K, alpha, every, ckpts
        return UK

    @staticmethod
    def backward(ctx, gUK):
        lat, K, alpha, every = ctx.lat, ctx.K, ctx.alpha, ctx.every
        g = gUK.contiguous()
        nseg = (K + every - 1) // every
        for si in reversed(range(nseg)):
            a, b = si * every, min(K, (si + 1) * every)
            states = [ctx.ckpts[si]]
            lat.load_links(states[0])
            for _ in range(b - a - 1):
                lat.fix(alpha, 0.0, 1)
                states.append(lat.save_links())
            for k in reversed(range(b - a)):
                lat.load_links(states[k])
                g = lat.step_bwd(g, alpha)
        return g, None, None, None, None


class GluonPmin(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, lat):
        U = U.detach().contiguous()
        lat.set_links(U)
        D, _ = lat.gluon_pmin()
        ctx.lat, ctx.U = lat, U
        return torch.tensor(D, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, gD):
        ctx.lat.set_links(ctx.U)
        return ctx.lat.gluon_pmin_bwd(float(gD), device=ctx.U.device), None


def gluon_after_fixing(U0, dims, K: int = 50, alpha: float = 0.08, every: int = 10, lat=None):
    """D(p_min) of the links after K gauge-fixing steps, differentiable in U0."""
    own = lat is None
    if own:
        lat = lgf.Lattice(dims, track_gauge=False)
    UK = GaugeFixUnroll.apply(U0, lat, K, alpha, every)
    D = GluonPmin.apply(UK, lat)
    return D, lat
