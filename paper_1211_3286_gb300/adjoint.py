"""Misfit gradients through the fused step: the librlb adjoint (rlb_adjoint)
behind a torch.autograd.Function.

The loss is J = w_P sum (P - P*)^2 + w_u sum |u - u*|^2 of the fields after
`nsteps` steps started from the equilibrium of (e0, u0, n0).  Gradients with
respect to tau_v, tau_e, tau_eps and the initial energy field e0 come from the
hand-written reverse-mode kernels of librlb with sqrt(T) checkpointing; PyTorch
only carries tensors and the autograd bookkeeping.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L
from .lattice import Lattice, _after_producer, _f64, _ptr


def misfit_gradient(lat: Lattice, nsteps, target_P, target_ux, target_uy, target_uz, w_P=1.0, w_u=1.0,
                    checkpoint_every=0):
    """Run rlb_adjoint on a lattice whose current state is the initial state.
    Returns (loss, dtau tensor (3,), de0 tensor shaped like the lattice, on the target's device)."""
    ts = [_f64(t) for t in (target_P, target_ux, target_uy, target_uz)]
    where = L.RLB_DEVICE if ts[0].is_cuda else L.RLB_HOST
    de0 = torch.empty(lat.shape, dtype=torch.float64, device=ts[0].device)
    _after_producer(lat.stream, ts + [de0])
    loss, dtau = L.rlb_adjoint(lat.handle, nsteps, checkpoint_every, *[_ptr(t) for t in ts], w_P, w_u, where,
                               _ptr(de0))
    return loss, torch.tensor(dtau, dtype=torch.float64), de0


class ShockTubeMisfit(torch.autograd.Function):
    """loss = J(tau_v, tau_e, tau_eps, e0); backward returns the adjoint gradients.

    forward(tau_v, tau_e, tau_eps, e0, u0x, u0y, u0z, n0, target_P, target_ux, target_uy,
            target_uz, nsteps, spec) where spec is a dict with keys collision, tau_f (or None
    for tau_f = tau_v), bc, w_P, w_u, checkpoint_every.  The tau arguments are 0-d tensors,
    e0 a (nz, ny, nx) FP64 tensor."""

    @staticmethod
    def forward(ctx, tau_v, tau_e, tau_eps, e0, u0x, u0y, u0z, n0, target_P, target_ux, target_uy, target_uz,
                nsteps, spec):
        tv, te, tp = float(tau_v), float(tau_e), float(tau_eps)
        tf = spec.get("tau_f") or tv
        lat = Lattice(tuple(e0.shape), collision=spec.get("collision", "mrt"), tau_f=tf, tau_v=tv, tau_e=te,
                      tau_eps=tp, tau_q=0.0, bc=spec.get("bc", ("zero_gradient", "periodic", "periodic")))
        dev = e0.device
        lat.set_fields(e0.detach(), u0x, u0y, u0z, n0)
        loss, dtau, de0 = misfit_gradient(lat, int(nsteps), target_P.to(dev), target_ux.to(dev), target_uy.to(dev),
                                          target_uz.to(dev), spec.get("w_P", 1.0), spec.get("w_u", 1.0),
                                          spec.get("checkpoint_every", 0))
        lat.close()
        ctx.save_for_backward(dtau.to(dev), de0)
        return torch.tensor(loss, dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, gout):
        dtau, de0 = ctx.saved_tensors
        return (gout * dtau[0], gout * dtau[1], gout * dtau[2], gout * de0,
                None, None, None, None, None, None, None, None, None, None)


def shock_tube_misfit(tau_v, tau_e, tau_eps, e0, u0, n0, targets, nsteps, **spec):
    """Convenience call of ShockTubeMisfit.apply; u0 and targets are (x, y, z) / (P, ux, uy, uz) tuples."""
    return ShockTubeMisfit.apply(tau_v, tau_e, tau_eps, e0, u0[0], u0[1], u0[2], n0, targets[0], targets[1],
                                 targets[2], targets[3], nsteps, spec)
