"""torch.autograd.Function around pic_adjoint.

PolarizationLoss gives the loss of pic_loss_t (the energy-weighted Eq. (4)
polarization of one species above an energy cut) after a run, as a function
of the laser amplitude a0 and of that species' particle weights and initial
spins; its backward pass returns the gradients pic_adjoint computes on the
GPU.  Parametrizations of those inputs (a density profile from which the
weights follow, a spin angle) are ordinary torch operations in front of it,
so torch chains the gradient to their parameters.
"""
from __future__ import annotations

import numpy as np

from . import Simulation

__all__ = ["LossRun", "PolarizationLoss", "forward_loss"]


class LossRun:
    """What one evaluation needs besides (a0, weights, spins): a factory
    a0 -> pic_config_t, every species' particles (dicts of arrays; float64
    values are uploaded exactly with precision 64), the loss species, the run
    length, the checkpoint interval, the pic_loss_t fields, and whether the
    immobile ions neutralize the initial plasma."""

    def __init__(self, make_config, particles, species, nsteps, checkpoint_every, loss, neutralize=False,
                 stream=None):
        self.make_config = make_config
        self.particles = particles
        self.species = species
        self.nsteps = nsteps
        self.checkpoint_every = checkpoint_every
        self.loss = dict(loss)
        self.neutralize = neutralize
        self.stream = stream

    def start(self, a0, weights, spins):
        """A fresh context holding the initial state with these inputs."""
        sim = Simulation(self.make_config(float(a0)), stream=self.stream)
        for s, d in enumerate(self.particles):
            d = dict(d)
            if s == self.species:
                d["w"] = np.asarray(weights, dtype=np.float64)
                sp = np.asarray(spins, dtype=np.float64)
                d["sx"], d["sy"], d["sz"] = sp[:, 0], sp[:, 1], sp[:, 2]
            sim.set_particles_f64(s, d)
        if self.neutralize:
            sim.capture_background()
        return sim


def forward_loss(run: LossRun, a0, weights, spins):
    """The loss alone, through the same forward steps pic_adjoint takes
    (no tile sorts; the fused kernel in FP32, the split kernels in FP64)."""
    with run.start(a0, weights, spins) as sim:
        for _ in range(run.nsteps):
            adjoint_forward_step(sim)
        return sim.loss(species=run.species, **run.loss)


def adjoint_forward_step(sim):
    """One forward step the way pic_adjoint takes it."""
    if sim.cfg.precision == 64:
        sim.gather_push_spin()
        sim.deposit()
    else:
        sim.push_deposit()
    sim.field_update()


def _slot_order(ids, slot_ids):
    sorter = np.argsort(ids)
    return sorter[np.searchsorted(ids, slot_ids, sorter=sorter)]


def _function():
    import torch

    class _PolarizationLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, a0, weights, spins, run):
            w = weights.detach().cpu().double().numpy()
            sp = spins.detach().cpu().double().numpy()
            with run.start(a0.item(), w, sp) as sim:
                value, dla0 = sim.adjoint(run.nsteps, run.checkpoint_every, species=run.species, **run.loss)
                g = sim.adjoint_particle_grads(run.species)
            idx = _slot_order(np.asarray(run.particles[run.species]["id"]), g["id"])
            gw = np.zeros(len(w))
            gs = np.zeros((len(w), 3))
            gw[idx] = g["w"]
            gs[idx, 0], gs[idx, 1], gs[idx, 2] = g["sx"], g["sy"], g["sz"]
            ctx.save_for_backward(torch.tensor(dla0, dtype=torch.float64), torch.from_numpy(gw),
                                  torch.from_numpy(gs))
            ctx.devices = (a0.device, weights.device, spins.device)   # each gradient goes back there
            return torch.tensor(value, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gout):
            dla0, gw, gs = ctx.saved_tensors
            gout = gout.cpu()
            d0, dw, ds = ctx.devices
            return (gout * dla0).to(d0), (gout * gw).to(dw), (gout * gs).to(ds), None

    return _PolarizationLoss


_FN = None


def PolarizationLoss(a0, weights, spins, run: LossRun):
    """L(a0, weights, spins) of `run`, differentiable (torch float64 tensors)."""
    global _FN
    if _FN is None:
        _FN = _function()
    return _FN.apply(a0, weights, spins, run)
