"""Gradient of a velocity loss with respect to the force field, for the oracle.

Test infrastructure (see the package docstring). The paper has no adjoint; the oracle's
gradient is the definition itself, obtained by reverse-mode automatic differentiation
(torch.autograd) through the oracle's own forward steps, from a fixed initial state.
Pinned by central finite differences of the same forward (tests/test_oracle_adjoint.py).
"""
import torch

from .lattice import DT
from .solver import OracleSim


def velocity_loss(sim_args, s0, F, target, steps, sim_kwargs=None):
    """L = mean over cells of |u_T - target|^2 after `steps` steps from s0 under force field F."""
    sim = OracleSim(*sim_args, **(sim_kwargs or {}))
    sim.F = F
    sim.s = s0
    for _ in range(steps):
        sim.step(1)
    _, u = sim.moments()
    return ((u - target) ** 2).sum(0).mean()


def loss_and_grad(sim_args, s0, F, target, steps, sim_kwargs=None):
    """(L, dL/dF) by reverse-mode automatic differentiation through the oracle's steps."""
    Fp = torch.as_tensor(F, dtype=DT).detach().clone().requires_grad_(True)
    L = velocity_loss(sim_args, torch.as_tensor(s0, dtype=DT).detach(), Fp, torch.as_tensor(target, dtype=DT),
                      steps, sim_kwargs)
    L.backward()
    return float(L.detach()), Fp.grad.detach()
