"""Smagorinsky eddy viscosity from the local non-equilibrium stress, with van Driest damping.

Test infrastructure (see the package docstring).

Paper silent on the formula: the paper asks that sub-grid models be inertial-frame invariant
(Sec. 1) and routes turbulence models through the filtered kinetic equation (Sec. 14). The
reading used here takes the non-equilibrium stress from second-order CENTRAL moments,
    Pi^neq_ij = kappa_ij - c_s^2 rho delta_ij,
which carry no F.u terms (second-order kappa of f equals that of fbar, Sec. 8), so the
eddy viscosity does not depend on the frame. With Delta = 1 and
    S_ij = -Pi^neq_ij / (2 rho c_s^2 tau_eff),   |S| = sqrt(2 S:S),
    tau_eff = tau_0 + 3 nu_t,   nu_t = (C_s Delta)^2 |S|,
tau_eff solves tau_eff^2 - tau_0 tau_eff - 9 C_s^2 Q / (sqrt(2) rho) = 0 with Q = sqrt(Pi:Pi):
    tau_eff = ( tau_0 + sqrt(tau_0^2 + 18 sqrt(2) C_s^2 Q / rho) ) / 2.
van Driest (paper silent): C_s -> C_s (1 - exp(-y+/A+)), y+ = y u_tau / nu_0, y the distance
to the nearest half-way wall.
"""
import math

import torch

from .lattice import CS2


def nonequilibrium_stress(kap, rho, lat):
    """Pi^neq as a dict {(i, j): tensor} over the d x d tensor (both orders of off-diagonals)."""
    idx = {a: k for k, a in enumerate(lat.monomials)}
    out = {}
    for i in range(lat.d):
        for j in range(lat.d):
            a = [0, 0, 0]
            a[i] += 1
            a[j] += 1
            v = kap[idx[tuple(a)]]
            if i == j:
                v = v - CS2 * rho
            out[(i, j)] = v
    return out


def stress_norm(Pi):
    """|Pi| = (Pi : Pi)^(1/2) of the symmetric non-equilibrium stress (reading of the Smagorinsky closure)."""
    return torch.sqrt(sum(v * v for v in Pi.values()))


def tau_effective(tau0, cs, Pi, rho):
    """Closed-form root of tau^2 - tau0 tau - 9 C_s^2 Q / (sqrt(2) rho) = 0."""
    Q = stress_norm(Pi)
    return 0.5 * (tau0 + torch.sqrt(tau0 * tau0 + 18.0 * math.sqrt(2.0) * cs * cs * Q / rho))


def tau_effective_fixed_point(tau0, cs, Pi, rho, iters=200):
    """The same quantity by iterating tau <- tau0 + 3 C_s^2 |S(tau)| (used as a pin)."""
    Q = stress_norm(Pi)
    tau = torch.full_like(rho, tau0)
    for _ in range(iters):
        Smag = math.sqrt(2.0) * Q / (2.0 * rho * CS2 * tau)
        tau = tau0 + 3.0 * cs * cs * Smag
    return tau


def van_driest_cs(cs, ny, nz, nx, aplus, utau_over_nu, wall_axis=1):
    """Per-cell damped constant C_s (1 - exp(-y+/A+)) for half-way walls on both ends of an axis."""
    n = (nx, ny, nz)[wall_axis]
    j = torch.arange(n, dtype=torch.float64)
    y = torch.minimum(j + 0.5, n - 0.5 - j)
    damp = 1.0 - torch.exp(-(y * utau_over_nu) / aplus)
    c = cs * damp
    if wall_axis == 1:
        return c.view(1, n, 1).expand(nz, n, nx).clone()
    if wall_axis == 2:
        return c.view(n, 1, 1).expand(n, ny, nx).clone()
    return c.view(1, 1, n).expand(nz, ny, n).clone()
