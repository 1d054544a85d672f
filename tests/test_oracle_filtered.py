"""Oracle pins for turbulence as forcing (Sec. 14; the closure itself is a stated reading)."""
import math

import torch

from oracle import filtered as FL
from oracle.solver import OracleSim
from oracle.collision import Params
from paper_1202_6074_gb300 import workloads as W

DT = torch.float64


def test_shear_mode_matches_discrete_closed_form():
    n, A, cs = 24, 0.03, 0.17
    k = 2 * math.pi * 3 / n
    y = torch.arange(n, dtype=DT).view(1, n, 1).expand(1, n, 5)
    u = torch.zeros(3, 1, n, 5, dtype=DT)
    u[0] = A * torch.sin(k * y)
    a = FL.turbulence_acceleration(u, cs, 3)
    ref = FL.discrete_shear_mode(A, k, cs, y)
    assert torch.allclose(a[0], ref, atol=1e-18, rtol=1e-12)
    assert a[1].abs().max().item() < 1e-18 and a[2].abs().max().item() < 1e-18


def test_acceleration_is_galilean_invariant_and_conserves_momentum():
    n = 10
    _, u = W.random_solenoidal(n, n, n, seed=9, u_rms=0.03)
    u = torch.tensor(u)
    a0 = FL.turbulence_acceleration(u, 0.12, 3)
    shifted = u + torch.tensor([0.05, -0.03, 0.02], dtype=DT).view(3, 1, 1, 1)
    a1 = FL.turbulence_acceleration(shifted, 0.12, 3)
    assert (a0 - a1).abs().max().item() < 1e-17
    # a divergence on a periodic box: no net momentum is injected
    assert a0.sum(dim=(1, 2, 3)).abs().max().item() < 1e-17
    assert a0.abs().max().item() > 1e-7


def test_eddy_stress_is_traceless_for_solenoidal_rigid_and_zero_for_uniform_flow():
    n = 8
    u = torch.zeros(3, n, n, n, dtype=DT) + torch.tensor([0.1, 0.2, -0.1], dtype=DT).view(3, 1, 1, 1)
    T = FL.eddy_stress(u, 0.1, 3)
    assert all(v.abs().max().item() == 0 for v in T.values())


def test_filtered_step_runs_and_conserves_mass():
    n = 8
    rho, u = W.random_solenoidal(n, n, n, seed=7, u_rms=0.02)
    sim = OracleSim("D3Q27", n, n, n, Params(tau=0.52, attractor="factorized", reduced_compressibility=True))
    sim.init(torch.tensor(rho), torch.tensor(u))
    m0 = sim.reduce()
    sim.step_filtered(5, 0.15)
    m1 = sim.reduce()
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-14
