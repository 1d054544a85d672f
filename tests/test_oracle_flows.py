"""Oracle pins from closed-form flows and exact invariants of the whole step (stream + collide).

* body-force Poiseuille: steady parabola u = F eta (H - eta) / (2 rho nu), exact with
  half-way walls when (1/omega_nu - 1/2)(1/omega_3 - 1/2) = 3/16 (nu = c_s^2 (1/omega_nu - 1/2),
  Sec. 10), and the same profile shifted by U with walls and fluid moving at U (Galilean
  invariance of the forced flow, the paper's central claim);
* Couette flow: exact linear profile (moving-wall bounce-back);
* 2D Taylor-Green decay rate gives nu = c_s^2 (1/omega_nu - 1/2);
* D3Q27 on a one-cell periodic z reproduces the paper's D2Q9 scheme;
* mass conservation and momentum growth equal to the applied force;
* the initial state returns the requested fields.
"""
import math

import numpy as np
import pytest
import torch

from oracle.solver import OracleSim
from oracle.collision import Params
from paper_1202_6074_gb300 import workloads as W

DT = torch.float64


def _walls(lower=(0.0, 0.0, 0.0), upper=(0.0, 0.0, 0.0)):
    z = [0.0, 0.0, 0.0]
    return [[z, z], [list(lower), list(upper)], [z, z]]


@pytest.mark.parametrize("U", [0.0, 0.05])
def test_poiseuille_exact_with_magic_parameter(U):
    ny, F, tau = 8, 1e-6, 0.8
    nu = (tau - 0.5) / 3
    w3 = 1.0 / (0.5 + (3.0 / 16.0) / (tau - 0.5))      # Lambda = 3/16
    sim = OracleSim("D2Q9", 1, ny, 1, Params(tau=tau, omega3=w3), bc=("periodic", "bounceback", "periodic"),
                    wall_velocity=_walls((U, 0, 0), (U, 0, 0)))
    sim.set_force((F, 0, 0))
    rho, u = W.rest(1, ny, 1, background=(U, 0, 0))
    sim.init(torch.tensor(rho), torch.tensor(u))
    sim.step(1600)
    r, uu = sim.moments()
    eta = np.arange(ny) + 0.5
    ref = F / (2 * nu) * eta * (ny - eta)
    err = np.abs(uu[0, 0, :, 0].numpy() - U - ref).max() / ref.max()
    assert err < 1e-9
    assert (r - 1).abs().max().item() < 1e-13
    assert uu[1].abs().max().item() < 1e-15


def test_poiseuille_default_rates_wall_error_is_small():
    ny, F, tau = 8, 1e-6, 0.8
    nu = (tau - 0.5) / 3
    sim = OracleSim("D2Q9", 1, ny, 1, Params(tau=tau), bc=("periodic", "bounceback", "periodic"))
    sim.set_force((F, 0, 0))
    sim.init()
    sim.step(1600)
    _, uu = sim.moments()
    eta = np.arange(ny) + 0.5
    ref = F / (2 * nu) * eta * (ny - eta)
    err = np.abs(uu[0, 0, :, 0].numpy() - ref).max() / ref.max()
    assert 1e-4 < err < 1e-2


def test_couette_exact():
    ny, U = 8, 0.01
    sim = OracleSim("D2Q9", 1, ny, 1, Params(tau=0.8), bc=("periodic", "bounceback", "periodic"),
                    wall_velocity=_walls((0, 0, 0), (U, 0, 0)))
    sim.init()
    sim.step(1600)
    _, uu = sim.moments()
    ref = U * (np.arange(ny) + 0.5) / ny
    assert np.abs(uu[0, 0, :, 0].numpy() - ref).max() / U < 1e-9


def test_taylor_green_decay_rate_gives_viscosity():
    N, tau, u0 = 32, 0.8, 0.01
    nu = (tau - 0.5) / 3
    rho, u = W.taylor_green(N, N, 1, u0=u0, two_d=True)
    sim = OracleSim("D2Q9", N, N, 1, Params(tau=tau))
    sim.init(torch.tensor(rho), torch.tensor(u))
    sim.step(20)
    _, u1 = sim.moments()
    sim.step(100)
    _, u2 = sim.moments()
    k = 2 * math.pi / N
    nu_fit = -math.log(float((u2 ** 2).sum()) / float((u1 ** 2).sum())) / (4 * k * k * 100)
    assert abs(nu_fit / nu - 1) < 1e-2


@pytest.mark.parametrize("attractor,reduced", [("maxwell", False), ("factorized", False), ("factorized", True),
                                               ("maxwell", True)])
def test_d3q27_one_cell_thick_reproduces_d2q9(attractor, reduced):
    """The 3D reading of the basis, attractors, sources and rates reduces to the paper's D2Q9:
    on a one-cell periodic z with u_z = F_z = 0 the z-marginal of the D3Q27 state is the D2Q9
    state. This holds for the factorized attractor (Sec. 13) too, which pins the 3D factorized
    rules of the moments without a z exponent to the D2Q9 ones, and for the reduced-
    compressibility form (Sec. 12)."""
    N = 12
    rho, u = W.taylor_green(N, N, 1, u0=0.03, two_d=True)
    p = Params(tau=0.7, omega3=1.2, omega4=0.9, attractor=attractor, reduced_compressibility=reduced, rho0=1.01)
    a = OracleSim("D2Q9", N, N, 1, p, bc=("periodic", "bounceback", "periodic"),
                  wall_velocity=_walls((0.01, 0, 0), (-0.02, 0, 0)))
    b = OracleSim("D3Q27", N, N, 1, p, bc=("periodic", "bounceback", "periodic"),
                  wall_velocity=_walls((0.01, 0, 0), (-0.02, 0, 0)))
    for s in (a, b):
        s.set_force((2e-5, -1e-5, 0.0))
        s.init(torch.tensor(rho), torch.tensor(u))
        s.step(20)
    ra, ua = a.moments()
    rb, ub = b.moments()
    assert (ra - rb).abs().max().item() < 1e-14
    assert (ua - ub).abs().max().item() < 1e-14
    # populations: sum over e_z of the D3Q27 state equals the D2Q9 state
    lat3, lat2 = b.lat, a.lat
    for i in range(9):
        ex, ey, _ = (int(v) for v in lat2.e[i])
        js = [j for j in range(27) if int(lat3.e[j, 0]) == ex and int(lat3.e[j, 1]) == ey]
        assert (b.s[js].sum(0) - a.s[i]).abs().max().item() < 1e-14


def test_mass_conserved_and_momentum_gains_force():
    N = 8
    rho, u = W.random_solenoidal(N, N, N, seed=7, u_rms=0.02)
    F = W.gaussian_force(N, N, N, seed=8, std=1e-4)
    sim = OracleSim("D3Q27", N, N, N, Params(tau=0.55, cs_smag=0.1))
    sim.set_force(field=torch.tensor(F))
    sim.init(torch.tensor(rho), torch.tensor(u))
    m0 = sim.reduce()
    sim.step(10)
    m1 = sim.reduce()
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-14
    for d in range(3):
        assert abs((m1[1 + d] - m0[1 + d]) - 10 * F[d].sum()) < 1e-13


def test_mass_conserved_with_walls():
    sim = OracleSim("D3Q27", 6, 8, 5, Params(tau=0.6, cs_smag=0.1), bc=("periodic", "bounceback", "periodic"),
                    wall_velocity=_walls((0.02, 0, 0.01), (-0.03, 0, 0)), van_driest=(26.0, 5.0))
    rho, u, F = W.channel(6, 8, 5, u_tau=0.01)
    sim.set_force(field=torch.tensor(F))
    sim.init(torch.tensor(rho), torch.tensor(u))
    m0 = sim.reduce()[0]
    sim.step(10)
    assert abs(sim.reduce()[0] - m0) / m0 < 1e-14


@pytest.mark.parametrize("bc", [("periodic",) * 3, ("periodic", "bounceback", "periodic"),
                                ("bounceback", "bounceback", "bounceback")])
def test_initial_state_returns_requested_fields(bc):
    N = (5, 6, 4)
    rho, u = W.taylor_green(*N, u0=0.04, background=(0.01, 0.0, -0.02))
    uw = [[[0.01, 0, 0], [0, 0.02, 0]], [[0.03, 0, 0], [0, 0, 0.01]], [[0, 0, 0], [0.02, 0.01, 0]]]
    sim = OracleSim("D3Q27", *N, Params(tau=0.7), bc=bc, wall_velocity=uw)
    sim.set_force((1e-4, 2e-4, -1e-4))
    sim.init(torch.tensor(rho), torch.tensor(u))
    r, uu = sim.moments()
    assert (r - torch.tensor(rho)).abs().max().item() < 1e-15
    assert (uu - torch.tensor(u)).abs().max().item() < 1e-15


def test_galilean_invariance_of_taylor_green_decay():
    """Kinetic energy in the frame of the mean flow decays alike with and without U; the residual
    is the velocity set's own cubic defect (Sec. 1) and shrinks with resolution."""
    N = 16
    E = []
    for U in ((0, 0, 0), (0.05, 0.03, 0.0)):
        rho, u = W.taylor_green(N, N, N, u0=0.05, background=U)
        sim = OracleSim("D3Q27", N, N, N, Params(tau=0.6))
        sim.init(torch.tensor(rho), torch.tensor(u))
        out = []
        for _ in range(3):
            sim.step(10)
            m = sim.reduce()
            out.append(m[4] - 0.5 * (m[1] ** 2 + m[2] ** 2 + m[3] ** 2) / m[0])
        E.append(np.array(out))
    E0 = E[0][0]
    assert np.abs(E[0] - E[1]).max() / E0 < 4e-3


@pytest.mark.parametrize("plane", ["xz", "yz"])
@pytest.mark.parametrize("attractor", ["maxwell", "factorized"])
def test_d3q27_one_cell_thick_in_other_planes_reproduces_d2q9(plane, attractor):
    """The same reduction with the flow in the x-z or y-z plane (one cell along the third axis):
    the D2Q9 axes (x, y) map to (x, z) or (y, z). With the factorized attractor this pins the
    3D rules of the (a, 0, c) and (0, b, c) moment families to the D2Q9 form as well."""
    N = 10
    rho, u = W.taylor_green(N, N, 1, u0=0.03, background=(0.01, -0.02, 0.0), two_d=True)
    F = W.gaussian_force(N, N, 1, seed=5, std=1e-4)
    p = Params(tau=0.68, omega3=1.15, omega4=0.85, attractor=attractor)
    a = OracleSim("D2Q9", N, N, 1, p)
    a.set_force(field=torch.tensor(np.stack([F[0], F[1], 0 * F[2]])))
    a.init(torch.tensor(rho), torch.tensor(u))
    # 2D arrays are [1, y, x]; the D3Q27 box is [z, 1, x] (plane xz) or [z, y, 1] (plane yz)
    if plane == "xz":
        shape3, axes = (N, 1, N), (0, 2)
        to3 = lambda f: f[0][:, None, :]
    else:
        shape3, axes = (N, N, 1), (1, 2)
        to3 = lambda f: f[0][:, :, None]
    nz3, ny3, nx3 = shape3
    u3 = np.zeros((3,) + shape3)
    F3 = np.zeros((3,) + shape3)
    for k, d in enumerate(axes):
        u3[d] = to3(u[k])
        F3[d] = to3(F[k])
    b = OracleSim("D3Q27", nx3, ny3, nz3, p)
    b.set_force(field=torch.tensor(F3))
    b.init(torch.tensor(to3(rho)), torch.tensor(u3))
    a.step(15)
    b.step(15)
    ra, ua = a.moments()
    rb, ub = b.moments()
    assert (torch.tensor(to3(ra.numpy())) - rb).abs().max().item() < 1e-14
    for k, d in enumerate(axes):
        assert (torch.tensor(to3(ua[k].numpy())) - ub[d]).abs().max().item() < 1e-14
