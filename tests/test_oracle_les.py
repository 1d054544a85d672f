"""Oracle pins for the eddy-viscosity reading (paper silent; frame invariance required by Sec. 1)."""
import math

import torch

from oracle import lattice as L, moments as M, collision as C, les

DT = torch.float64


def test_closed_form_matches_fixed_point():
    g = torch.Generator().manual_seed(30)
    n = 64
    Pi = {(i, j): 1e-3 * torch.randn(n, generator=g, dtype=DT) for i in range(3) for j in range(3)}
    for i in range(3):
        for j in range(i):
            Pi[(i, j)] = Pi[(j, i)]
    rho = 1 + 0.05 * torch.randn(n, generator=g, dtype=DT)
    for tau0, cs in [(0.5005, 0.1), (0.51067, 0.17), (0.8, 0.3)]:
        a = les.tau_effective(tau0, cs, Pi, rho)
        b = les.tau_effective_fixed_point(tau0, cs, Pi, rho)
        assert torch.allclose(a, b, atol=0, rtol=1e-13)


def test_uniform_shear_gives_smagorinsky_viscosity():
    """A cell whose non-equilibrium stress is that of a steady shear S_xy = s at tau_eff gives
    nu_t = C_s^2 |S| with |S| = sqrt(2 S:S) = sqrt(2) * sqrt(2 s^2) = 2|s|."""
    lat = L.D3Q27
    tau0, cs, s, rho = 0.52, 0.15, 2e-3, 1.0
    # nu_t from the defining relation: tau_eff = tau0 + 3 cs^2 * 2|s| ... with S fixed
    nu_t = cs * cs * 2 * abs(s)
    tau_eff = tau0 + 3 * nu_t
    Pi_xy = -2 * rho * (1 / 3) * tau_eff * s
    # build populations: Maxwellian plus a pure xy non-equilibrium part through the inverse
    r = torch.tensor([rho], dtype=DT)
    u = torch.zeros(3, 1, dtype=DT)
    kM = C.maxwell_central(r, lat)
    idx = {a: k for k, a in enumerate(lat.monomials)}
    k = kM.clone()
    k[idx[(1, 1, 0)]] = Pi_xy
    f = M.central_to_populations(k, u, lat)
    _, kap = C.source_central(M.central_moments(f, u, lat), r, torch.zeros(3, 1, dtype=DT), lat)
    Pi = les.nonequilibrium_stress(kap, r, lat)
    got = les.tau_effective(tau0, cs, Pi, r).item()
    assert abs(got - tau_eff) < 1e-14
    assert abs((got - tau0) / 3 - nu_t) < 1e-15


def test_eddy_viscosity_is_frame_invariant():
    """Shifting every population's velocity frame (same central moments about u + U) leaves
    tau_eff unchanged: Pi^neq is built from central moments."""
    lat = L.D3Q27
    g = torch.Generator().manual_seed(31)
    n = 32
    r = 1 + 0.02 * torch.randn(n, generator=g, dtype=DT)
    u = 0.05 * torch.randn(3, n, generator=g, dtype=DT)
    k = C.maxwell_central(r, lat) + 1e-3 * torch.randn(27, n, generator=g, dtype=DT)
    k[0] = r
    k[1:4] = 0
    F = torch.zeros(3, n, dtype=DT)
    out = []
    for U in (torch.zeros(3, 1, dtype=DT), torch.tensor([[0.05], [0.03], [0.0]], dtype=DT)):
        f = M.central_to_populations(k, u + U, lat)
        rho, uu = C.hydrodynamics(f, F, lat)
        _, kap = C.source_central(M.central_moments(f, uu, lat), rho, F, lat)
        out.append(les.tau_effective(0.5005, 0.1, les.nonequilibrium_stress(kap, rho, lat), rho))
    assert torch.allclose(out[0], out[1], atol=0, rtol=1e-12)


def test_van_driest_profile():
    c = les.van_driest_cs(0.1, 8, 1, 1, 26.0, 10.0)
    y = torch.tensor([0.5, 1.5, 2.5, 3.5, 3.5, 2.5, 1.5, 0.5], dtype=DT)
    ref = 0.1 * (1 - torch.exp(-y * 10.0 / 26.0))
    assert torch.allclose(c[0, :, 0], ref, atol=0, rtol=1e-15)
    assert math.isclose(c[0, 0, 0].item(), c[0, 7, 0].item())


def test_van_driest_damping_properties():
    """Properties the damping must have whatever its formula: symmetric about the channel centre,
    increasing from the wall to the centre, below the undamped constant everywhere, close to it
    far from the walls, and vanishing as the wall distance in wall units goes to zero."""
    ny = 16
    c = les.van_driest_cs(0.1, ny, 1, 1, 26.0, 3.0)[0, :, 0]
    assert torch.equal(c, c.flip(0))
    half = c[: ny // 2]
    assert bool((half[1:] > half[:-1]).all())
    assert bool((c < 0.1).all())
    far = les.van_driest_cs(0.1, ny, 1, 1, 26.0, 1e3)[0, :, 0]
    assert bool(((0.1 - far) < 1e-6).all())
    near = les.van_driest_cs(0.1, ny, 1, 1, 26.0, 1e-6)[0, :, 0]
    assert bool((near < 1e-7).all())
