"""Oracle pins: velocity set, orthogonal basis, exact inverse, equilibrium (Secs. 2, 4, 7, 9)."""
import os

import pytest
import torch

from oracle import lattice as L, moments as M, collision as C

DT = torch.float64


def _read_basis(golden_dir):
    K, D = [], None
    with open(os.path.join(golden_dir, "d2q9_basis.txt")) as fh:
        for line in fh:
            if line.startswith("K "):
                K.append([int(v) for v in line.split()[1:]])
            elif line.startswith("D "):
                D = [int(v) for v in line.split()[1:]]
    return torch.tensor(K, dtype=DT), torch.tensor(D, dtype=DT)


def _read_monomial_vectors(golden_dir):
    out = {}
    with open(os.path.join(golden_dir, "d2q9_monomial_vectors.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, *vals = line.split()
            out[name] = torch.tensor([int(v) for v in vals], dtype=DT)
    return out


def test_d2q9_velocities_match_printed_vectors(golden_dir):
    v = _read_monomial_vectors(golden_dir)
    e = L.D2Q9.e.to(DT)
    assert torch.equal(e[:, 0], v["ex"])
    assert torch.equal(e[:, 1], v["ey"])
    assert torch.equal(e[:, 0] ** 2 + e[:, 1] ** 2, v["ex2+ey2"])
    assert torch.equal(e[:, 0] ** 2 * e[:, 1] ** 2, v["ex2ey2"])
    assert torch.equal(e[:, 0] ** 2 * e[:, 1], v["ex2ey"])
    assert torch.equal(e[:, 0] * e[:, 1] ** 2, v["exey2"])


def test_d2q9_basis_equals_printed_matrix(golden_dir):
    K, _ = _read_basis(golden_dir)
    assert torch.equal(L.D2Q9.K, K)


def test_d2q9_orthogonality_printed_D(golden_dir):
    K, D = _read_basis(golden_dir)
    KtK = L.D2Q9.K.T @ L.D2Q9.K
    assert torch.equal(KtK, torch.diag(D))


def test_d3q27_basis_is_orthogonal_with_product_norms():
    lat = L.D3Q27
    KtK = lat.K.T @ lat.K
    D = torch.diag(KtK)
    assert torch.equal(KtK, torch.diag(D))
    norm1 = {0: 3.0, 1: 2.0, 2: 6.0}
    for b, a in enumerate(lat.monomials):
        assert D[b].item() == norm1[a[0]] * norm1[a[1]] * norm1[a[2]]


def test_d3q27_basis_reduces_to_d2q9_on_the_plane():
    # K_(b0,b1,0) restricted to ez = 0 is, up to the combinations K3/K4 of Sec. 2, the D2Q9 basis
    lat3 = L.D3Q27
    plane = [i for i in range(27) if int(lat3.e[i, 2]) == 0]
    idx = {tuple(int(x) for x in lat3.e[i]): i for i in plane}
    order = [idx[tuple(int(x) for x in L.D2Q9.e[i])] for i in range(9)]
    m3 = {a: k for k, a in enumerate(lat3.monomials)}
    K2 = L.D2Q9.K
    assert torch.equal(lat3.K[order, m3[(1, 0, 0)]], K2[:, 1])
    assert torch.equal(lat3.K[order, m3[(2, 0, 0)]] + lat3.K[order, m3[(0, 2, 0)]], K2[:, 3])
    assert torch.equal((lat3.K[order, m3[(2, 0, 0)]] - lat3.K[order, m3[(0, 2, 0)]]) / 3, K2[:, 4])
    assert torch.equal(-lat3.K[order, m3[(2, 1, 0)]], K2[:, 6])
    assert torch.equal(lat3.K[order, m3[(2, 2, 0)]], K2[:, 8])


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27"])
def test_weights_and_opposites(name):
    lat = L.get(name)
    assert abs(lat.w.sum().item() - 1.0) < 1e-15
    for i in range(lat.Q):
        assert torch.equal(lat.e[lat.opp[i]], -lat.e[i])
    # second moment of the weights is c_s^2 = 1/3 (Sec. 4)
    assert abs((lat.w * lat.e[:, 0].to(DT) ** 2).sum().item() - 1.0 / 3.0) < 1e-15


def _random_state(lat, n, seed, force=True):
    g = torch.Generator().manual_seed(seed)
    rho = 1 + 0.05 * torch.randn(n, generator=g, dtype=DT)
    u = 0.1 * torch.randn(3, n, generator=g, dtype=DT)
    F = 1e-2 * torch.randn(3, n, generator=g, dtype=DT) if force else torch.zeros(3, n, dtype=DT)
    if lat.d == 2:
        u[2] = 0
        F[2] = 0
    feq = C.equilibrium(rho, u, torch.zeros_like(F), lat)
    fb = feq * (1 + 0.05 * torch.randn(feq.shape, generator=g, dtype=DT))
    return fb, F


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27"])
def test_transform_round_trip(name):
    lat = L.get(name)
    fb, F = _random_state(lat, 64, 1)
    _, u = C.hydrodynamics(fb, F, lat)
    k = M.central_moments(fb, u, lat)
    back = M.central_to_populations(k, u, lat)
    assert (back - fb).abs().max().item() < 1e-15


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27"])
def test_central_at_zero_velocity_equals_raw(name):
    lat = L.get(name)
    fb, _ = _random_state(lat, 16, 2)
    z = torch.zeros(3, 16, dtype=DT)
    assert torch.allclose(M.central_moments(fb, z, lat), M.raw_moments(fb, lat), atol=0, rtol=1e-15)


def test_d2q9_central_from_raw_printed_closed_forms():
    """Eqs. kxxtransform - kxxytransform against the explicit central-moment sums."""
    lat = L.D2Q9
    fb, F = _random_state(lat, 64, 3)
    rho, u = C.hydrodynamics(fb, F, lat)
    ux, uy, Fx, Fy = u[0], u[1], F[0], F[1]
    r = M.raw_moments(fb, lat)
    kxx_r, kyy_r, kxy_r, kxxy_r, kxyy_r = r[3], r[4], r[5], r[6], r[7]
    k = M.central_moments(fb, u, lat)
    tol = 1e-15
    assert torch.allclose(k[3], kxx_r + Fx * ux - rho * ux ** 2, atol=tol)
    assert torch.allclose(k[4], kyy_r + Fy * uy - rho * uy ** 2, atol=tol)
    assert torch.allclose(k[5], kxy_r + 0.5 * (Fx * uy + Fy * ux) - rho * ux * uy, atol=tol)
    assert torch.allclose(k[7], kxyy_r - 2 * uy * kxy_r - ux * kyy_r - 0.5 * Fx * uy ** 2
                          - Fy * ux * uy + 2 * rho * ux * uy ** 2, atol=tol)
    assert torch.allclose(k[6], kxxy_r - 2 * ux * kxy_r - uy * kxx_r - 0.5 * Fy * ux ** 2
                          - Fx * ux * uy + 2 * rho * ux ** 2 * uy, atol=tol)
    # conserved moments of fbar (Sec. 8): kbar_0 = rho, kbar_x = -F_x/2
    assert torch.allclose(k[1], -0.5 * Fx, atol=1e-16)
    assert torch.allclose(k[2], -0.5 * Fy, atol=1e-16)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27"])
def test_equilibrium_is_product_of_1d_maxwellians(name):
    """The discrete Maxwellian matched to Eq. centralmomentMaxwelldistribution equals the
    closed-form product of 1D populations (2/3 - u^2, (1/3 + u^2 +- u)/2)."""
    lat = L.get(name)
    g = torch.Generator().manual_seed(4)
    n = 32
    rho = 1 + 0.1 * torch.randn(n, generator=g, dtype=DT)
    u = 0.2 * torch.randn(3, n, generator=g, dtype=DT)
    if lat.d == 2:
        u[2] = 0
    feq = C.equilibrium(rho, u, torch.zeros(3, n, dtype=DT), lat)

    def phi(e, v):
        return 2.0 / 3.0 - v * v if e == 0 else 0.5 * (1.0 / 3.0 + v * v + e * v)

    for i in range(lat.Q):
        ex, ey, ez = (int(x) for x in lat.e[i])
        ref = rho * phi(ex, u[0]) * phi(ey, u[1]) * (phi(ez, u[2]) if lat.d == 3 else 1.0)
        assert torch.allclose(feq[i], ref, atol=1e-15, rtol=0)
    # rest state gives the weights
    w = C.equilibrium(torch.ones(1, dtype=DT), torch.zeros(3, 1, dtype=DT), torch.zeros(3, 1, dtype=DT), lat)
    assert torch.allclose(w[:, 0], lat.w, atol=1e-16, rtol=0)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27"])
def test_equilibrium_central_moments(name):
    lat = L.get(name)
    n = 16
    rho = torch.linspace(0.9, 1.1, n, dtype=DT)
    u = torch.stack([torch.linspace(-0.1, 0.1, n, dtype=DT), torch.linspace(0.05, -0.05, n, dtype=DT),
                     torch.linspace(-0.02, 0.03, n, dtype=DT) * (lat.d == 3)])
    feq = C.equilibrium(rho, u, torch.zeros(3, n, dtype=DT), lat)
    k = M.central_moments(feq, u, lat)
    for j, a in enumerate(lat.monomials):
        if all(x % 2 == 0 for x in a):
            ref = rho * (1.0 / 3.0) ** (sum(a) // 2)
        else:
            ref = torch.zeros_like(rho)
        assert torch.allclose(k[j], ref, atol=1e-15, rtol=0)
