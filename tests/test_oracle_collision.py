"""Oracle pins: source hierarchy, source populations, conservation, relaxation, literal form.

Secs. 5-11 of the paper. Each pin compares the generic oracle against a route the paper
prints independently (explicit formulas, velocity-space sources, element-wise update) or
against an exact invariant.
"""
import pytest
import torch

from oracle import lattice as L, moments as M, collision as C, literal as LIT

DT = torch.float64


def _state(lat, n, seed, amp=0.05, famp=1e-2):
    g = torch.Generator().manual_seed(seed)
    rho = 1 + amp * torch.randn(n, generator=g, dtype=DT)
    u = 0.1 * torch.randn(3, n, generator=g, dtype=DT)
    F = famp * torch.randn(3, n, generator=g, dtype=DT)
    if lat.d == 2:
        u[2] = 0
        F[2] = 0
    feq = C.equilibrium(rho, u, torch.zeros_like(F), lat)
    fb = feq * (1 + amp * torch.randn(feq.shape, generator=g, dtype=DT))
    return fb, F


def test_source_hierarchy_matches_printed_d2q9_expressions():
    """sigma from the generic recursion vs the expanded Eq. centralmomentforcingtransformed."""
    lat = L.D2Q9
    fb, F = _state(lat, 128, 10)
    rho, u = C.hydrodynamics(fb, F, lat)
    kb = M.central_moments(fb, u, lat)
    sig, _ = C.source_central(kb, rho, F, lat)
    Fx, Fy = F[0], F[1]
    kxx, kyy, kxy, kxxy, kxyy = kb[3], kb[4], kb[5], kb[6], kb[7]
    ref = [torch.zeros_like(rho), Fx, Fy, torch.zeros_like(rho), torch.zeros_like(rho), torch.zeros_like(rho),
           2 * Fx / rho * kxy + Fy / rho * kxx,
           Fx / rho * kyy + 2 * Fy / rho * kxy,
           2 * Fx / rho * kxyy + 2 * Fy / rho * kxxy + Fy ** 2 / rho ** 2 * kxx + Fx ** 2 / rho ** 2 * kyy
           + 4 * Fx * Fy / rho ** 2 * kxy]
    for j in range(9):
        assert torch.allclose(sig[j], ref[j], atol=1e-17, rtol=1e-13), j


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27"])
def test_source_populations_satisfy_exact_identity(name):
    """Central moments of S (explicit sums) equal Eq. centralmomentforceexactidentity2 applied to
    the central moments of f = fbar + S/2 (Eq. transformedcentralmoments)."""
    lat = L.get(name)
    fb, F = _state(lat, 64, 11)
    rho, u = C.hydrodynamics(fb, F, lat)
    S = C.source_populations(fb, F, lat)
    f = fb + 0.5 * S
    kap = M.central_moments(f, u, lat)
    sig = M.central_moments(S, u, lat)
    idx = {a: k for k, a in enumerate(lat.monomials)}
    for a in lat.monomials:
        ref = torch.zeros_like(rho)
        for d in range(3):
            if a[d]:
                lo = list(a)
                lo[d] -= 1
                ref = ref + a[d] * F[d] / rho * kap[idx[tuple(lo)]]
        assert torch.allclose(sig[idx[a]], ref, atol=1e-15, rtol=1e-12), a
    # conserved moments of f: kappa_0 = rho, kappa_x = 0 (Sec. 8)
    for d in range(lat.d):
        e = [0, 0, 0]
        e[d] = 1
        assert kap[idx[tuple(e)]].abs().max().item() < 1e-15


def test_d2q9_source_equals_printed_velocity_space_terms():
    """Generic S = T(u)^-1 sigma vs Eqs. vsourceterms0-8 built from Eqs. sourceterm0-8."""
    lat = L.D2Q9
    for seed in (12, 13):
        fb, F = _state(lat, 128, seed)
        _, _, S_lit = LIT.collide_literal(fb, F, (1.0,) * 6)
        S_gen = C.source_populations(fb, F, lat)
        assert (S_lit - S_gen).abs().max().item() < 1e-17


def test_d2q9_source_raw_moments_printed():
    """Raw moments of S vs Eqs. rawmomentsourceterm0-8 (sigma'_yy read as 2 F_y u_y)."""
    lat = L.D2Q9
    fb, F = _state(lat, 64, 14)
    rho, u = C.hydrodynamics(fb, F, lat)
    S = C.source_populations(fb, F, lat)
    r = M.raw_moments(S, lat)
    kb = M.central_moments(fb, u, lat)
    ux, uy, Fx, Fy = u[0], u[1], F[0], F[1]
    kxx, kyy, kxy, kxxy, kxyy = kb[3], kb[4], kb[5], kb[6], kb[7]
    ref = [torch.zeros_like(rho), Fx, Fy, 2 * Fx * ux, 2 * Fy * uy, Fx * uy + Fy * ux,
           2 * Fx * (kxy / rho + ux * uy) + Fy * (kxx / rho + ux * ux),
           Fx * (kyy / rho + uy * uy) + 2 * Fy * (kxy / rho + ux * uy),
           2 * Fx * ux * (kyy / rho + uy * uy) + 2 * Fy * uy * (kxx / rho + ux * ux)
           + 2 * Fx / rho * kxyy + 2 * Fy / rho * kxxy + Fx ** 2 / rho ** 2 * kyy + Fy ** 2 / rho ** 2 * kxx
           + 4 * (Fx * uy / rho + Fy * ux / rho + Fx * Fy / rho ** 2) * kxy]
    for j in range(9):
        assert torch.allclose(r[j], ref[j], atol=1e-17, rtol=1e-12), j
    # the printed sigma'_yy = 2 F_x u_y is not the raw moment (typo reading)
    assert (r[4] - 2 * Fx * uy).abs().max().item() > 1e-4


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27"])
def test_collision_conserves_mass_and_adds_force(name):
    lat = L.get(name)
    fb, F = _state(lat, 64, 15)
    p = C.Params(tau=0.62, omega_bulk=1.1, omega3=1.3, omega4=0.8)
    post = C.collide(fb, F, lat, p)
    d = post - fb
    assert d.sum(0).abs().max().item() < 1e-15
    for ax in range(3):
        mom = (d * lat.e[:, ax].to(DT).view(-1, 1)).sum(0)
        assert torch.allclose(mom, F[ax], atol=1e-15, rtol=0)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27"])
def test_equilibrium_is_fixed_point_without_force(name):
    lat = L.get(name)
    g = torch.Generator().manual_seed(16)
    rho = 1 + 0.05 * torch.randn(32, generator=g, dtype=DT)
    u = 0.1 * torch.randn(3, 32, generator=g, dtype=DT)
    if lat.d == 2:
        u[2] = 0
    F = torch.zeros(3, 32, dtype=DT)
    feq = C.equilibrium(rho, u, F, lat)
    post = C.collide(feq, F, lat, C.Params(tau=0.7, omega3=1.2, omega4=0.9))
    assert (post - feq).abs().max().item() < 1e-15


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27"])
def test_relaxation_rates_by_order(name):
    """Post-collision central moments (explicit sums about the pre-collision u): trace with
    omega_b, deviator and off-diagonals with omega_nu = 1/tau, orders 3 and >= 4 with omega3, omega4."""
    lat = L.get(name)
    fb, F = _state(lat, 64, 17, famp=0.0)
    p = C.Params(tau=0.62, omega_bulk=1.1, omega3=1.3, omega4=0.8)
    rho, u = C.hydrodynamics(fb, F, lat)
    pre = M.central_moments(fb, u, lat)
    post = M.central_moments(C.collide(fb, F, lat, p), u, lat)
    idx = {a: k for k, a in enumerate(lat.monomials)}
    wnu = 1 / p.tau
    diag = [idx[tuple(2 if c == d else 0 for c in range(3))] for d in range(lat.d)]
    tr_pre = sum(pre[k] for k in diag) - lat.d * rho / 3
    tr_post = sum(post[k] for k in diag) - lat.d * rho / 3
    assert torch.allclose(tr_post, (1 - p.omega_bulk) * tr_pre, atol=1e-15)
    dev_pre = pre[diag[0]] - pre[diag[1]]
    dev_post = post[diag[0]] - post[diag[1]]
    assert torch.allclose(dev_post, (1 - wnu) * dev_pre, atol=1e-15)
    for a in lat.monomials:
        n = sum(a)
        k = idx[a]
        if n == 2 and max(a) == 1:
            assert torch.allclose(post[k], (1 - wnu) * pre[k], atol=1e-15)
        if n >= 3:
            w = p.omega3 if n == 3 else p.omega4
            ref = (1 - w) * pre[k] + w * (rho * (1 / 3) ** (n // 2) if all(x % 2 == 0 for x in a) else 0)
            assert torch.allclose(post[k], ref, atol=1e-15), a


def test_literal_equals_generic_without_force():
    lat = L.D2Q9
    fb, F = _state(lat, 128, 18)
    F = torch.zeros_like(F)
    for tau, w_b, w3, w4 in [(0.8, 0.0, 1.0, 1.0), (0.55, 1.4, 1.7, 0.6)]:
        wnu = 1 / tau
        p = C.Params(tau=tau, omega_bulk=w_b, omega3=w3, omega4=w4)
        om = (w_b if w_b else wnu, wnu, wnu, w3, w3, w4)
        post_l, _, _ = LIT.collide_literal(fb, F, om)
        post_g = C.collide(fb, F, lat, p)
        assert (post_l - post_g).abs().max().item() < 1e-15


def test_literal_vs_generic_with_force_residual_structure():
    """With F != 0 the printed g6-g8 differ from relaxing toward Eq. centralmomenttransformed by
    exactly +omega3 sigma at third order and -omega4 (u_y sigma_xxy + u_x sigma_xyy) at fourth
    order; orders <= 2 agree. This pins both forms and documents the reading."""
    lat = L.D2Q9
    fb, F = _state(lat, 256, 19)
    p = C.Params(tau=0.7, omega3=1.3, omega4=0.9)
    om = (1 / 0.7, 1 / 0.7, 1 / 0.7, 1.3, 1.3, 0.9)
    post_l, _, _ = LIT.collide_literal(fb, F, om)
    post_g = C.collide(fb, F, lat, p)
    rho, u = C.hydrodynamics(fb, F, lat)
    kl = M.central_moments(post_l, u, lat)
    kg = M.central_moments(post_g, u, lat)
    sig, _ = C.source_central(M.central_moments(fb, u, lat), rho, F, lat)
    for j in range(6):
        assert (kl[j] - kg[j]).abs().max().item() < 1e-15
    assert torch.allclose(kl[6] - kg[6], 1.3 * sig[6], atol=1e-16, rtol=1e-10)
    assert torch.allclose(kl[7] - kg[7], 1.3 * sig[7], atol=1e-16, rtol=1e-10)
    assert torch.allclose(kl[8] - kg[8], -0.9 * (u[1] * sig[6] + u[0] * sig[7]), atol=1e-16, rtol=1e-10)


def test_literal_collision_kernel_raw_moments():
    """Raw moments of K g (Eq. collisionkernelmoment) from the element-wise update."""
    lat = L.D2Q9
    fb, F = _state(lat, 64, 20)
    post, (g3, g4, g5, g6, g7, g8), S = LIT.collide_literal(fb, F, (1.2, 1.3, 1.3, 1.1, 0.9, 1.0))
    Om = post - fb - S
    r = M.raw_moments(Om, lat)
    z = torch.zeros_like(g3)
    ref = [z, z, z, 6 * g3 + 2 * g4, 6 * g3 - 2 * g4, 4 * g5, -4 * g6, -4 * g7, 8 * g3 + 4 * g8]
    for j in range(9):
        assert torch.allclose(r[j], ref[j], atol=1e-16, rtol=1e-12), j


def _unit_state(lat, n, seed):
    fb, F = _state(lat, n, seed)
    return fb / fb.sum(0), F


def test_reduced_compressibility_literal_equals_generic_without_force():
    """Eqs. collisionkernelcompact3-8 (Sec. 12) equal the generic step with u = (sum fbar e + F/2)/rho0."""
    lat = L.D2Q9
    fb, F = _state(lat, 128, 21)
    F = torch.zeros_like(F)
    om = (1 / 0.7, 1 / 0.7, 1 / 0.7, 1.3, 1.3, 0.9)
    for rho0 in (1.0, 1.02):
        post_l, _, _ = LIT.collide_literal(fb, F, om, rho0=rho0)
        p = C.Params(tau=0.7, omega3=1.3, omega4=0.9, reduced_compressibility=True, rho0=rho0)
        post_g = C.collide(fb, F, lat, p)
        assert (post_l - post_g).abs().max().item() < 1e-15


def test_reduced_compressibility_equals_standard_at_reference_density():
    lat = L.D3Q27
    fb, F = _unit_state(lat, 32, 22)
    p0 = C.Params(tau=0.62, omega3=1.2, omega4=0.8)
    p1 = C.Params(tau=0.62, omega3=1.2, omega4=0.8, reduced_compressibility=True, rho0=1.0)
    assert (C.collide(fb, F, lat, p0) - C.collide(fb, F, lat, p1)).abs().max().item() < 1e-15


def test_factorized_literal_equals_generic_at_unit_density_without_force():
    """Eq. factorxxyyfinal (Sec. 13) as printed equals the generic factorized attractor at rho = 1
    (the reading divides the product by rho, which the paper writes for unit density)."""
    lat = L.D2Q9
    fb, F = _unit_state(lat, 128, 23)
    F = torch.zeros_like(F)
    om = (1 / 0.7, 1 / 0.7, 1 / 0.7, 1.3, 1.3, 0.9)
    post_l, _, _ = LIT.collide_literal(fb, F, om, factorized=True)
    post_g = C.collide(fb, F, lat, C.Params(tau=0.7, omega3=1.3, omega4=0.9, attractor="factorized"))
    assert (post_l - post_g).abs().max().item() < 1e-15
    # and it is a different collision from the Maxwellian attractor away from equilibrium
    post_m = C.collide(fb, F, lat, C.Params(tau=0.7, omega3=1.3, omega4=0.9))
    assert (post_g - post_m).abs().max().item() > 1e-4


@pytest.mark.parametrize("name", ["D2Q9", "D3Q27"])
def test_factorized_attractor_keeps_the_maxwellian_fixed_point(name):
    """At equilibrium the relaxed second-order moments are Maxwellian and the products reduce to
    rho c_s^(a+b+c): the factorized step leaves f^M unchanged (F = 0)."""
    lat = L.get(name)
    g = torch.Generator().manual_seed(24)
    rho = 1 + 0.05 * torch.randn(32, generator=g, dtype=DT)
    u = 0.1 * torch.randn(3, 32, generator=g, dtype=DT)
    if lat.d == 2:
        u[2] = 0
    F = torch.zeros(3, 32, dtype=DT)
    feq = C.equilibrium(rho, u, F, lat)
    post = C.collide(feq, F, lat, C.Params(tau=0.7, omega3=1.2, omega4=0.9, attractor="factorized"))
    assert (post - feq).abs().max().item() < 1e-15


def test_factorized_literal_vs_generic_with_force_residual_structure():
    """Eq. factorxxyyfinal as printed (Sec. 13), with F != 0 and rho != 1, against the generic
    factorized step. The printed brackets are the post-collision second-order central moments
    k~_xx, k~_yy (pre-collision kbar_dd plus the 6 g3 +- 2 g4 of the kernel), and the printed force
    terms are sigma_xxyy / 2 of the hierarchy (Eq. centralmomentforcingtransformed expanded), so
    the printed transformed attractor is k~_xx k~_yy - sigma_xxyy / 2, where the reading divides the
    product by rho: k~_xx k~_yy / rho - sigma_xxyy / 2. It replaces rho / 9 in g8, which itself
    subtracts sigma'_xxyy / 2 again, as for the Maxwellian attractor. Hence, printed minus generic
    post-collision central moments: 0 at orders <= 2; omega3 sigma at third order (g6, g7 are
    those of Sec. 10); omega4 [k~_xx k~_yy (1 - 1/rho) - sigma_xxyy / 2 - u_y sigma_xxy
    - u_x sigma_xyy] at fourth order."""
    lat = L.D2Q9
    fb, F = _state(lat, 256, 25)
    p = C.Params(tau=0.7, omega3=1.3, omega4=0.9, attractor="factorized")
    om = (1 / 0.7, 1 / 0.7, 1 / 0.7, 1.3, 1.3, 0.9)
    post_l, _, _ = LIT.collide_literal(fb, F, om, factorized=True)
    post_g = C.collide(fb, F, lat, p)
    rho, u = C.hydrodynamics(fb, F, lat)
    assert (rho - 1).abs().min().item() > 1e-4 and F.abs().max().item() > 1e-3
    kl = M.central_moments(post_l, u, lat)
    kg = M.central_moments(post_g, u, lat)
    sig, _ = C.source_central(M.central_moments(fb, u, lat), rho, F, lat)
    for j in range(6):
        assert (kl[j] - kg[j]).abs().max().item() < 2e-15, j
    assert torch.allclose(kl[6] - kg[6], 1.3 * sig[6], atol=1e-16, rtol=1e-10)
    assert torch.allclose(kl[7] - kg[7], 1.3 * sig[7], atol=1e-16, rtol=1e-10)
    ref8 = 0.9 * (kg[3] * kg[4] * (1 - 1 / rho) - 0.5 * sig[8] - u[1] * sig[6] - u[0] * sig[7])
    assert ref8.abs().max().item() > 1e-3
    assert torch.allclose(kl[8] - kg[8], ref8, atol=1e-15, rtol=1e-10)


def _one_axis(g, n, u, theta):
    """Populations on e = -1, 0, 1 with mean u and central second moment theta:
    p(+-1) = (theta + u^2 +- u) / 2, p(0) = 1 - theta - u^2."""
    q = theta + u * u
    return torch.stack([(q - u) / 2, 1 - q, (q + u) / 2])


def _partially_factorized_state(split, n, seed):
    """rho p_a(e_a) q_bc(e_b, e_c): axis a independent of the pair (b, c), with a random 1D
    marginal p_a and a random positive 9-point joint q_bc (correlated b and c)."""
    g = torch.Generator().manual_seed(seed)
    lat = L.D3Q27
    rho = 0.8 + 0.5 * torch.rand(n, generator=g, dtype=DT)
    ua = 0.1 * torch.randn(n, generator=g, dtype=DT)
    ta = 0.28 + 0.1 * torch.rand(n, generator=g, dtype=DT)
    pa = _one_axis(g, n, ua, ta)                                         # [3, n] over e_a
    q = 0.5 + torch.rand(3, 3, n, generator=g, dtype=DT)                 # [e_b, e_c, n]
    q = q / q.sum((0, 1))
    b, c = [d for d in range(3) if d != split]
    f = torch.empty(27, n, dtype=DT)
    for i in range(27):
        e = [int(v) for v in lat.e[i]]
        f[i] = rho * pa[e[split] + 1] * q[e[b] + 1, e[c] + 1]
    return f, rho


@pytest.mark.parametrize("split", [0, 1, 2])
def test_factorized_3d_attractors_of_partially_factorized_states(split):
    """Sec. 13's postulate: the attractors are products of post-collision lower-order central
    moments, as for a distribution that factorizes over its Cartesian components. For a state
    whose axis a is independent of the pair (b, c), its central moments are products
    kappa_(a-part, bc-part) = rho m_a * M_bc of the marginals' moments (m_0 = 1, m_1 = 0,
    m_2 = theta_a; M_00 = 1, M_10 = M_01 = 0, M_20 = theta_b, M_02 = theta_c, M_11 = c_bc, and,
    with the pair at its own (D2Q9) factorized attractor, M_21 = M_12 = 0, M_22 = theta_b theta_c).
    With omega3 = omega4 = 1 and F = 0 a step leaves every moment of order >= 3 at its attractor,
    so those of the output must be these products of the output's own second-order moments
    (theta = kappa~_dd / rho, c_bc = kappa~_bc / rho). Every one of the eight moments with three
    non-zero exponents enters: (2,1,1) with the 2 on axis a is rho theta_a c_bc, (2,2,2) is
    rho theta_x theta_y theta_z, the others vanish."""
    lat = L.D3Q27
    fb, rho = _partially_factorized_state(split, 64, 30 + split)
    F = torch.zeros(3, fb.shape[1], dtype=DT)
    p = C.Params(tau=0.7, omega_bulk=1.3, omega3=1.0, omega4=1.0, attractor="factorized")
    post = C.collide(fb, F, lat, p)
    _, u = C.hydrodynamics(fb, F, lat)
    K = M.central_moments(post, u, lat)
    idx = {a: k for k, a in enumerate(lat.monomials)}
    b, c = [d for d in range(3) if d != split]

    def mono(exps):
        return idx[tuple(exps)]

    theta = []
    for d in range(3):
        e = [0, 0, 0]
        e[d] = 2
        theta.append(K[mono(e)] / rho)
    e = [0, 0, 0]
    e[b] = e[c] = 1
    cbc = K[mono(e)] / rho
    assert cbc.abs().max().item() > 1e-2                 # the pair really is correlated
    m = {0: torch.ones_like(rho), 1: torch.zeros_like(rho), 2: theta[split]}
    Mbc = {(0, 0): torch.ones_like(rho), (1, 0): 0 * rho, (0, 1): 0 * rho, (2, 0): theta[b], (0, 2): theta[c],
           (1, 1): cbc, (2, 1): 0 * rho, (1, 2): 0 * rho, (2, 2): theta[b] * theta[c]}
    nonzero_three = 0
    for a in lat.monomials:
        if sum(a) < 3:
            continue
        want = rho * m[a[split]] * Mbc[(a[b], a[c])]
        assert torch.allclose(K[idx[a]], want, atol=1e-15, rtol=1e-12), a
        if min(a) > 0 and want.abs().max().item() > 1e-6:
            nonzero_three += 1
    assert nonzero_three == 2            # (2,1,1) on axis a and (2,2,2)
    # the Maxwellian attractor gives different higher moments for the same state
    post_m = C.collide(fb, F, lat, C.Params(tau=0.7, omega_bulk=1.3))
    assert (M.central_moments(post_m, u, lat) - K).abs().max().item() > 1e-4
