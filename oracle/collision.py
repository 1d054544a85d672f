"""Cascaded central-moment collision with Galilean-invariant forcing, generic form.

Test infrastructure (see the package docstring).

One collision, in the paper's order (Secs. 6-11):
  1. rho = sum fbar, rho u = sum fbar e + F/2          (Eqs. densitycalculation, velocitycalculation)
  2. kbar_a = central moments of fbar about u          (definition below Eq. centralmomentforcing)
  3. sigma_a from the exact hierarchical identity      (Eq. centralmomentforceexactidentity2 with
     kappa = kbar + sigma/2, Eq. transformedcentralmoments; kappa_0 = rho, kappa_x = 0 as
     stated under the relations of Sec. 8)
  4. attractor kbar^M_a = kappa^M_a - sigma_a/2        (Eq. centralmomenttransformed)
  5. relax the non-conserved moments toward the attractor and add the source:
     post_a = kbar_a + omega_a (kbar^M_a - kbar_a) + sigma_a   (Sec. 10 procedure; Eq. cascadedcollision1)
  6. back to populations through the exact inverse (Sec. 9).
The element-wise D2Q9 formulas as printed live in ``literal.py``; where they differ from
this form at third and fourth order in the force, this form is the normative reading
(it follows the stated principle: relax toward Eq. centralmomenttransformed, then add S).

Rates (Sec. 10, below Eq. collisionkernelg8): the trace of the second-order moments relaxes
with the bulk rate, the deviatoric and off-diagonal second-order moments with the shear
rate omega_nu = 1/tau (nu = c_s^2 (1/omega_nu - 1/2)); third order with omega3, fourth and
higher with omega4. Where the eddy viscosity is on, omega_nu comes from ``les.py``.
"""
from dataclasses import dataclass

import torch

from .lattice import CS2, DT
from . import moments as M
from . import les


@dataclass
class Params:
    tau: float = 0.8               # shear relaxation time, omega_nu = 1/tau
    omega_bulk: float = 0.0        # 0 -> equal to the (effective) shear rate
    omega3: float = 1.0            # third-order central moments
    omega4: float = 1.0            # fourth and higher orders
    cs_smag: float = 0.0           # Smagorinsky constant, 0 = no eddy viscosity
    attractor: str = "maxwell"     # "maxwell" (Eq. centralmomenttransformed) or "factorized" (Sec. 13)
    reduced_compressibility: bool = False   # Sec. 12: rho0 u = sum fbar e + F/2
    rho0: float = 1.0


def hydrodynamics(fbar, F, lat, p=None):
    """rho = sum fbar (Eq. densitycalculation); rho u = sum fbar e + F/2 (Eq. velocitycalculation).

    With reduced compressibility (Sec. 12) the momentum is rho0 u instead of rho u.
    """
    rho = fbar.sum(0)
    mom = []
    for d in range(3):
        acc = torch.zeros_like(rho)
        for i in range(lat.Q):
            c = float(lat.e[i, d])
            if c != 0.0:
                acc = acc + c * fbar[i]
        mom.append(acc + 0.5 * F[d])
    mom = torch.stack(mom)
    if p is not None and p.reduced_compressibility:
        u = mom / p.rho0
    else:
        u = mom / rho
    return rho, u


def maxwell_central(rho, lat):
    """Central moments of the Maxwellian: rho c_s^(a0+a1+a2) if every exponent is even, else 0.

    Sec. 4 (Eq. after centralmomentfeqdefinition) and its discrete match, Eq.
    centralmomentMaxwelldistribution; the third exponent is the 3D reading.
    """
    out = []
    for a in lat.monomials:
        if all(x % 2 == 0 for x in a):
            out.append(rho * CS2 ** (sum(a) // 2))
        else:
            out.append(torch.zeros_like(rho))
    return torch.stack(out)


def source_central(kbar, rho, F, lat):
    """Central moments sigma_a of the source, in increasing order (Sec. 5 and Sec. 8).

    The exact identity Gamma_(x^m y^n) = m (F_x/rho) Pi_(x^(m-1) y^n) + n (F_y/rho) Pi_(x^m y^(n-1))
    (Eq. centralmomentforceexactidentity2), with a third term in 3D, applied to the central
    moments kappa of the untransformed f, kappa_a = kbar_a + sigma_a / 2 (Eq.
    transformedcentralmoments). The conserved central moments are kappa_0 = rho and
    kappa_x = kappa_y = kappa_z = 0 by definition (Sec. 8, text above the reduced
    relations), which gives sigma_x = F_x and zero second-order sources (Eq.
    centralmomentforcingtransformed).

    Returns (sigma, kappa) with kappa the central moments of f.
    """
    idx = {a: k for k, a in enumerate(lat.monomials)}
    sigma = [None] * len(lat.monomials)
    kappa = [None] * len(lat.monomials)
    for a in lat.monomials:          # monomials are stored in increasing total order
        k = idx[a]
        s = torch.zeros_like(rho)
        for d in range(3):
            if a[d] > 0:
                lower = list(a)
                lower[d] -= 1
                s = s + a[d] * (F[d] / rho) * kappa[idx[tuple(lower)]]
        sigma[k] = s
        n = sum(a)
        if n == 0:
            kappa[k] = rho
        elif n == 1:
            kappa[k] = torch.zeros_like(rho)
        else:
            kappa[k] = kbar[k] + 0.5 * s
    return torch.stack(sigma), torch.stack(kappa)


def equilibrium(rho, u, F, lat):
    """Initial transformed populations fbar = f^M - S/2 with the Maxwellian moments.

    The discrete Maxwellian is the population whose central moments are kappa^M (matching
    principle, Sec. 7). Its source is the identity evaluated at kappa = kappa^M (the special
    case noted under Eq. exactidentitycomponents). Initialisation itself is paper silent.
    """
    kM = maxwell_central(rho, lat)
    idx = {a: k for k, a in enumerate(lat.monomials)}
    sig = []
    for a in lat.monomials:
        s = torch.zeros_like(rho)
        for d in range(3):
            if a[d] > 0:
                lower = list(a)
                lower[d] -= 1
                s = s + a[d] * (F[d] / rho) * kM[idx[tuple(lower)]]
        sig.append(s)
    sig = torch.stack(sig)
    return M.central_to_populations(kM - 0.5 * sig, u, lat)


def _factorized_attractor(kM, post2, rho, lat):
    """Factorized attractors (Sec. 13): products of post-collision second-order central moments.

    D2Q9: kappa^at_xxy = kappa^at_xyy = 0 and kappa^at_xxyy = k~_xx k~_yy (Eq. factorxxyy).
    Reading: the product is divided by rho so that it equals the Maxwellian rho c_s^4 when the
    second-order moments are at equilibrium (the paper writes it for unit density). 3D reading:
    each axis with exponent 2 contributes k~_dd, two axes with exponent 1 contribute one
    off-diagonal k~_de, any other pattern gives 0; k factors are divided by rho^(k-1).
    Second order keeps the Maxwellian attractor.

    The paper gives the factorized attractor for D2Q9 only. The D2Q9 form is pinned against the
    printed element-wise kernel (``literal.py``) with and without a force and at rho != 1 (the
    printed product lacks the 1/rho, and its force terms are sigma_xxyy / 2: the residual between
    the two forms is derived and asserted order by order). The 3D rules of every moment with at
    most two non-zero exponents are pinned to it: a one-cell-thick D3Q27 run of a 2D flow in the
    x-y, x-z or y-z plane reproduces the D2Q9 run. The moments with three non-zero exponents are
    pinned by Sec. 13's postulate itself: for a state with one axis independent of the other two
    (a product of a 1D marginal and a 2D joint at its own factorized attractor) the attractors of
    every order are that state's own central moments, products of the marginals' moments.
    """
    idx = {a: k for k, a in enumerate(lat.monomials)}
    out = kM.clone()
    for a in lat.monomials:
        if sum(a) < 3:
            continue
        ones = [d for d in range(3) if a[d] == 1]
        twos = [d for d in range(3) if a[d] == 2]
        if len(ones) not in (0, 2):
            out[idx[a]] = torch.zeros_like(rho)
            continue
        factors = []
        for d in twos:
            e2 = [0, 0, 0]
            e2[d] = 2
            factors.append(post2[idx[tuple(e2)]])
        if len(ones) == 2:
            e11 = [0, 0, 0]
            e11[ones[0]] = 1
            e11[ones[1]] = 1
            factors.append(post2[idx[tuple(e11)]])
        prod = factors[0]
        for f_ in factors[1:]:
            prod = prod * f_
        out[idx[a]] = prod / rho ** (len(factors) - 1)
    return out


def collide(fbar, F, lat, p, cs_eff=None):
    """Post-collision transformed populations (generic central-moment form).

    fbar[Q, ...], F[3, ...]; cs_eff (broadcastable to the cell shape) is the Smagorinsky
    constant per cell after wall damping, or None to use p.cs_smag everywhere.
    Returns fbar_post[Q, ...].
    """
    rho, u = hydrodynamics(fbar, F, lat, p)
    kbar = M.central_moments(fbar, u, lat)
    sigma, kap = source_central(kbar, rho, F, lat)
    kM = maxwell_central(rho, lat)
    idx = {a: k for k, a in enumerate(lat.monomials)}

    omega_nu = torch.full_like(rho, 1.0 / p.tau)
    cs = p.cs_smag if cs_eff is None else cs_eff
    if p.cs_smag > 0.0 or cs_eff is not None:
        Pi = les.nonequilibrium_stress(kap, rho, lat)
        omega_nu = 1.0 / les.tau_effective(p.tau, cs, Pi, rho)
    omega_b = omega_nu if p.omega_bulk == 0.0 else torch.full_like(rho, p.omega_bulk)

    post = torch.empty_like(kbar)
    # orders 0 and 1: collision invariants, only the source is added
    for a in lat.monomials:
        if sum(a) <= 1:
            post[idx[a]] = kbar[idx[a]] + sigma[idx[a]]

    # order 2: attractor kbar^M = kappa^M (sigma = 0 at second order)
    axes = list(range(lat.d))
    diag = [idx[tuple(2 if d == c else 0 for d in range(3))] for c in axes]
    delta = [kM[k] - 0.5 * sigma[k] - kbar[k] for k in diag]
    mean = sum(delta) / len(delta)
    for c, k in enumerate(diag):
        post[k] = kbar[k] + omega_b * mean + omega_nu * (delta[c] - mean) + sigma[k]
    for a in lat.monomials:
        if sum(a) == 2 and max(a) == 1:
            k = idx[a]
            post[k] = kbar[k] + omega_nu * (kM[k] - 0.5 * sigma[k] - kbar[k]) + sigma[k]

    # orders >= 3
    attract = kM
    if p.attractor == "factorized":
        # post-collision central moments of f at second order (collision part only)
        post2 = post.clone()
        attract = _factorized_attractor(kM, post2, rho, lat)
    for a in lat.monomials:
        n = sum(a)
        if n >= 3:
            k = idx[a]
            w = p.omega3 if n == 3 else p.omega4
            post[k] = kbar[k] + w * (attract[k] - 0.5 * sigma[k] - kbar[k]) + sigma[k]

    return M.central_to_populations(post, u, lat)


def source_populations(fbar, F, lat, p=None):
    """S_alpha: the populations whose central moments about u are sigma (Sec. 9, S = K D^-1 m^s)."""
    rho, u = hydrodynamics(fbar, F, lat, p)
    kbar = M.central_moments(fbar, u, lat)
    sigma, _ = source_central(kbar, rho, F, lat)
    return M.central_to_populations(sigma, u, lat)
