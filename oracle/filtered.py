"""Turbulence as forcing in the filtered lattice kinetic equation (Sec. 14), for the oracle.

Test infrastructure (see the package docstring).

The filtered equation carries the unresolved stresses as a body force: a'_i = -d_j (u'_i u'_j)
(the Cartesian components printed below Eq. resolvedcentralmomentforce), entering the step as
F = rho a' with the resolved momentum rho0 u = sum fbar e + rho a' / 2 (Eq.
resolvedvelocitycalculation). The paper leaves the macroscopic closure open ("any
conventional macroscopic turbulence model"); the reading used here is the Smagorinsky model
for the deviatoric part, u'_i u'_j - delta_ij u'_k u'_k / 3 = -2 nu_t S_ij with
nu_t = (C_s Delta)^2 |S|, |S| = sqrt(2 S:S), Delta = 1, the isotropic part going into the
pressure. Derivatives are second-order central differences on the periodic lattice,
d_j phi(x) = (phi(x + e_j) - phi(x - e_j)) / 2, applied once to the velocity and once to the
stress. The closure velocity is the resolved velocity of the current pre-collision field with
the force of the previous evaluation (paper silent on the time discretisation).
"""
import math

import torch


def _d(phi, axis):
    """Central difference along grid axis (0 = x, 1 = y, 2 = z) of a [nz, ny, nx] field."""
    dim = {0: 2, 1: 1, 2: 0}[axis]
    return 0.5 * (torch.roll(phi, -1, dims=dim) - torch.roll(phi, 1, dims=dim))


def strain_rate(u, d):
    """S_ij = (d_i u_j + d_j u_i) / 2 for i, j < d; returns {(i, j): tensor}."""
    grad = {(i, j): _d(u[j], i) for i in range(d) for j in range(d)}       # d_i u_j
    return {(i, j): 0.5 * (grad[(i, j)] + grad[(j, i)]) for i in range(d) for j in range(d)}


def eddy_stress(u, cs, d):
    """T_ij = 2 nu_t S_ij = -(u'_i u'_j)^dev with nu_t = cs^2 |S|, |S| = sqrt(2 S:S)."""
    S = strain_rate(u, d)
    mag = torch.sqrt(2.0 * sum(v * v for v in S.values()))
    nu_t = cs * cs * mag
    return {k: 2.0 * nu_t * v for k, v in S.items()}


def turbulence_acceleration(u, cs, d):
    """a'_i = -d_j (u'_i u'_j) = d_j T_ij (the isotropic part is left in the pressure)."""
    T = eddy_stress(u, cs, d)
    a = torch.zeros_like(u)
    for i in range(d):
        for j in range(d):
            a[i] = a[i] + _d(T[(i, j)], j)
    return a


def discrete_shear_mode(A, k, cs, y):
    """Closed form of the chain above for u_x = A sin(k y) on the periodic lattice (pin).

    The central difference of sin(k y) is sin(k) cos(k y), so S_xy = A sin(k) cos(k y) / 2,
    |S| = |A sin(k) cos(k y)| and T_xy = cs^2 A^2 sin(k)^2 |cos(k y)| cos(k y); then
    a'_x(y) = (T_xy(y + 1) - T_xy(y - 1)) / 2 and a'_y = 0.
    """
    s1 = math.sin(k)

    def T(yy):
        """T_xy at rows yy."""
        c = torch.cos(k * yy)
        return cs * cs * A * A * s1 * s1 * c.abs() * c

    return 0.5 * (T(y + 1.0) - T(y - 1.0))
