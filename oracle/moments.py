"""Raw and central moments, the binomial frame shift and the exact inverse transform.

Test infrastructure (see the package docstring).

Shapes: populations f[Q, ...], velocity u[3, ...] (u[2] = 0 in 2D), moments m[M, ...]
with M = Q and the moment index following ``lattice.monomials``.
"""
from math import comb

import torch

from .lattice import DT


def raw_moments(f, lat):
    """kappa'_a = sum_alpha f_alpha e_x^a0 e_y^a1 e_z^a2 (Sec. 9, Eq. rawmomentdistributionfunction1)."""
    out = []
    for (a0, a1, a2) in lat.monomials:
        acc = torch.zeros_like(f[0])
        for i in range(lat.Q):
            ex, ey, ez = (float(v) for v in lat.e[i])
            c = ex ** a0 * ey ** a1 * ez ** a2
            if c != 0.0:
                acc = acc + c * f[i]
        out.append(acc)
    return torch.stack(out)


def central_moments(f, u, lat):
    """kappa_a = sum_alpha f_alpha (e_x-u_x)^a0 (e_y-u_y)^a1 (e_z-u_z)^a2.

    Definition of Sec. 7 (Eqs. centralmomentdistributionfunction1 and the transformed
    version below Eq. centralmomentforcing), written out as an explicit sum over the
    directions; the third factor is the three-dimensional reading.
    """
    out = []
    for (a0, a1, a2) in lat.monomials:
        acc = torch.zeros_like(f[0])
        for i in range(lat.Q):
            ex, ey, ez = (float(v) for v in lat.e[i])
            term = f[i]
            if a0:
                term = term * (ex - u[0]) ** a0
            if a1:
                term = term * (ey - u[1]) ** a1
            if a2:
                term = term * (ez - u[2]) ** a2
            acc = acc + term
        out.append(acc)
    return torch.stack(out)


def central_to_raw(kappa, u, lat):
    """Binomial theorem of Sec. 9 (Eq. binomialtheorem), used in the rest-frame direction.

    Since e = (e - u) + u, the raw moment of exponent a is
        kappa'_a = sum_{b <= a} prod_d C(a_d, b_d) u_d^(a_d - b_d) kappa_b.
    """
    idx = {a: k for k, a in enumerate(lat.monomials)}
    out = []
    for a in lat.monomials:
        acc = torch.zeros_like(kappa[0])
        for b0 in range(a[0] + 1):
            for b1 in range(a[1] + 1):
                for b2 in range(a[2] + 1):
                    coef = comb(a[0], b0) * comb(a[1], b1) * comb(a[2], b2)
                    term = coef * kappa[idx[(b0, b1, b2)]]
                    if a[0] - b0:
                        term = term * u[0] ** (a[0] - b0)
                    if a[1] - b1:
                        term = term * u[1] ** (a[1] - b1)
                    if a[2] - b2:
                        term = term * u[2] ** (a[2] - b2)
                    acc = acc + term
        out.append(acc)
    return torch.stack(out)


def raw_to_populations(raw, lat):
    """Exact inverse through the orthogonal basis (Sec. 9, below Eq. sourceformulation1).

    The projections <K_beta|f> are combinations of raw monomial moments with the
    coefficients that define K_beta; then f = K D^-1 (K^T f) with D = diag(<K_beta|K_beta>).
    """
    mhat = torch.einsum("ba,a...->b...", lat.Kcoef, raw)
    D = (lat.K * lat.K).sum(0)
    return torch.einsum("ib,b...->i...", lat.K, mhat / D.view(-1, *([1] * (raw.dim() - 1))))


def central_to_populations(kappa, u, lat):
    """Populations with the given central moments about u: central -> raw -> K D^-1."""
    return raw_to_populations(central_to_raw(kappa, u, lat), lat)


def zeros_like_field(shape):
    """An FP64 zero field of the given shape."""
    return torch.zeros(shape, dtype=DT)
