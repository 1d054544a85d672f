"""The D2Q9 collision exactly as printed, element by element (Secs. 9-11).

Test infrastructure (see the package docstring). This is a regression form; the normative
step is ``collision.collide``. Readings of the printed text:
  * Eq. rawmomentsourceterm4 prints sigma'_yy = 2 F_x u_y; by the x<->y symmetry of
    Eq. rawmomentsourceterm3 and of the projected source Eq. sourceterm4 it is 2 F_y u_y.
  * Eqs. collisionkernelg6/g7 write sigma_xxy, sigma_xyy without a prime inside the
    braces; the text after Eq. collisionkernelg8 says the raw source moments of
    Eqs. rawmomentsourceterm0-8 are the ones needed, so they are read as raw moments.
All arrays are float64 tensors with a trailing cell shape; F has at least two components.
"""
import torch


def collide_literal(fb, F, omega, sigma_central_in_g67=False, rho0=None, factorized=False):
    """Post-collision fbar by Eqs. collisionkernelg3-g8 and the element-wise update of Sec. 11.

    fb[9, ...] in the paper's direction order, F[>=2, ...], omega = (w3, w4, w5, w6, w7, w8).
    rho0: when given, the reduced-compressibility kernels of Sec. 12 (Eqs.
    collisionkernelcompact3-8) with rho0 u = sum fbar e + F/2. factorized: g8 with the
    factorized attractor of Sec. 13 (Eq. factorxxyyfinal, product as printed) in place of rho/9.
    Returns (fbar_post, g, S) with g = (g3..g8) and S[9, ...] (Eqs. vsourceterms0-8).
    """
    w3, w4, w5, w6, w7, w8 = omega
    Fx, Fy = F[0], F[1]
    f0, f1, f2, f3, f4, f5, f6, f7, f8 = (fb[i] for i in range(9))

    # Eqs. rawmomenttransformed0-2 and Eq. velocitycalculation
    rho = f0 + f1 + f2 + f3 + f4 + f5 + f6 + f7 + f8
    kx_r = f1 - f3 + f5 - f6 - f7 + f8
    ky_r = f2 - f4 + f5 + f6 - f7 - f8
    den = rho if rho0 is None else rho0
    ux = (kx_r + 0.5 * Fx) / den
    uy = (ky_r + 0.5 * Fy) / den
    # density factors of the kernels: rho (Sec. 10) or (rho0 - drho), (2 rho0 - drho), (3 rho0 - drho)
    if rho0 is None:
        r1 = r2 = r3 = rho
    else:
        drho = rho - rho0
        r1, r2, r3 = rho0 - drho, 2 * rho0 - drho, 3 * rho0 - drho

    # Eqs. rawmomenttransformed3-8 with the direction subsets A3..A8, B5..B7
    kxx_r = f1 + f3 + f5 + f6 + f7 + f8
    kyy_r = f2 + f4 + f5 + f6 + f7 + f8
    kxy_r = (f5 + f7) - (f6 + f8)
    kxxy_r = (f5 + f6) - (f7 + f8)
    kxyy_r = (f5 + f8) - (f6 + f7)
    kxxyy_r = f5 + f6 + f7 + f8

    # Eqs. kxxtransform - kxxytransform
    kxx = kxx_r + Fx * ux - rho * ux * ux
    kyy = kyy_r + Fy * uy - rho * uy * uy
    kxy = kxy_r + 0.5 * (Fx * uy + Fy * ux) - rho * ux * uy
    kxyy = kxyy_r - 2 * uy * kxy_r - ux * kyy_r - 0.5 * Fx * uy * uy - Fy * ux * uy + 2 * rho * ux * uy * uy
    kxxy = kxxy_r - 2 * ux * kxy_r - uy * kxx_r - 0.5 * Fy * ux * ux - Fx * ux * uy + 2 * rho * ux * ux * uy

    # Eqs. rawmomentsourceterm3-8 (sigma'_yy read as 2 F_y u_y)
    s_xx = 2 * Fx * ux
    s_yy = 2 * Fy * uy
    s_xy = Fx * uy + Fy * ux
    s_xxy = 2 * Fx * (kxy / rho + ux * uy) + Fy * (kxx / rho + ux * ux)
    s_xyy = Fx * (kyy / rho + uy * uy) + 2 * Fy * (kxy / rho + ux * uy)
    s_xxyy = (2 * Fx * ux * (kyy / rho + uy * uy) + 2 * Fy * uy * (kxx / rho + ux * ux)
              + 2 * Fx / rho * kxyy + 2 * Fy / rho * kxxy
              + Fx * Fx / rho ** 2 * kyy + Fy * Fy / rho ** 2 * kxx
              + 4 * (Fx * uy / rho + Fy * ux / rho + Fx * Fy / rho ** 2) * kxy)

    # Eqs. sourceterm0-8
    m1 = Fx
    m2 = Fy
    m3 = 6 * (Fx * ux + Fy * uy)
    m4 = 2 * (Fx * ux - Fy * uy)
    m5 = Fx * uy + Fy * ux
    m6 = -6 * Fx * (kxy / rho + ux * uy) - 3 * Fy * (kxx / rho + ux * ux - 2.0 / 3.0)
    m7 = -3 * Fx * (kyy / rho + uy * uy - 2.0 / 3.0) - 6 * Fy * (kxy / rho + ux * uy)
    m8 = (18 * Fx * ux * (kyy / rho + uy * uy - 2.0 / 3.0)
          + 18 * Fy * uy * (kxx / rho + ux * ux - 2.0 / 3.0)
          + 18 * Fx / rho * kxyy + 18 * Fy / rho * kxxy
          + 9 * Fx * Fx / rho ** 2 * kyy + 9 * Fy * Fy / rho ** 2 * kxx
          + 36 * (Fx * uy / rho + Fy * ux / rho + Fx * Fy / rho ** 2) * kxy)

    # Eqs. vsourceterms0-8
    S = torch.stack([
        (-m3 + m8) / 9.0,
        (6 * m1 - m3 + 9 * m4 + 6 * m7 - 2 * m8) / 36.0,
        (6 * m2 - m3 - 9 * m4 + 6 * m6 - 2 * m8) / 36.0,
        (-6 * m1 - m3 + 9 * m4 - 6 * m7 - 2 * m8) / 36.0,
        (-6 * m2 - m3 - 9 * m4 - 6 * m6 - 2 * m8) / 36.0,
        (6 * m1 + 6 * m2 + 2 * m3 + 9 * m5 - 3 * m6 - 3 * m7 + m8) / 36.0,
        (-6 * m1 + 6 * m2 + 2 * m3 - 9 * m5 - 3 * m6 + 3 * m7 + m8) / 36.0,
        (-6 * m1 - 6 * m2 + 2 * m3 + 9 * m5 + 3 * m6 + 3 * m7 + m8) / 36.0,
        (6 * m1 - 6 * m2 + 2 * m3 - 9 * m5 + 3 * m6 - 3 * m7 + m8) / 36.0,
    ])

    if sigma_central_in_g67:
        # alternative reading: central source moments (Eq. centralmomentforcingtransformed)
        sg6 = 2 * Fx / rho * kxy + Fy / rho * kxx
        sg7 = Fx / rho * kyy + 2 * Fy / rho * kxy
    else:
        sg6, sg7 = s_xxy, s_xyy

    # Eqs. collisionkernelg3-g8 (Eqs. collisionkernelcompact3-8 with rho0)
    g3 = w3 / 12.0 * (2.0 / 3.0 * rho + r1 * (ux * ux + uy * uy) - (kxx_r + kyy_r) - 0.5 * (s_xx + s_yy))
    g4 = w4 / 4.0 * (r1 * (ux * ux - uy * uy) - (kxx_r - kyy_r) - 0.5 * (s_xx - s_yy))
    g5 = w5 / 4.0 * (r1 * ux * uy - kxy_r - 0.5 * s_xy)
    g6 = (w6 / 4.0 * ((r2 if rho0 is not None else 2 * rho) * ux * ux * uy + kxxy_r - 2 * ux * kxy_r - uy * kxx_r
                      - 0.5 * sg6)
          - 0.5 * uy * (3 * g3 + g4) - 2 * ux * g5)
    g7 = (w7 / 4.0 * ((r2 if rho0 is not None else 2 * rho) * ux * uy * uy + kxyy_r - 2 * uy * kxy_r - ux * kyy_r
                      - 0.5 * sg7)
          - 0.5 * ux * (3 * g3 - g4) - 2 * uy * g5)
    if factorized:
        # Eq. factorxxyyfinal (and its reduced-compressibility form)
        att = ((kxx_r - r1 * ux * ux + Fx * ux + (6 * g3 + 2 * g4))
               * (kyy_r - r1 * uy * uy + Fy * uy + (6 * g3 - 2 * g4))
               - Fx / rho * kxyy - Fy / rho * kxxy - Fy * Fy / (2 * rho ** 2) * kxx - Fx * Fx / (2 * rho ** 2) * kyy
               - 2 * Fx * Fy / rho ** 2 * kxy)
    else:
        att = rho / 9.0
    g8 = (w8 / 4.0 * (att + (r3 if rho0 is not None else 3 * rho) * ux * ux * uy * uy
                      - (kxxyy_r - 2 * ux * kxyy_r - 2 * uy * kxxy_r + ux * ux * kyy_r + uy * uy * kxx_r
                         + 4 * ux * uy * kxy_r)
                      - 0.5 * s_xxyy)
          - 2 * g3 - 0.5 * uy * uy * (3 * g3 + g4) - 0.5 * ux * ux * (3 * g3 - g4)
          - 4 * ux * uy * g5 - 2 * uy * g6 - 2 * ux * g7)

    # element-wise update of Sec. 11 (g0 = g1 = g2 = 0, collision invariants)
    post = torch.stack([
        f0 + (-4 * (g3 - g8)) + S[0],
        f1 + (-g3 + g4 + 2 * (g7 - g8)) + S[1],
        f2 + (-g3 - g4 + 2 * (g6 - g8)) + S[2],
        f3 + (-g3 + g4 - 2 * (g7 + g8)) + S[3],
        f4 + (-g3 - g4 - 2 * (g6 + g8)) + S[4],
        f5 + (2 * g3 + g5 - g6 - g7 + g8) + S[5],
        f6 + (2 * g3 - g5 - g6 + g7 + g8) + S[6],
        f7 + (2 * g3 + g5 + g6 + g7 + g8) + S[7],
        f8 + (2 * g3 - g5 + g6 - g7 + g8) + S[8],
    ])
    return post, (g3, g4, g5, g6, g7, g8), S
