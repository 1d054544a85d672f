"""Velocity sets, rest weights, monomial orders and the orthogonal moment basis.

Test infrastructure (see the package docstring).

D2Q9 follows the paper's numbering (Sec. 2, Eq. velocityd2q9, with the direction order
fixed by the columns of the basis vectors |e_x>, |e_y>):
  0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
D3Q27 (paper silent; the paper says the procedure extends to three dimensions, Sec. 2
and Sec. 15) uses the lexicographic order i = 9*(ez+1) + 3*(ey+1) + (ex+1).

The orthogonal basis K for D2Q9 is built from the Gram-Schmidt combinations of
monomials printed in Sec. 2 (Eq. collisionmatrix1 and the list above it). For D3Q27 the
reading is the tensor product of the one-dimensional orthogonal set {1, e, 3e^2-2} on
{-1,0,1}, which reproduces the D2Q9 basis in two dimensions.
"""
from dataclasses import dataclass
import itertools

import torch

DT = torch.float64


@dataclass(frozen=True)
class Lattice:
    name: str
    d: int                      # spatial dimension of the velocity set (2 or 3)
    e: torch.Tensor             # [Q, 3] integer velocities (ez = 0 in 2D)
    w: torch.Tensor             # [Q] rest weights (f^eq at rho=1, u=0)
    opp: list                   # opposite direction of each i
    monomials: list             # list of exponent tuples (a, b, c), increasing total order
    K: torch.Tensor             # [Q, Q] columns = orthogonal basis vectors K_beta
    Kcoef: torch.Tensor         # [Q, nmono]: K_beta = sum_a Kcoef[beta, a] * e^a

    @property
    def Q(self):
        """Number of particle velocities."""
        return self.e.shape[0]


def _d2q9_velocities():
    """D2Q9 particle velocities in the order of the basis columns (Sec. 2, Eq. velocityd2q9)."""
    return [(0, 0, 0), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0),
            (1, 1, 0), (-1, 1, 0), (-1, -1, 0), (1, -1, 0)]


def _d3q27_velocities():
    """D3Q27 velocities {-1, 0, 1}^3 at index 9 (e_z + 1) + 3 (e_y + 1) + (e_x + 1) (3D reading of Sec. 2)."""
    v = [None] * 27
    for ez, ey, ex in itertools.product((-1, 0, 1), repeat=3):
        v[9 * (ez + 1) + 3 * (ey + 1) + (ex + 1)] = (ex, ey, ez)
    return v


def _weights(vel):
    """Rest weights w_alpha of the discrete Maxwellian at rho = 1, u = 0 (Sec. 4)."""
    # Textbook rest weights: products of the 1D weights (1/6, 2/3, 1/6) per axis.
    # Pinned by the test that the equilibrium at rho=1, u=0 reproduces them.
    w1 = {-1: 1.0 / 6.0, 0: 2.0 / 3.0, 1: 1.0 / 6.0}
    out = []
    for (ex, ey, ez) in vel:
        out.append(w1[ex] * w1[ey] * (w1[ez] if len(vel) == 27 else 1.0))
    return torch.tensor(out, dtype=DT)


def _opposites(vel):
    """Index of -e_alpha for every alpha (the bounce-back partner)."""
    idx = {v: i for i, v in enumerate(vel)}
    return [idx[(-a, -b, -c)] for (a, b, c) in vel]


# D2Q9 monomial order of Sec. 2: 1, x, y, (x^2, y^2 entering K3/K4), xy, x^2y, xy^2, x^2y^2.
D2Q9_MONOMIALS = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (2, 0, 0), (0, 2, 0),
                  (1, 1, 0), (2, 1, 0), (1, 2, 0), (2, 2, 0)]


def _d3q27_monomials():
    """The 27 monomials x^a y^b z^c, a, b, c in {0, 1, 2}, by increasing total order (3D reading of Sec. 2)."""
    m = list(itertools.product((0, 1, 2), repeat=3))
    m.sort(key=lambda a: (sum(a), a[::-1]))   # increasing total order
    return m


def _d2q9_K_coefficients():
    """The orthogonal basis of Sec. 2 written over the monomials D2Q9_MONOMIALS.

    K0 = 1; K1 = e_x; K2 = e_y; K3 = 3(e_x^2 + e_y^2) - 4; K4 = e_x^2 - e_y^2;
    K5 = e_x e_y; K6 = -3 e_x^2 e_y + 2 e_y; K7 = -3 e_x e_y^2 + 2 e_x;
    K8 = 9 e_x^2 e_y^2 - 6 (e_x^2 + e_y^2) + 4.
    Columns: [1, x, y, xx, yy, xy, xxy, xyy, xxyy].
    """
    c = torch.zeros(9, 9, dtype=DT)
    c[0, 0] = 1
    c[1, 1] = 1
    c[2, 2] = 1
    c[3, 3], c[3, 4], c[3, 0] = 3, 3, -4
    c[4, 3], c[4, 4] = 1, -1
    c[5, 5] = 1
    c[6, 6], c[6, 2] = -3, 2
    c[7, 7], c[7, 1] = -3, 2
    c[8, 8], c[8, 3], c[8, 4], c[8, 0] = 9, -6, -6, 4
    return c


def _d3q27_K_coefficients(monomials):
    """Tensor-product basis K_(b0,b1,b2) = p_b0(e_x) p_b1(e_y) p_b2(e_z) (reading for 3D).

    p_0 = 1, p_1 = e, p_2 = 3e^2 - 2; q[b][a] = coefficient of e^a in p_b.
    Basis vectors are indexed in the same order as the monomials.
    """
    q = [[1, 0, 0], [0, 1, 0], [-2, 0, 3]]
    n = len(monomials)
    c = torch.zeros(n, n, dtype=DT)
    for bi, b in enumerate(monomials):
        for ai, a in enumerate(monomials):
            c[bi, ai] = q[b[0]][a[0]] * q[b[1]][a[1]] * q[b[2]][a[2]]
    return c


def monomial_matrix(e, monomials):
    """P[a, i] = e_ix^a0 e_iy^a1 e_iz^a2 (the non-orthogonal basis of Sec. 2)."""
    P = torch.zeros(len(monomials), e.shape[0], dtype=DT)
    for ai, (a0, a1, a2) in enumerate(monomials):
        for i in range(e.shape[0]):
            ex, ey, ez = (float(v) for v in e[i])
            P[ai, i] = ex ** a0 * ey ** a1 * ez ** a2
    return P


def _build(name):
    """Velocities, weights, opposites, monomials and the orthogonal basis K of a lattice (Sec. 2)."""
    if name == "D2Q9":
        vel = _d2q9_velocities()
        mono = D2Q9_MONOMIALS
        coef = _d2q9_K_coefficients()
        d = 2
    elif name == "D3Q27":
        vel = _d3q27_velocities()
        mono = _d3q27_monomials()
        coef = _d3q27_K_coefficients(mono)
        d = 3
    else:
        raise ValueError(name)
    e = torch.tensor(vel, dtype=torch.int64)
    P = monomial_matrix(e, mono)
    K = (coef @ P).T.contiguous()      # K[i, beta] = sum_a coef[beta, a] P[a, i]
    return Lattice(name, d, e, _weights(vel), _opposites(vel), list(mono), K, coef)


D2Q9 = _build("D2Q9")
D3Q27 = _build("D3Q27")


def get(name):
    """The lattice object for \"D2Q9\" or \"D3Q27\"."""
    return {"D2Q9": D2Q9, "D3Q27": D3Q27}[name]


CS2 = 1.0 / 3.0   # c_s^2 (Sec. 4, below Eq. Maxwellian)
