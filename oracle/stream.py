"""Streaming with periodic and half-way bounce-back boundaries; the initial state.

Test infrastructure (see the package docstring).

The paper uses the standard streaming step (Sec. 6 after Eq. cascadedLBE3; Eq.
cascadedstreaming1). Boundaries are paper silent. Readings used here:

* The stored state s_i(x) is the post-collision transformed population of cell x. One step
  pulls g_i(x) = s_i(x - e_i) (this is Eq. cascadedstreaming1) and collides g.
* Periodic axes wrap the index.
* On a bounce-back axis the walls sit half-way outside the first and last cells. When
  x - e_i is behind a wall, g_i(x) = s_ibar(x) + 2 w_i rho_w (e_i . u_w) / c_s^2 with
  rho_w = 1 and u_w the velocity of the crossed wall (the mean of the walls' velocities
  where an edge link crosses two).
* The initial state is chosen so that the first pull returns the requested pre-collision
  field fbar(x, 0) exactly: s_i(x) = fbar_i(x + e_i), or the reflected value at a wall.
"""
import torch

from .lattice import DT

PERIODIC = "periodic"
BOUNCEBACK = "bounceback"


def _coord(n, shape_axis, ndim=3):
    """Integer coordinates 0 .. n-1 along one axis of a [nz, ny, nx] field, broadcastable."""
    view = [1, 1, 1]
    view[shape_axis] = n
    return torch.arange(n).view(*view)


def _wall_terms(lat, i, shape, bc, wall_velocity, sign):
    """Mask of cells whose link x + sign*e_i... crosses a wall, and the mean wall velocity there.

    sign = -1: the pull source x - e_i; sign = +1: the push target x + e_i.
    Returns (mask[nz,ny,nx] bool, uw[3,nz,ny,nx]).
    """
    nz, ny, nx = shape
    n_by_axis = (nx, ny, nz)
    grid_axis = (2, 1, 0)     # tensor dim of axis x, y, z
    mask = torch.zeros(shape, dtype=torch.bool)
    count = torch.zeros(shape, dtype=DT)
    uw = torch.zeros((3,) + tuple(shape), dtype=DT)
    for ax in range(3):
        if bc[ax] != BOUNCEBACK:
            continue
        c = int(lat.e[i, ax]) * sign
        if c == 0:
            continue
        n = n_by_axis[ax]
        coord = _coord(n, grid_axis[ax]).expand(shape)
        if c < 0:      # neighbour below index 0 -> lower wall
            hit = coord == 0
            side = 0
        else:          # neighbour above n-1 -> upper wall
            hit = coord == n - 1
            side = 1
        mask = mask | hit
        count = count + hit.to(DT)
        for d in range(3):
            uw[d] = uw[d] + hit.to(DT) * wall_velocity[ax][side][d]
    uw = uw / torch.clamp(count, min=1.0)
    return mask, uw


def pull(s, lat, bc, wall_velocity):
    """g_i(x) = s_i(x - e_i), or the bounce-back value when x - e_i is behind a wall."""
    shape = s.shape[1:]
    g = torch.empty_like(s)
    for i in range(lat.Q):
        ex, ey, ez = (int(v) for v in lat.e[i])
        shifted = torch.roll(s[i], shifts=(ez, ey, ex), dims=(0, 1, 2))
        mask, uw = _wall_terms(lat, i, shape, bc, wall_velocity, sign=-1)
        if mask.any():
            eu = sum(float(lat.e[i, d]) * uw[d] for d in range(3))
            bounced = s[lat.opp[i]] + 6.0 * float(lat.w[i]) * eu
            g[i] = torch.where(mask, bounced, shifted)
        else:
            g[i] = shifted
    return g


def unstream(fbar, lat, bc, wall_velocity):
    """Inverse of ``pull``: the state whose pull gives fbar."""
    shape = fbar.shape[1:]
    s = torch.empty_like(fbar)
    for i in range(lat.Q):
        ex, ey, ez = (int(v) for v in lat.e[i])
        shifted = torch.roll(fbar[i], shifts=(-ez, -ey, -ex), dims=(0, 1, 2))
        mask, uw = _wall_terms(lat, i, shape, bc, wall_velocity, sign=+1)
        if mask.any():
            eu = sum(float(lat.e[i, d]) * uw[d] for d in range(3))
            refl = fbar[lat.opp[i]] + 6.0 * float(lat.w[i]) * eu
            s[i] = torch.where(mask, refl, shifted)
        else:
            s[i] = shifted
    return s
