"""Test-side helpers: decoding the library's state format and pulling sampled cells.

These restate the interface conventions of include/cmlbm.h (direction order, rest weights,
d = fbar / w - 1, pull with wrap or half-way bounce-back) in plain torch; they share no code
with the CUDA library or with the oracle's time loop.
"""
import numpy as np
import torch

from oracle import lattice as OL

DT = torch.float64


def lattice(name):
    return OL.get(name)


def decode(state, name):
    """[Q, ...] raw storage -> float64 populations fbar = w (1 + d) on the CPU."""
    lat = OL.get(name)
    d = state.detach().to("cpu", DT)
    w = lat.w.view(-1, *([1] * (d.dim() - 1)))
    return w * (1.0 + d)


def encode_f64(f, name):
    lat = OL.get(name)
    w = lat.w.view(-1, *([1] * (f.dim() - 1)))
    return f / w - 1.0


def rel_l2(a, b):
    a = torch.as_tensor(a, dtype=DT).cpu()
    b = torch.as_tensor(b, dtype=DT).cpu()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def sample_cells(shape, n, seed):
    nz, ny, nx = shape
    g = np.random.default_rng(seed)
    cells = set()
    # always include the corners and faces (walls / wrap), then random cells
    for z in (0, nz - 1):
        for y in (0, ny - 1):
            for x in (0, nx - 1):
                cells.add((z, y, x))
    while len(cells) < n:
        cells.add((int(g.integers(nz)), int(g.integers(ny)), int(g.integers(nx))))
    return sorted(cells)


def pull_sampled(state_dev, cells, name, bc, wall_velocity):
    """Pre-collision populations g_i(x) = s_i(x - e_i) (or bounce-back) at the given cells.

    state_dev: raw device state [Q, nz, ny, nx]. Returns float64 CPU tensor [Q, n].
    """
    lat = OL.get(name)
    Q = lat.Q
    nz, ny, nx = state_dev.shape[1:]
    n_by_axis = (nx, ny, nz)
    w = lat.w
    out = torch.empty(Q, len(cells), dtype=DT)
    for k, (z, y, x) in enumerate(cells):
        pos = (x, y, z)
        src_idx = []
        corr = []
        for i in range(Q):
            e = [int(v) for v in lat.e[i]]
            s = [pos[a] - e[a] for a in range(3)]
            crossed = []
            for a in range(3):
                if s[a] < 0 or s[a] >= n_by_axis[a]:
                    if bc[a] == "periodic":
                        s[a] %= n_by_axis[a]
                    else:
                        crossed.append((a, 0 if s[a] < 0 else 1))
            if crossed:
                uw = [sum(wall_velocity[a][sd][c] for a, sd in crossed) / len(crossed) for c in range(3)]
                eu = sum(e[c] * uw[c] for c in range(3))
                src_idx.append((lat.opp[i], z, y, x))
                corr.append(6.0 * eu)
            else:
                src_idx.append((i, s[2], s[1], s[0]))
                corr.append(0.0)
        idx = torch.tensor(src_idx, device=state_dev.device)
        vals = state_dev[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]].to("cpu", DT)
        d = vals + torch.tensor(corr, dtype=DT)
        out[:, k] = w * (1.0 + d)
    return out


def zero_walls():
    z = [0.0, 0.0, 0.0]
    return [[z, z], [z, z], [z, z]]


# Trajectory bounds against the FP64 oracle, on the velocity fluctuation u - U about the
# background U (the stricter measure; equal to rel-L2(u) at rest): 1e-5 for FP32 and 2e-3, the
# stated target, for 16-bit storage.
#
# A 16-bit run is also compared with the oracle whose stored state is rounded to the same format
# after every step (OracleSim(storage=...)): that oracle's own error against FP64 is what the
# storage format costs. The GPU run and that oracle round different values (FP32 against FP64
# arithmetic), so their rounding decisions decorrelate within a few steps, but their errors
# against FP64 must be statistically the same: |err - err_format| <= 20 % of err_format says
# the kernels add nothing the format does not. BF16 keeps 8 significant bits; where the format
# alone exceeds 2e-3 (a background flow, whose deviations the stored values carry too, or the
# 100-step LES runs), BF16 misses the target and BF16_MISS holds the bound asserted instead,
# next to the measured values.
TARGET = {"f32": 1e-5, "f16": 2e-3, "bf16": 2e-3}
BF16_MISS = {                 # case: (asserted bound, measured GPU error, measured format error)
    "tgv_moving_frame": (6e-3, 4.30e-3, 4.31e-3),
    "hit_les": (3.5e-3, 2.45e-3, 2.45e-3),
    "channel": (3e-3, 2.18e-3, 2.18e-3),
}
FORMAT_AGREEMENT = 0.2


def check_16bit(storage, case, err, err_format=None):
    """Assert the trajectory bounds for a storage type (see the comment above)."""
    if storage == "f32":
        assert err < TARGET["f32"], f"f32 {case}: rel-L2 = {err:.3e}"
        return
    assert err_format is not None
    assert abs(err - err_format) <= FORMAT_AGREEMENT * err_format, \
        f"{storage} {case}: GPU {err:.3e} against the {storage} format alone {err_format:.3e}"
    if storage == "bf16" and case in BF16_MISS:
        bound = BF16_MISS[case][0]
        assert err < bound, f"BF16 {case}: rel-L2 = {err:.3e} (bound {bound:.1e})"
        assert err_format > TARGET["bf16"], f"BF16 {case} now meets the 2e-3 target ({err:.3e}): update BF16_MISS"
        print(f"BF16 misses the 2e-3 target on {case}: rel-L2 = {err:.3e} (the storage format alone: {err_format:.3e})")
    else:
        assert err < TARGET[storage], f"{storage} {case}: rel-L2 = {err:.3e}"
