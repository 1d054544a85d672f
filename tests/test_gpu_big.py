"""Grids with 27 N >= 2^32 state elements (64-bit element offsets).

Each case steps a D3Q27 grid just above the limit and compares sampled cells of one step with
the oracle collision of their pulled populations (as tests/test_gpu_fullsize.py does at the
workload sizes), including the corner cells, whose last direction planes lie beyond element
2^32; the FP64 reductions and the moments of the whole grid are checked against each other.
"""
import math

import pytest
import torch

import helpers as H
from oracle.collision import Params
from oracle.solver import collide_cells
from paper_1202_6074_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ATOL = {"f64": 1e-13, "f32": 4e-6, "bf16": 4e-6, "f16": 4e-6}
RTOL = {"f64": 0.0, "f32": 0.0, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}


@pytest.fixture(scope="module")
def cm():
    import __graft_entry__ as G

    G.build()
    from paper_1202_6074_gb300 import cmlbm

    return cmlbm


def _sampled_step(s, storage, params, bc, F_at, cs_at=None, nsample=64, seed=0):
    cells = H.sample_cells(s.shape, nsample, seed)
    s0 = s.get_state()
    g = H.pull_sampled(s0, cells, "D3Q27", bc, H.zero_walls())
    del s0
    s.step(1)
    s1 = s.get_state()
    idx = torch.tensor(cells, device=s1.device)
    got = s1[:, idx[:, 0], idx[:, 1], idx[:, 2]].to("cpu", torch.float64)
    del s1
    torch.cuda.empty_cache()
    w = H.lattice("D3Q27").w.view(-1, 1)
    ref = collide_cells(g, F_at(cells), "D3Q27", params, None if cs_at is None else cs_at(cells))
    d_ref = ref / w - 1
    err = (got - d_ref).abs()
    tol = ATOL[storage] + RTOL[storage] * d_ref.abs()
    assert bool((err <= tol).all()), f"max |dd| = {err.max().item():.3e}"


def _reduce_vs_moments(s, tol):
    red = s.reduce()
    rho, u = s.moments()
    mass = float(rho.sum())
    assert abs(red[0] - mass) <= tol * mass
    assert all(math.isfinite(v) for v in red)
    del rho, u
    torch.cuda.empty_cache()


def _zero_force(cells):
    return torch.zeros(3, len(cells), dtype=torch.float64)


@pytest.mark.parametrize("storage", ["bf16", "f32"])
def test_large_grid_unforced_step(cm, storage):
    """Taylor-Green vortex on 1024 x 1024 x 152 (27 N = 4.30e9): the unforced pair kernel."""
    nx, ny, nz = 1024, 1024, 152
    assert 27 * nx * ny * nz >= 2 ** 32
    tau = 0.52
    s = cm.Solver(lattice="D3Q27", nx=nx, ny=ny, nz=nz, storage=storage, tau=tau, omega_bulk=1.0)
    assert s.step_kernel == "pair"
    rho, u = W.taylor_green(nx, ny, nz, u0=0.05, background=(0.01, 0.0, 0.0), xp=torch, device="cuda")
    s.init(rho, u)
    del rho, u
    s.step(2)
    _sampled_step(s, storage, Params(tau=tau, omega_bulk=1.0), ("periodic",) * 3, _zero_force)
    _reduce_vs_moments(s, 1e-12)
    s.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("form", ["les_field", "factorized"])
def test_large_grid_forced_bf16_step(cm, form):
    """The forced isotropic-turbulence LES (force field, Smagorinsky) and the factorized
    attractor with a uniform force, BF16 storage on 576^3 (27 N = 5.16e9)."""
    n = 576
    if form == "les_field":
        kw = dict(tau=0.5005, smagorinsky_cs=0.1, omega_bulk=1.0)
        p = Params(tau=0.5005, omega_bulk=1.0, cs_smag=0.1)
    else:
        kw = dict(tau=0.55, omega_bulk=1.0, attractor="factorized")
        p = Params(tau=0.55, omega_bulk=1.0, attractor="factorized")
    s = cm.Solver(lattice="D3Q27", nx=n, ny=n, nz=n, storage="bf16", **kw)
    if form == "les_field":
        F = W.hit_forcing(n, n, n, seed=1, xp=torch, device="cuda")
        s.set_force((0, 0, 0), F)
        s.init()

        def F_at(cells):
            idx = torch.tensor(cells, device=F.device)
            return F[:, idx[:, 0], idx[:, 1], idx[:, 2]].float().double().cpu()
    else:
        Fu = (1e-6, -2e-6, 5e-7)
        s.set_force(Fu)
        rho, u = W.taylor_green(n, n, n, u0=0.04, xp=torch, device="cuda")
        s.init(rho, u)
        del rho, u

        def F_at(cells):
            return torch.tensor([[float(torch.tensor(v, dtype=torch.float32))] for v in Fu],
                                dtype=torch.float64).expand(3, len(cells))
    s.step(2)
    _sampled_step(s, "bf16", p, ("periodic",) * 3, F_at)
    _reduce_vs_moments(s, 1e-12)
    s.close()
    if form == "les_field":
        del F
    torch.cuda.empty_cache()


def test_large_grid_fp64_channel_step(cm):
    """FP64 storage (the one-cell kernel) on a 1024 x 1024 x 152 channel with y walls, a uniform
    force and the eddy viscosity."""
    nx, ny, nz = 1024, 1024, 152
    bc = ("periodic", "bounceback", "periodic")
    kw = dict(tau=0.52, smagorinsky_cs=0.1, omega_bulk=1.0, bc=bc)
    s = cm.Solver(lattice="D3Q27", nx=nx, ny=ny, nz=nz, storage="f64", **kw)
    assert s.step_kernel == "direct"
    Fu = (2e-7, 0.0, 0.0)
    s.set_force(Fu)
    y = (torch.arange(ny, device="cuda", dtype=torch.float64) + 0.5).view(1, ny, 1)
    u = torch.zeros((3, nz, ny, nx), device="cuda", dtype=torch.float64)
    u[0] += 0.04 * 4 * y * (ny - y) / ny ** 2
    s.init(None, u)
    del u
    s.step(2)
    p = Params(tau=0.52, omega_bulk=1.0, cs_smag=0.1)
    F_at = lambda cells: torch.tensor([[v] for v in Fu], dtype=torch.float64).expand(3, len(cells))  # noqa: E731
    _sampled_step(s, "f64", p, bc, F_at)
    _reduce_vs_moments(s, 1e-12)
    s.close()
    torch.cuda.empty_cache()
