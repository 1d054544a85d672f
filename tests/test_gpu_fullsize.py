"""GPU checks at the full workload sizes (the launch configurations bench.py times).

The oracle cannot run these grids, so:
  * one step is compared element-wise on sampled cells (all 27 populations of each cell; the
    pull of each sampled cell is done on the test side from the GPU's own input state and the
    oracle collides those cells);
  * the Taylor-Green energy decay at 256^3 over the stated 2000 steps is compared between the
    resting frame and a frame moving at U = (0.05, 0.03, 0) (Galilean invariance, the paper's
    central claim), GPU against GPU.
Reduced-size trajectories against the oracle cover the same configurations over many steps.
"""
import math

import numpy as np
import pytest
import torch

import helpers as H
from oracle.solver import collide_cells, OracleSim
from oracle.collision import Params
from oracle import les as OL
from paper_1202_6074_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ATOL = {"f32": 4e-6, "bf16": 4e-6, "f16": 4e-6}
RTOL = {"f32": 0.0, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}


@pytest.fixture(scope="module")
def cm():
    import __graft_entry__ as G

    G.build()
    from paper_1202_6074_gb300 import cmlbm

    return cmlbm


def _sampled_step(cm, s, lattice, params, bc, uw, F_at, cs_at=None, nsample=96, seed=0):
    """Step s once; compare sampled cells with the oracle collision of their pulled populations."""
    shape = s.shape
    cells = H.sample_cells(shape, nsample, seed)
    s0 = s.get_state()
    g = H.pull_sampled(s0, cells, lattice, bc, uw)
    del s0
    s.step(1)
    s1 = s.get_state()
    idx = torch.tensor(cells, device=s1.device)
    got = s1[:, idx[:, 0], idx[:, 1], idx[:, 2]].to("cpu", torch.float64)
    del s1
    w = H.lattice(lattice).w.view(-1, 1)
    got_f = w * (1.0 + got)
    F = F_at(cells)
    cs_eff = None if cs_at is None else cs_at(cells)
    ref = collide_cells(g, F, lattice, params, cs_eff)
    d_got, d_ref = got_f / w - 1, ref / w - 1
    storage = {torch.float32: "f32", torch.bfloat16: "bf16", torch.float16: "f16"}[s.state_dtype]
    tol = ATOL[storage] + RTOL[storage] * d_ref.abs()
    err = (d_got - d_ref).abs()
    assert bool((err <= tol).all()), f"max |dd| = {err.max().item():.3e}"


def test_tgv_256_fp32_sampled_step(cm):
    n = 256
    tau = 3 * 0.05 * (n / (2 * math.pi)) / 1600 + 0.5
    s = cm.Solver(lattice="D3Q27", nx=n, ny=n, nz=n, storage="f32", tau=tau, omega_bulk=1.0)
    rho, u = W.taylor_green(n, n, n, u0=0.05, xp=torch, device="cuda")
    s.init(rho, u)
    del rho, u
    s.step(5)
    p = Params(tau=tau, omega_bulk=1.0)
    zero = lambda cells: torch.zeros(3, len(cells), dtype=torch.float64)  # noqa: E731
    _sampled_step(cm, s, "D3Q27", p, ("periodic",) * 3, H.zero_walls(), zero)
    s.close()


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_hit_les_512_sampled_step(cm, storage):
    n = 512
    s = cm.Solver(lattice="D3Q27", nx=n, ny=n, nz=n, storage=storage, tau=0.5005, smagorinsky_cs=0.1, omega_bulk=1.0)
    F = W.hit_forcing(n, n, n, seed=1, xp=torch, device="cuda")
    s.set_force((0, 0, 0), F)
    s.init()
    s.step(5)
    p = Params(tau=0.5005, omega_bulk=1.0, cs_smag=0.1)

    def F_at(cells):
        idx = torch.tensor(cells, device=F.device)
        # the library keeps the field in FP32 for FP32/16-bit arithmetic
        return F[:, idx[:, 0], idx[:, 1], idx[:, 2]].float().double().cpu()

    _sampled_step(cm, s, "D3Q27", p, ("periodic",) * 3, H.zero_walls(), F_at)
    s.close()
    del F


def test_channel_1024_bf16_sampled_step(cm):
    nx, ny, nz = 1024, 256, 256
    u_tau, h = 0.005, ny / 2
    nu0 = u_tau * h / 180.0
    tau = 3 * nu0 + 0.5
    bc = ("periodic", "bounceback", "periodic")
    s = cm.Solver(lattice="D3Q27", nx=nx, ny=ny, nz=nz, storage="bf16", tau=tau, smagorinsky_cs=0.1,
                  van_driest=(26.0, u_tau / nu0), bc=bc, omega_bulk=1.0)
    Fx = u_tau * u_tau / h
    s.set_force((Fx, 0.0, 0.0))
    g = torch.Generator(device="cuda").manual_seed(5)
    y = (torch.arange(ny, device="cuda", dtype=torch.float64) + 0.5).view(1, ny, 1)
    shape = 6.0 * y * (ny - y) / ny ** 2
    u = 0.05 * 1.5 * 15.7 * u_tau * torch.randn((3, nz, ny, nx), generator=g, device="cuda", dtype=torch.float64) * (shape / 1.5)
    u[0] += 15.7 * u_tau * shape
    s.init(None, u)
    del u
    s.step(5)
    p = Params(tau=tau, omega_bulk=1.0, cs_smag=0.1)
    F_at = lambda cells: torch.tensor([[np.float32(Fx)], [0.0], [0.0]], dtype=torch.float64).expand(3, len(cells))  # noqa: E731
    cs_full = OL.van_driest_cs(0.1, ny, 1, 1, 26.0, u_tau / nu0)[0, :, 0]

    def cs_at(cells):
        return torch.stack([cs_full[c[1]] for c in cells])

    _sampled_step(cm, s, "D3Q27", p, bc, H.zero_walls(), F_at, cs_at)
    s.close()


def test_tgv_256_galilean_invariance_over_2000_steps(cm):
    """max_t |E(t) - E_U(t)| / E(0) <= 1e-3, E measured in the frame of the mean velocity."""
    n, steps, every = 256, 2000, 200
    tau = 3 * 0.05 * (n / (2 * math.pi)) / 1600 + 0.5
    curves = []
    for U in ((0.0, 0.0, 0.0), (0.05, 0.03, 0.0)):
        s = cm.Solver(lattice="D3Q27", nx=n, ny=n, nz=n, storage="f32", tau=tau, omega_bulk=1.0)
        rho, u = W.taylor_green(n, n, n, u0=0.05, background=U, xp=torch, device="cuda")
        s.init(rho, u)
        del rho, u
        E = []
        for _ in range(steps // every + 1):
            m = s.reduce()
            E.append(m[4] - 0.5 * (m[1] ** 2 + m[2] ** 2 + m[3] ** 2) / m[0])
            s.step(every)
        curves.append(np.array(E))
        s.close()
    dev = np.abs(curves[0] - curves[1]).max() / curves[0][0]
    print(f"TGV 256^3 Galilean invariance: max |dE| / E0 = {dev:.3e}")
    assert dev <= 1e-3
    assert curves[0][-1] < curves[0][0]          # it decays


# Reduced-size trajectories of the forced-LES and channel configurations (64^3 and
# 128 x 32 x 32, the sizes at which the oracle runs in well under a minute), 100 steps, against
# the FP64 oracle; 16-bit runs also against the error of their storage format alone (the oracle
# with the same rounding of its stored state). The bounds are those of helpers.check_16bit
# (2e-3 for 16-bit storage; the recorded BF16 misses where the format alone exceeds it).
_ORACLE = {}


def _hit_case():
    n, steps = 64, 100
    F = W.hit_forcing(n, n, n, seed=1, f_rms=5e-5)
    rho, u = W.random_solenoidal(n, n, n, seed=2, u_rms=0.03)
    kw = dict(tau=0.5005, smagorinsky_cs=0.1, omega_bulk=1.0)
    return dict(name="hit_les", shape=(n, n, n), steps=steps, rho=rho, u=u, F=F, uniform=None, kw=kw,
                oracle=dict(params=Params(tau=0.5005, omega_bulk=1.0, cs_smag=0.1)))


def _channel_case():
    nx, ny, nz, steps = 128, 32, 32, 100
    u_tau = 0.01
    nu0 = u_tau * (ny / 2) / 180.0
    tau = 3 * nu0 + 0.5
    rho, u, F = W.channel(nx, ny, nz, u_tau=u_tau, seed=5)
    bc = ("periodic", "bounceback", "periodic")
    kw = dict(tau=tau, smagorinsky_cs=0.1, van_driest=(26.0, u_tau / nu0), bc=bc, omega_bulk=1.0)
    return dict(name="channel", shape=(nz, ny, nx), steps=steps, rho=rho, u=u, F=None,
                uniform=(float(F[0, 0, 0, 0]), 0.0, 0.0), kw=kw,
                oracle=dict(params=Params(tau=tau, omega_bulk=1.0, cs_smag=0.1), bc=bc,
                            van_driest=(26.0, u_tau / nu0)))


def _oracle_u(case, storage):
    key = (case["name"], storage)
    if key not in _ORACLE:
        nz, ny, nx = case["shape"]
        oc = case["oracle"]
        o = OracleSim("D3Q27", nx, ny, nz, oc["params"], bc=oc.get("bc", ("periodic",) * 3),
                      van_driest=oc.get("van_driest"), storage=storage)
        if case["F"] is not None:
            o.set_force(field=torch.tensor(case["F"]))
        else:
            o.set_force(case["uniform"])
        o.init(torch.tensor(case["rho"]), torch.tensor(case["u"]))
        o.step(case["steps"])
        _ORACLE[key] = o.moments()[1]
    return _ORACLE[key]


def _gpu_u(cm, case, storage):
    nz, ny, nx = case["shape"]
    s = cm.Solver(lattice="D3Q27", nx=nx, ny=ny, nz=nz, storage=storage, **case["kw"])
    if case["F"] is not None:
        s.set_force((0, 0, 0), torch.tensor(case["F"], device="cuda"))
    else:
        s.set_force(case["uniform"])
    s.init(torch.tensor(case["rho"], device="cuda"), torch.tensor(case["u"], device="cuda"))
    s.step(case["steps"])
    _, ug = s.moments()
    s.close()
    return ug.cpu()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("make", [_hit_case, _channel_case], ids=["hit_les_64", "channel_128x32x32"])
def test_les_trajectory_reduced_size(cm, make, storage):
    case = make()
    ug = _gpu_u(cm, case, storage)
    uo = _oracle_u(case, None)
    u16 = _oracle_u(case, storage) if storage != "f32" else uo
    err = H.rel_l2(ug, uo)
    err_format = H.rel_l2(u16, uo)
    fmt = "" if storage == "f32" else f"; the {storage} format alone (oracle with {storage} storage) {err_format:.3e}"
    print(f"{case['name']} {case['shape']} x {case['steps']} {storage}: rel-L2(u) = {err:.3e}{fmt}")
    H.check_16bit(storage, case["name"], err, err_format)
