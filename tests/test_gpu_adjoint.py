"""GPU adjoint (hand-written reverse of the step, behind torch.autograd.Function) against the
oracle gradient (autograd through the FP64 oracle) and against central finite differences.

Tolerances: FP64 storage rel-L2 <= 1e-10 against the oracle; FP32 rel-L2 <= 1e-4 against the
oracle on small cases (the stated GPU bound is 1e-2); directional derivative vs central FD of
the FP64 GPU forward <= 1e-6 (FP64) and <= 1e-2 (FP32) at the 128^3 workload size.
"""
import numpy as np
import pytest
import torch

import helpers as H
from oracle import adjoint as OA
from oracle.solver import OracleSim
from oracle.collision import Params
from paper_1202_6074_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__ as G

    G.build()
    from paper_1202_6074_gb300 import cmlbm, rollout

    return cmlbm, rollout


CASES = {
    "d3q27_periodic": dict(lattice="D3Q27", shape=(5, 6, 37), bc=("periodic",) * 3),
    "d3q27_walls": dict(lattice="D3Q27", shape=(4, 7, 9), bc=("periodic", "bounceback", "bounceback"),
                        wall_velocity=[[[0, 0, 0], [0, 0, 0]], [[0.02, 0, 0], [-0.01, 0, 0]], [[0, 0.01, 0], [0, 0, 0]]]),
    "d2q9_walls": dict(lattice="D2Q9", shape=(1, 9, 11), bc=("periodic", "bounceback", "periodic"),
                       wall_velocity=[[[0, 0, 0], [0, 0, 0]], [[0.03, 0, 0], [0.0, 0, 0]], [[0, 0, 0], [0, 0, 0]]]),
}


def _setup(cm, case, storage, steps_kw=None, unit_rates=False):
    nz, ny, nx = case["shape"]
    lat = case["lattice"]
    # unit higher-order rates select the adjoint's unit-rate kernel variant
    p = dict(tau=0.6, omega_3=1.0, omega_4=1.0) if unit_rates else dict(tau=0.6, omega_3=1.1, omega_4=0.9)
    rho, u = W.random_solenoidal(nx, ny, nz, seed=2, u_rms=0.03)
    F = W.gaussian_force(nx, ny, nz, seed=3, std=1e-3)
    target = W.gaussian_force(nx, ny, nz, seed=4, std=1e-2)
    if lat == "D2Q9":
        u[2] = 0
        F[2] = 0
        target[2] = 0
    uw = case.get("wall_velocity", H.zero_walls())
    s = cm.Solver(lattice=lat, nx=nx, ny=ny, nz=nz, storage=storage, bc=case["bc"], wall_velocity=uw, **p)
    s.set_force((0, 0, 0), torch.tensor(F, device="cuda"))
    s.init(torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"))
    s0 = s.get_state()
    return s, s0, F, target, uw, p


def _oracle_grad(case, s0_dev, F, target, uw, p, steps):
    nz, ny, nx = case["shape"]
    params = Params(tau=p["tau"], omega3=p["omega_3"], omega4=p["omega_4"])
    s0 = H.decode(s0_dev, case["lattice"])
    return OA.loss_and_grad((case["lattice"], nx, ny, nz, params), s0, torch.tensor(F), torch.tensor(target), steps,
                            {"bc": case["bc"], "wall_velocity": uw})


def _gpu_grad(rollout, s, s0, F, target, steps, segment):
    Fp = torch.tensor(F, device="cuda").requires_grad_(True)
    u = rollout.velocity_after(s, Fp, s0, steps, segment)
    L = ((u - torch.tensor(target, device="cuda")) ** 2).sum(0).mean()
    L.backward()
    return float(L), Fp.grad.detach().cpu()


@pytest.mark.parametrize("unit_rates", [False, True])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("f32", 1e-4)])
@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_matches_oracle_gradient(mods, name, storage, tol, unit_rates):
    cm, rollout = mods
    case = CASES[name]
    steps = 6
    s, s0, F, target, uw, p = _setup(cm, case, storage, unit_rates=unit_rates)
    Lg, gg = _gpu_grad(rollout, s, s0, F, target, steps, segment=4)
    Lo, go = _oracle_grad(case, s0, F, target, uw, p, steps)
    assert abs(Lg - Lo) <= 1e-12 + (1e-12 if storage == "f64" else 1e-6) * abs(Lo)
    if case["lattice"] == "D2Q9":
        gg, go = gg[:2], go[:2]
    err = H.rel_l2(gg, go)
    assert err < tol, f"rel-L2(grad) = {err:.3e}"
    s.close()


@pytest.mark.parametrize("storage,tol", [("f64", 1e-14), ("f32", 1e-6)])
def test_checkpoint_segment_does_not_change_gradient(mods, storage, tol):
    """The checkpoint interval changes only where the per-segment sums of the force gradient (in
    the arithmetic precision) are folded into the FP64 total: the gradients agree to the rounding
    of those sums (a few units of the arithmetic precision over at most seven terms)."""
    cm, rollout = mods
    case = CASES["d3q27_walls"]
    s, s0, F, target, _, _ = _setup(cm, case, storage)
    grads = [_gpu_grad(rollout, s, s0, F, target, 7, seg)[1] for seg in (1, 3, 7, 50)]
    for g in grads[1:]:
        assert H.rel_l2(g, grads[0]) < tol
    s.close()


def test_segment_accumulation_matches_fp64_accumulation(mods):
    """cmlbm_step_adjoint_segment (FP32 sums per segment, folded into FP64) against
    cmlbm_step_adjoint (FP64 accumulation every step) over one 6-step reverse sweep."""
    cm, _ = mods
    case = CASES["d3q27_periodic"]
    s, s0, F, target, _, _ = _setup(cm, case, "f32")
    states = [s0]
    for _ in range(6):
        nxt = s.new_state()
        s.step_buffers(states[-1], nxt)
        states.append(nxt)
    shape = (27,) + s.shape
    gen = torch.Generator(device="cuda").manual_seed(5)
    lam0 = torch.randn(shape, generator=gen, device="cuda", dtype=torch.float32)
    outs = []
    for mode in ("f64", "segment"):
        lam, lam2 = lam0.clone(), torch.empty_like(lam0)
        dLdF = torch.zeros((3,) + s.shape, dtype=torch.float64, device="cuda")
        seg = torch.zeros((3,) + s.shape, dtype=torch.float32, device="cuda")
        for t in reversed(range(6)):
            if mode == "f64":
                s.step_adjoint(states[t], lam, lam2, dLdF)
            else:
                s.step_adjoint_segment(states[t], lam, lam2, seg, dLdF, fold=(t in (0, 3)))
            lam, lam2 = lam2, lam
        outs.append((lam.clone(), dLdF.clone(), seg.clone()))
    assert torch.equal(outs[0][0], outs[1][0])           # the adjoint state itself is unchanged
    assert torch.count_nonzero(outs[1][2]).item() == 0   # the last fold leaves seg at zero
    assert H.rel_l2(outs[1][1], outs[0][1]) < 1e-6
    s.close()


@pytest.mark.parametrize("storage,steps,tol", [("f64", 20, 1e-6), ("f32", 500, 1e-2)])
def test_full_size_directional_derivative(mods, storage, steps, tol):
    """128^3 adjoint workload: <dL/dF, v> vs central differences of the FP64 GPU forward."""
    cm, rollout = mods
    n = 128
    rho, u0 = W.random_solenoidal(n, n, n, seed=2, u_rms=0.02)
    F = torch.tensor(W.gaussian_force(n, n, n, seed=3, std=1e-5), device="cuda")
    # the target comes from a run with a different seeded force
    ref = cm.Solver(lattice="D3Q27", nx=n, ny=n, nz=n, storage="f64", tau=0.6)
    ref.set_force((0, 0, 0), torch.tensor(W.gaussian_force(n, n, n, seed=4, std=1e-5), device="cuda"))
    ref.init(torch.tensor(rho, device="cuda"), torch.tensor(u0, device="cuda"))
    ref.step(steps)
    _, target = ref.moments()
    ref.close()

    s = cm.Solver(lattice="D3Q27", nx=n, ny=n, nz=n, storage=storage, tau=0.6)
    s.set_force((0, 0, 0), F)
    s.init(torch.tensor(rho, device="cuda"), torch.tensor(u0, device="cuda"))
    s0 = s.get_state()
    Fp = F.clone().requires_grad_(True)
    u = rollout.velocity_after(s, Fp, s0, steps, 50)
    ((u - target) ** 2).sum(0).mean().backward()
    g = Fp.grad.detach()
    s.close()

    # FP64 forward from the same (decoded) initial state for the finite differences
    f64 = cm.Solver(lattice="D3Q27", nx=n, ny=n, nz=n, storage="f64", tau=0.6)
    s0_64 = H.encode_f64(H.decode(s0, "D3Q27"), "D3Q27").to("cuda")
    gen = torch.Generator(device="cuda").manual_seed(11)
    v = torch.randn(F.shape, generator=gen, device="cuda", dtype=torch.float64) * 1e-5
    h = 1e-2

    def loss(Fx):
        f64.set_force((0, 0, 0), Fx)
        f64.set_state(s0_64)
        f64.step(steps)
        _, uu = f64.moments()
        return float(((uu - target) ** 2).sum(0).mean())

    fd = (loss(F + h * v) - loss(F - h * v)) / (2 * h)
    ad = float((g * v).sum())
    assert abs(ad - fd) <= tol * abs(fd), (ad, fd)
    f64.close()
