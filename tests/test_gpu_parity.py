"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU oracle.

Tolerances (derived from the arithmetic):
  * FP64 storage (FP64 arithmetic): element-wise |d_gpu - d_oracle| <= 1e-13 after one step,
    trajectories rel-L2 <= 1e-11.
  * FP32: one step element-wise |d_gpu - d_oracle| <= 4e-6 (about 1000 FP32 operations on
    O(0.1) quantities); trajectories rel-L2(u) <= 1e-5 (the stated target).
  * BF16 / FP16 storage: one step |d_gpu - d_oracle| <= |d| 2^-8 (2^-11) + 4e-6, i.e. one
    rounding of the stored deviation; trajectories rel-L2(u) <= 2e-3 (the stated target).
"""
import math

import numpy as np
import pytest
import torch

import helpers as H
from oracle.solver import OracleSim
from oracle.collision import Params
from paper_1202_6074_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ONE_STEP_ATOL = {"f64": 1e-13, "f32": 4e-6, "bf16": 4e-6, "f16": 4e-6}
ONE_STEP_RTOL = {"f64": 0.0, "f32": 0.0, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}


@pytest.fixture(scope="module")
def cm():
    import __graft_entry__ as G

    G.build()
    from paper_1202_6074_gb300 import cmlbm

    assert torch.cuda.is_available()
    return cmlbm


def _params(kw):
    return Params(tau=kw.get("tau", 0.8), omega_bulk=kw.get("omega_bulk", 0.0), omega3=kw.get("omega_3", 1.0),
                  omega4=kw.get("omega_4", 1.0), cs_smag=kw.get("smagorinsky_cs", 0.0),
                  attractor=kw.get("attractor", "maxwell"),
                  reduced_compressibility=kw.get("reduced_compressibility", False), rho0=kw.get("rho0", 1.0))


def _pair(cm, lattice, shape, storage, rho, u, F=None, uniform=(0.0, 0.0, 0.0), **kw):
    nz, ny, nx = shape
    bc = kw.get("bc", ("periodic",) * 3)
    uw = kw.get("wall_velocity", H.zero_walls())
    s = cm.Solver(lattice=lattice, nx=nx, ny=ny, nz=nz, storage=storage, **kw)
    s.set_force(uniform, None if F is None else torch.tensor(F, device="cuda"))
    s.init(None if rho is None else torch.tensor(rho, device="cuda"), None if u is None else torch.tensor(u, device="cuda"))
    o = OracleSim(lattice, nx, ny, nz, _params(kw), bc=bc, wall_velocity=uw, van_driest=kw.get("van_driest"))
    o.set_force(uniform, None if F is None else torch.tensor(F))
    o.init(None if rho is None else torch.tensor(rho), None if u is None else torch.tensor(u))
    return s, o


CASES = {
    "periodic_tgv": dict(lattice="D3Q27", shape=(7, 10, 150), flow="tgv", kw=dict(tau=0.62, omega_3=1.2, omega_4=0.9)),
    "walls_les_field": dict(lattice="D3Q27", shape=(6, 9, 37), flow="channel",
                            kw=dict(tau=0.52, smagorinsky_cs=0.15, van_driest=(26.0, 8.0),
                                    bc=("periodic", "bounceback", "periodic"),
                                    wall_velocity=[[[0, 0, 0], [0, 0, 0]], [[0.02, 0, 0.01], [-0.03, 0.0, 0.0]],
                                                   [[0, 0, 0], [0, 0, 0]]])),
    "all_walls_bulk": dict(lattice="D3Q27", shape=(5, 6, 7), flow="tgv",
                           kw=dict(tau=0.7, omega_bulk=1.3, bc=("bounceback",) * 3,
                                   wall_velocity=[[[0, 0.01, 0], [0, 0, 0.02]], [[0.03, 0, 0], [0, 0, -0.01]],
                                                  [[0.01, 0.01, 0], [-0.02, 0, 0]]])),
    "d2q9_channel": dict(lattice="D2Q9", shape=(1, 12, 140), flow="channel",
                         kw=dict(tau=0.8, omega_3=8.0 / 9.0, bc=("periodic", "bounceback", "periodic"),
                                 wall_velocity=[[[0, 0, 0], [0, 0, 0]], [[0.05, 0, 0], [0.05, 0, 0]], [[0, 0, 0], [0, 0, 0]]])),
    "d2q9_les_tgv": dict(lattice="D2Q9", shape=(1, 33, 31), flow="tgv", kw=dict(tau=0.55, smagorinsky_cs=0.2)),
    "factorized": dict(lattice="D3Q27", shape=(6, 5, 40), flow="tgv",
                       kw=dict(tau=0.58, omega_3=1.1, omega_4=1.3, attractor="factorized")),
    "reduced": dict(lattice="D3Q27", shape=(5, 8, 33), flow="channel",
                    kw=dict(tau=0.6, reduced_compressibility=True, rho0=1.0, bc=("periodic", "bounceback", "periodic"))),
    "d2q9_factorized_reduced": dict(lattice="D2Q9", shape=(1, 17, 36), flow="tgv",
                                    kw=dict(tau=0.7, attractor="factorized", reduced_compressibility=True, rho0=1.01)),
    # no force and omega_3 = omega_4 = 1: the kernels' SIMPLE variant (one cell / two cells per thread)
    "unforced_unit_rates": dict(lattice="D3Q27", shape=(5, 7, 45), flow="tgv_unforced", kw=dict(tau=0.56, omega_bulk=1.1)),
    "unforced_unit_rates_pair_walls_les": dict(lattice="D3Q27", shape=(6, 8, 128), flow="tgv_unforced",
                                               kw=dict(tau=0.51, smagorinsky_cs=0.12,
                                                       bc=("periodic", "bounceback", "bounceback"),
                                                       wall_velocity=[[[0, 0, 0], [0, 0, 0]], [[0.02, 0, 0], [0, 0, 0]],
                                                                      [[0, 0, 0.01], [0, -0.02, 0]]])),
    "d2q9_unforced_unit_rates": dict(lattice="D2Q9", shape=(1, 20, 30), flow="tgv_unforced", kw=dict(tau=0.6)),
    # tiny and degenerate boxes: 4^3 periodic, an odd 3 x 5 x 7 box with walls on every axis, and
    # a channel one cell thick between its walls (both y links of every cell bounce back)
    "tiny_periodic_4cube": dict(lattice="D3Q27", shape=(4, 4, 4), flow="tgv", kw=dict(tau=0.6)),
    "tiny_odd_all_walls": dict(lattice="D3Q27", shape=(7, 5, 3), flow="tgv", kw=dict(tau=0.65, bc=("bounceback",) * 3)),
    "one_cell_thick_channel": dict(lattice="D3Q27", shape=(6, 1, 8), flow="channel",
                                   kw=dict(tau=0.7, bc=("periodic", "bounceback", "periodic"))),
}


def _inputs(case):
    nz, ny, nx = case["shape"]
    two_d = case["lattice"] == "D2Q9"
    if case["flow"] in ("tgv", "tgv_unforced"):
        rho, u = W.taylor_green(nx, ny, nz, u0=0.05, background=(0.02, -0.01, 0.0 if two_d else 0.015), two_d=two_d)
        F = W.gaussian_force(nx, ny, nz, seed=3, std=1e-4) if case["flow"] == "tgv" else None
    else:
        rho, u, F = W.channel(nx, ny, nz, u_tau=0.01, seed=5)
        F = F + W.gaussian_force(nx, ny, nz, seed=4, std=1e-5)
    if two_d:
        u[2] = 0.0
        if F is not None:
            F[2] = 0.0
    return rho, u, F


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("name", list(CASES))
def test_one_step_elementwise(cm, name, storage):
    case = CASES[name]
    rho, u, F = _inputs(case)
    s, o = _pair(cm, case["lattice"], case["shape"], storage, rho, u, F, **case["kw"])
    # both sides start from the same (GPU-encoded) state
    s0 = s.get_state()
    o.set_state(H.decode(s0, case["lattice"]))
    s.step(1)
    o.step(1)
    got = H.decode(s.get_state(), case["lattice"])
    ref = o.s
    lat = H.lattice(case["lattice"])
    w = lat.w.view(-1, 1, 1, 1)
    d_got, d_ref = got / w - 1, ref / w - 1
    tol = ONE_STEP_ATOL[storage] + ONE_STEP_RTOL[storage] * d_ref.abs()
    err = (d_got - d_ref).abs()
    assert bool((err <= tol).all()), f"max |dd| = {err.max().item():.3e}"
    s.close()


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("name", ["periodic_tgv", "walls_les_field", "all_walls_bulk", "d2q9_channel"])
def test_init_returns_requested_fields(cm, name, storage):
    case = CASES[name]
    rho, u, F = _inputs(case)
    s, _ = _pair(cm, case["lattice"], case["shape"], storage, rho, u, F, **case["kw"])
    r, uu = s.moments()
    tol = {"f64": 1e-14, "f32": 1e-6, "bf16": 3e-3, "f16": 5e-4}[storage]
    assert (r.cpu() - torch.tensor(rho)).abs().max().item() < tol
    assert (uu.cpu() - torch.tensor(u)).abs().max().item() < tol * 0.2 + 1e-15
    s.close()


@pytest.mark.parametrize("name", list(CASES))
def test_trajectory_fp64(cm, name):
    case = CASES[name]
    rho, u, F = _inputs(case)
    s, o = _pair(cm, case["lattice"], case["shape"], "f64", rho, u, F, **case["kw"])
    s.step(20)
    o.step(20)
    rg, ug = s.moments()
    ro, uo = o.moments()
    assert H.rel_l2(ug, uo) < 1e-11
    assert (rg.cpu() - ro).abs().max().item() < 1e-13
    s.close()


@pytest.mark.parametrize("background", [(0.0, 0.0, 0.0), (0.05, 0.03, 0.0)])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_trajectory_reduced_precision_tgv(cm, storage, background):
    """D3Q27 Taylor-Green 24^3, optional background velocity, force field, 60 steps."""
    n = 24
    rho, u = W.taylor_green(n, n, n, u0=0.05, background=background)
    F = W.gaussian_force(n, n, n, seed=3, std=1e-5)
    s, o = _pair(cm, "D3Q27", (n, n, n), storage, rho, u, F, tau=0.55)
    o16 = OracleSim("D3Q27", n, n, n, _params(dict(tau=0.55)), storage=storage)
    o16.set_force((0, 0, 0), torch.tensor(F))
    o16.init(torch.tensor(rho), torch.tensor(u))
    s.step(60)
    o.step(60)
    o16.step(60)
    _, ug = s.moments()
    _, uo = o.moments()
    _, u16 = o16.moments()
    bg = torch.tensor(background, dtype=torch.float64).view(3, 1, 1, 1)
    ug = ug.cpu() - bg
    err = H.rel_l2(ug, uo - bg)
    err_format = H.rel_l2(u16 - bg, uo - bg)
    print(f"{storage} U={background}: rel-L2(u - U) = {err:.3e}; the {storage} format alone (oracle with "
          f"{storage} storage) {err_format:.3e}")
    case = "tgv_moving_frame" if any(background) else "tgv_rest"
    H.check_16bit(storage, case, err, err_format)
    s.close()


def test_poiseuille_cfg1_fp64_matches_oracle_and_closed_form(cm):
    """64 x 32 D2Q9 FP64 body-force channel, tau = 0.8, F = 1e-6, 5000 steps; and the rerun with
    walls and fluid moving at U = 0.05 (Galilean invariance)."""
    nx, ny, F, tau, steps = 64, 32, 1e-6, 0.8, 5000
    nu = (tau - 0.5) / 3
    bc = ("periodic", "bounceback", "periodic")
    res = {}
    for U in (0.0, 0.05):
        uw = [[[0, 0, 0], [0, 0, 0]], [[U, 0, 0], [U, 0, 0]], [[0, 0, 0], [0, 0, 0]]]
        rho, u = W.rest(nx, ny, 1, background=(U, 0, 0))
        s, o = _pair(cm, "D2Q9", (1, ny, nx), "f64", rho, u, None, uniform=(F, 0, 0), tau=tau, bc=bc, wall_velocity=uw)
        s.step(steps)
        o.step(steps)
        _, ug = s.moments()
        _, uo = o.moments()
        assert H.rel_l2(ug.cpu() - U, uo - U) < 1e-10
        res[U] = ug.cpu()[0, 0, :, 0].numpy() - U
        s.close()
    # start-up closed form (series), eta = y + 1/2, H = ny
    eta = np.arange(ny) + 0.5
    H_ = float(ny)
    ref = F / (2 * nu) * eta * (H_ - eta)
    for n in range(1, 200, 2):
        ref -= 4 * F * H_ ** 2 / (nu * math.pi ** 3 * n ** 3) * np.sin(n * math.pi * eta / H_) * math.exp(
            -n * n * math.pi ** 2 * nu * steps / H_ ** 2)
    assert np.abs(res[0.0] - ref).max() / ref.max() < 1e-2
    assert np.abs(res[0.05] - res[0.0]).max() / ref.max() < 1e-3


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_reduce_matches_compensated_sum(cm, storage):
    n = (19, 23, 130)
    rho, u = W.taylor_green(n[2], n[1], n[0], u0=0.05, background=(0.01, 0.02, 0.03))
    s, _ = _pair(cm, "D3Q27", n, storage, rho, u, None, uniform=(1e-5, 0, 0), tau=0.6)
    s.step(3)
    red = s.reduce()
    r, uu = s.moments()
    r = r.cpu().numpy().ravel()
    uu = uu.cpu().numpy().reshape(3, -1)
    ref = [math.fsum(r), math.fsum(r * uu[0]), math.fsum(r * uu[1]), math.fsum(r * uu[2]),
           math.fsum(0.5 * r * (uu ** 2).sum(0))]
    for k in range(5):
        if k in (1, 2, 3) and storage == "f32":
            # the library sums the momentum j itself; rho u from the FP32 moments carries the
            # rounding of u = j / rho (a few FP32 ulps of each cell's |j|)
            tol = 1e-6 * math.fsum(abs(r * uu[k - 1]))
        else:
            tol = 1e-12 * abs(ref[k]) + 1e-300
        assert abs(red[k] - ref[k]) <= tol, (k, red[k], ref[k])
    s.close()


def test_reduce_sums_the_momentum_with_reduced_compressibility(cm):
    """Sec. 12 form with rho0 != 1: the reported momentum is j = rho0 u (not rho u), and it grows
    by exactly the applied force per cell and step."""
    n = (6, 7, 11)
    rho0 = 1.25
    rho, u = W.taylor_green(n[2], n[1], n[0], u0=0.05, background=(0.01, -0.02, 0.03))
    F = W.gaussian_force(n[2], n[1], n[0], seed=12, std=1e-4)
    kw = dict(tau=0.6, reduced_compressibility=True, rho0=rho0)
    s, o = _pair(cm, "D3Q27", n, "f64", rho, u, F, **kw)
    a = s.reduce()
    _, uo = o.moments()
    for d in range(3):
        j = rho0 * math.fsum(uo[d].numpy().ravel())
        assert abs(a[1 + d] - j) <= 1e-12 * math.fsum(abs(rho0 * uo[d].numpy().ravel())), (d, a[1 + d], j)
    s.step(5)
    b = s.reduce()
    for d in range(3):
        assert abs((b[1 + d] - a[1 + d]) - 5 * F[d].sum()) < 1e-12
    s.close()


def test_mass_drift_fp64(cm):
    """Mass is conserved to round-off in FP64 with walls, moving walls, LES and a force field."""
    case = CASES["walls_les_field"]
    rho, u, F = _inputs(case)
    s, _ = _pair(cm, "D3Q27", case["shape"], "f64", rho, u, F, **case["kw"])
    m0 = s.reduce()[0]
    s.step(200)
    m1 = s.reduce()[0]
    assert abs(m1 - m0) / m0 < 1e-12
    s.close()


def test_momentum_gain_equals_force_fp64(cm):
    n = 12
    rho, u = W.random_solenoidal(n, n, n, seed=7, u_rms=0.02)
    F = W.gaussian_force(n, n, n, seed=8, std=1e-4)
    s, _ = _pair(cm, "D3Q27", (n, n, n), "f64", rho, u, F, tau=0.55, smagorinsky_cs=0.1)
    a = s.reduce()
    s.step(10)
    b = s.reduce()
    for d in range(3):
        assert abs((b[1 + d] - a[1 + d]) - 10 * F[d].sum()) < 1e-12
    s.close()


def test_deterministic(cm):
    case = CASES["walls_les_field"]
    rho, u, F = _inputs(case)
    outs = []
    for _ in range(2):
        s, _ = _pair(cm, "D3Q27", case["shape"], "f32", rho, u, F, **case["kw"])
        s.step(7)
        outs.append((s.get_state().cpu(), s.reduce()))
        s.close()
    assert torch.equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


def test_host_buffers_match_device(cm):
    n = (4, 6, 40)
    rho, u = W.taylor_green(n[2], n[1], n[0], u0=0.03)
    F = W.gaussian_force(n[2], n[1], n[0], seed=9, std=1e-5)
    a = cm.Solver(lattice="D3Q27", nx=n[2], ny=n[1], nz=n[0], storage="f32", tau=0.6)
    a.set_force((0, 0, 0), F)              # numpy -> host path
    a.init(rho, u)
    a.step(5)
    ra, ua = a.moments(host=True)
    b = cm.Solver(lattice="D3Q27", nx=n[2], ny=n[1], nz=n[0], storage="f32", tau=0.6)
    b.set_force((0, 0, 0), torch.tensor(F, device="cuda"))
    b.init(torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"))
    b.step(5)
    rb, ub = b.moments()
    assert np.array_equal(ra, rb.cpu().numpy()) and np.array_equal(ua, ub.cpu().numpy())
    a.close()
    b.close()


def test_step_buffers_equals_step(cm):
    n = (5, 8, 33)
    rho, u = W.taylor_green(n[2], n[1], n[0], u0=0.03)
    s = cm.Solver(lattice="D3Q27", nx=n[2], ny=n[1], nz=n[0], storage="f32", tau=0.6)
    s.init(torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"))
    a = s.get_state()
    b = s.new_state()
    s.step_buffers(a, b)
    s.step(1)
    assert torch.equal(s.get_state(), b)
    r1, u1 = s.moments()
    r2, u2 = s.moments(state=b)
    assert torch.equal(r1, r2) and torch.equal(u1, u2)
    s.close()


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 5), (3, 1, 1), (2, 2, 2)])
def test_degenerate_grids(cm, shape):
    """One-cell axes wrap onto themselves (periodic) or reflect (walls)."""
    nz, ny, nx = shape
    rho, u = W.taylor_green(nx, ny, nz, u0=0.02, background=(0.01, 0.0, 0.0))
    for bc in (("periodic",) * 3, ("bounceback",) * 3):
        s, o = _pair(cm, "D3Q27", shape, "f64", rho, u, None, uniform=(1e-4, 0, 0), tau=0.7, bc=bc)
        s.step(3)
        o.step(3)
        got = H.decode(s.get_state(), "D3Q27")
        assert (got - o.s).abs().max().item() < 1e-14
        s.close()


def test_invalid_arguments_return_errors(cm):
    s = cm.Solver(lattice="D3Q27", nx=4, ny=4, nz=4, storage="f32")
    with pytest.raises(cm.CmlbmError) as e:
        s.step(-1)
    assert e.value.code == cm.ERR_INVALID
    st = s.new_state()
    with pytest.raises(cm.CmlbmError) as e:
        s.step_buffers(st, st)
    assert e.value.code == cm.ERR_INVALID
    lam = torch.zeros((27, 4, 4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(cm.CmlbmError) as e:
        s.step_adjoint(st, lam, lam, torch.zeros(3, 64, dtype=torch.float64, device="cuda"))
    assert e.value.code == cm.ERR_INVALID
    with pytest.raises(cm.CmlbmError) as e:
        s.set_state(torch.zeros(5, dtype=torch.float32, device="cuda"))
    assert e.value.code == cm.ERR_INVALID
    s.close()
    # the adjoint is not provided for 16-bit storage or with the eddy viscosity
    for kw in (dict(storage="bf16"), dict(storage="f32", smagorinsky_cs=0.1)):
        b = cm.Solver(lattice="D3Q27", nx=4, ny=4, nz=4, **kw)
        with pytest.raises(cm.CmlbmError) as e:
            b.step_adjoint(b.new_state(), lam, torch.zeros_like(lam), torch.zeros(3, 64, dtype=torch.float64, device="cuda"))
        assert e.value.code == cm.ERR_UNSUPPORTED
        b.close()


# D3Q27 cases the TMA-staged kernel takes (nx a multiple of 128)
TMA_CASES = {
    "tma_periodic_field": dict(lattice="D3Q27", shape=(5, 7, 256), flow="tgv", kw=dict(tau=0.6, omega_bulk=1.0)),
    "tma_walls_les_vd": dict(lattice="D3Q27", shape=(6, 9, 128), flow="channel",
                             kw=dict(tau=0.52, smagorinsky_cs=0.15, van_driest=(26.0, 8.0),
                                     bc=("periodic", "bounceback", "bounceback"),
                                     wall_velocity=[[[0, 0, 0], [0, 0, 0]], [[0.02, 0, 0.01], [-0.03, 0.0, 0.0]],
                                                    [[0.01, 0, 0], [0, 0.02, 0]]])),
    "tma_x_walls": dict(lattice="D3Q27", shape=(4, 5, 128), flow="tgv",
                        kw=dict(tau=0.7, bc=("bounceback", "periodic", "periodic"),
                                wall_velocity=[[[0, 0.01, 0], [0, 0, -0.02]], [[0, 0, 0], [0, 0, 0]], [[0, 0, 0], [0, 0, 0]]])),
}


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("name", list(TMA_CASES))
def test_tma_kernel_one_step_elementwise(cm, name, storage):
    case = TMA_CASES[name]
    rho, u, F = _inputs(case)
    s, o = _pair(cm, case["lattice"], case["shape"], storage, rho, u, F, kernel="tma", **case["kw"])
    s0 = s.get_state()
    o.set_state(H.decode(s0, case["lattice"]))
    s.step(1)
    o.step(1)
    got = H.decode(s.get_state(), case["lattice"])
    w = H.lattice(case["lattice"]).w.view(-1, 1, 1, 1)
    d_got, d_ref = got / w - 1, o.s / w - 1
    tol = ONE_STEP_ATOL[storage] + ONE_STEP_RTOL[storage] * d_ref.abs()
    err = (d_got - d_ref).abs()
    assert bool((err <= tol).all()), f"max |dd| = {err.max().item():.3e}"
    assert s.reduce()[0] > 0      # also checks the pipeline error flag
    s.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_tma_and_direct_kernels_agree(cm, storage):
    case = TMA_CASES["tma_walls_les_vd"]
    rho, u, F = _inputs(case)
    states = []
    for kernel in ("tma", "direct"):
        s, _ = _pair(cm, case["lattice"], case["shape"], storage, rho, u, F, kernel=kernel, **case["kw"])
        s.step(15)
        states.append(H.decode(s.get_state(), case["lattice"]))
        s.close()
    w = H.lattice(case["lattice"]).w.view(-1, 1, 1, 1)
    diff = ((states[0] - states[1]) / w).abs().max().item()
    assert diff < (1e-5 if storage == "f32" else 2e-2)


def test_tma_requested_on_ineligible_config_is_rejected(cm):
    with pytest.raises(cm.CmlbmError) as e:
        cm.Solver(lattice="D3Q27", nx=150, ny=4, nz=4, storage="f32", kernel="tma")
    assert e.value.code == cm.ERR_UNSUPPORTED


# D3Q27 cases the two-cells-per-thread kernel takes (periodic x, nx a multiple of 64)
PAIR_CASES = {
    "pair_factorized_field": dict(lattice="D3Q27", shape=(5, 6, 64), flow="tgv",
                                  kw=dict(tau=0.58, omega_3=1.1, omega_4=1.3, attractor="factorized")),
    "pair_field_general_rates": dict(lattice="D3Q27", shape=(5, 5, 64), flow="tgv",
                                     kw=dict(tau=0.59, omega_3=1.2, omega_4=0.8)),
    "pair_factorized_unit_rates": dict(lattice="D3Q27", shape=(4, 7, 64), flow="tgv",
                                       kw=dict(tau=0.57, attractor="factorized", smagorinsky_cs=0.1)),
    "pair_reduced_walls_les": dict(lattice="D3Q27", shape=(5, 8, 128), flow="channel",
                                   kw=dict(tau=0.6, reduced_compressibility=True, rho0=1.02, smagorinsky_cs=0.1,
                                           bc=("periodic", "bounceback", "periodic"))),
    "pair_periodic_field": dict(lattice="D3Q27", shape=(5, 7, 128), flow="tgv", kw=dict(tau=0.6, omega_bulk=1.0)),
    "pair_walls_les_vd": dict(lattice="D3Q27", shape=(6, 9, 64), flow="channel",
                              kw=dict(tau=0.52, smagorinsky_cs=0.15, van_driest=(26.0, 8.0),
                                      bc=("periodic", "bounceback", "bounceback"),
                                      wall_velocity=[[[0, 0, 0], [0, 0, 0]], [[0.02, 0, 0.01], [-0.03, 0.0, 0.0]],
                                                     [[0.01, 0, 0], [0, 0.02, 0]]])),
    "pair_bulk_follows_shear_les": dict(lattice="D3Q27", shape=(4, 6, 192), flow="tgv",
                                        kw=dict(tau=0.51, smagorinsky_cs=0.12, omega_3=1.3, omega_4=0.9)),
    # unforced, unit higher-order rates: the SIMPLE collision with the form fixed at compile time
    "pair_factorized_unforced": dict(lattice="D3Q27", shape=(5, 6, 64), flow="tgv_unforced",
                                     kw=dict(tau=0.57, attractor="factorized", omega_bulk=1.1)),
    "pair_reduced_unforced_walls_les": dict(lattice="D3Q27", shape=(5, 8, 128), flow="tgv_unforced",
                                            kw=dict(tau=0.6, reduced_compressibility=True, rho0=1.02,
                                                    smagorinsky_cs=0.1, bc=("periodic", "bounceback", "periodic"))),
}


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("name", list(PAIR_CASES))
def test_pair_kernel_one_step_elementwise(cm, name, storage):
    case = PAIR_CASES[name]
    rho, u, F = _inputs(case)
    s, o = _pair(cm, case["lattice"], case["shape"], storage, rho, u, F, kernel="pair", **case["kw"])
    s0 = s.get_state()
    o.set_state(H.decode(s0, case["lattice"]))
    s.step(1)
    o.step(1)
    got = H.decode(s.get_state(), case["lattice"])
    w = H.lattice(case["lattice"]).w.view(-1, 1, 1, 1)
    d_got, d_ref = got / w - 1, o.s / w - 1
    tol = ONE_STEP_ATOL[storage] + ONE_STEP_RTOL[storage] * d_ref.abs()
    err = (d_got - d_ref).abs()
    assert bool((err <= tol).all()), f"max |dd| = {err.max().item():.3e}"
    s.close()


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("name", list(PAIR_CASES) + ["unforced_unit_rates_pair_walls_les"])
def test_pair_kernel_cell_pairings_agree_bitwise(cm, name, storage):
    """The two-cells-per-thread step pairs adjacent cells (x0, x0 + 1) when both state buffers
    are aligned to two entries, and (x, x + nx/2) otherwise (buffers offset by one entry here).
    Every cell goes through the same lane arithmetic either way: the bits must agree."""
    case = PAIR_CASES.get(name) or CASES[name]
    rho, u, F = _inputs(case)
    s, _ = _pair(cm, case["lattice"], case["shape"], storage, rho, u, F, kernel="pair", **case["kw"])
    s0 = s.get_state().reshape(-1)
    n = s0.numel()
    outs = []
    for off in (0, 1):
        a = torch.zeros(n + 1, dtype=s0.dtype, device="cuda")
        b = torch.zeros_like(a)
        src, dst = a[off:off + n], b[off:off + n]
        src.copy_(s0)
        s.step_buffers(src, dst)
        outs.append(dst.clone())
    torch.cuda.synchronize()
    assert torch.equal(outs[0].view(torch.uint8), outs[1].view(torch.uint8))
    s.close()


@pytest.mark.parametrize("name", list(PAIR_CASES))
def test_pair_kernel_fp32_trajectory(cm, name):
    case = PAIR_CASES[name]
    rho, u, F = _inputs(case)
    s, o = _pair(cm, case["lattice"], case["shape"], "f32", rho, u, F, kernel="pair", **case["kw"])
    s.step(30)
    o.step(30)
    _, ug = s.moments()
    _, uo = o.moments()
    assert H.rel_l2(ug, uo) < 1e-5
    s.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_pair_and_direct_kernels_agree(cm, storage):
    case = PAIR_CASES["pair_walls_les_vd"]
    rho, u, F = _inputs(case)
    states = []
    for kernel in ("pair", "direct"):
        s, _ = _pair(cm, case["lattice"], case["shape"], storage, rho, u, F, kernel=kernel, **case["kw"])
        s.step(15)
        states.append(H.decode(s.get_state(), case["lattice"]))
        s.close()
    w = H.lattice(case["lattice"]).w.view(-1, 1, 1, 1)
    diff = ((states[0] - states[1]) / w).abs().max().item()
    assert diff < (1e-5 if storage == "f32" else 2e-2)


@pytest.mark.parametrize("kw,expect", [
    (dict(nx=128), "pair"), (dict(nx=128, storage="bf16"), "pair"), (dict(nx=96), "direct"),
    (dict(nx=128, storage="f64"), "direct"), (dict(nx=128, attractor="factorized"), "pair"),
    (dict(nx=128, reduced_compressibility=True, storage="f16"), "pair"), (dict(nx=96, attractor="factorized"), "direct"),
    (dict(nx=128, bc=("bounceback", "periodic", "periodic")), "direct"), (dict(nx=128, kernel="direct"), "direct"),
    (dict(nx=128, kernel="tma"), "tma"), (dict(nx=64, bc=("periodic", "periodic", "halo")), "pair"),
    (dict(nx=64, nz=16), "pair"), (dict(nx=64, nz=16, kernel="pair_two_steps"), "pair_two_steps"),
    (dict(nx=64, nz=16, storage="bf16"), "pair"),
    (dict(nx=64, nz=16, kernel="pair"), "pair"), (dict(nx=64, nz=16, bc=("periodic", "periodic", "halo")), "pair")])
def test_automatic_kernel_choice(cm, kw, expect):
    args = dict(lattice="D3Q27", ny=4, nz=4, storage="f32")
    args.update(kw)
    s = cm.Solver(**args)
    assert s.step_kernel == expect
    s.close()


@pytest.mark.parametrize("kw", [dict(nx=96), dict(nx=128, bc=("bounceback", "periodic", "periodic")),
                                dict(nx=96, attractor="factorized"), dict(nx=128, storage="f64"),
                                dict(nx=128, lattice="D2Q9", nz=1)])
def test_pair_requested_on_ineligible_config_is_rejected(cm, kw):
    args = dict(lattice="D3Q27", ny=4, nz=4, storage="f32", kernel="pair")
    args.update(kw)
    with pytest.raises(cm.CmlbmError) as e:
        cm.Solver(**args)
    assert e.value.code == cm.ERR_UNSUPPORTED


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_filtered_step_on_a_ragged_box_matches_oracle(cm, storage, tol):
    """Turbulence as forcing on a 70 x 13 x 19 box: several thread blocks in every direction with
    ragged tails, and the closure's central differences wrapping across the periodic edges."""
    shape = (19, 13, 70)
    nz, ny, nx = shape
    rho, u = W.random_solenoidal(nx, ny, nz, seed=11, u_rms=0.04)
    kw = dict(tau=0.56)
    s, o = _pair(cm, "D3Q27", shape, storage, rho, u, None, uniform=(1e-6, -2e-6, 0.0), **kw)
    s.step_filtered(3, 0.17)
    o.step_filtered(3, 0.17)
    _, ug = s.moments()
    _, uo = o.moments()
    assert H.rel_l2(ug, uo) < tol
    s.close()


@pytest.mark.parametrize("lattice,storage,tol", [("D3Q27", "f64", 1e-12), ("D3Q27", "f32", 2e-5), ("D2Q9", "f64", 1e-12)])
def test_filtered_step_matches_oracle(cm, lattice, storage, tol):
    """Turbulence as forcing (Sec. 14): Smagorinsky closure force + factorized, reduced step."""
    shape = (6, 10, 12) if lattice == "D3Q27" else (1, 14, 18)
    nz, ny, nx = shape
    rho, u = W.random_solenoidal(nx, ny, nz, seed=7, u_rms=0.04)
    if lattice == "D2Q9":
        u[2] = 0
    kw = dict(tau=0.55, attractor="factorized", reduced_compressibility=True, rho0=1.0)
    s, o = _pair(cm, lattice, shape, storage, rho, u, None, uniform=(2e-6, 0.0, 0.0), **kw)
    s.step_filtered(5, 0.18)
    o.step_filtered(5, 0.18)
    rg, ug = s.moments()
    ro, uo = o.moments()
    assert H.rel_l2(ug, uo) < tol
    s.close()
    # with C_s = 0 the closure force is exactly the uniform force: same state as a plain step
    a, _ = _pair(cm, lattice, shape, storage, rho, u, None, uniform=(2e-6, 0.0, 0.0), **kw)
    b, _ = _pair(cm, lattice, shape, storage, rho, u, None, uniform=(2e-6, 0.0, 0.0), **kw)
    a.step_filtered(3, 0.0)
    b.step(3)
    assert torch.equal(a.get_state(), b.get_state())
    a.close()
    b.close()


def test_filtered_step_rejects_walls(cm):
    s = cm.Solver(lattice="D3Q27", nx=8, ny=8, nz=8, storage="f32", bc=("periodic", "bounceback", "periodic"))
    with pytest.raises(cm.CmlbmError) as e:
        s.turbulence_force(0.1)
    assert e.value.code == cm.ERR_UNSUPPORTED
    s.close()


@pytest.mark.parametrize("kernel", ["pair", "direct"])
def test_graph_replayed_steps_equal_single_steps(cm, kernel):
    """cmlbm_step replays pairs of steps as a CUDA graph; the result must equal one-by-one steps,
    also across a force change (the captured parameters are dropped) and odd step counts."""
    case = PAIR_CASES["pair_walls_les_vd"]
    rho, u, F = _inputs(case)
    a, _ = _pair(cm, case["lattice"], case["shape"], "f32", rho, u, F, kernel=kernel, **case["kw"])
    b, _ = _pair(cm, case["lattice"], case["shape"], "f32", rho, u, F, kernel=kernel, **case["kw"])
    la, lb = a.launch_count, b.launch_count
    a.step(7)
    for _ in range(7):
        b.step(1)
    assert torch.equal(a.get_state(), b.get_state())
    a.set_force((3e-5, 0.0, -1e-5))
    b.set_force((3e-5, 0.0, -1e-5))
    a.step(6)
    for _ in range(6):
        b.step(1)
    assert torch.equal(a.get_state(), b.get_state())
    assert a.launch_count - la == b.launch_count - lb == 13
    a.close()
    b.close()


TWO_STEP_CASES = {
    "periodic_field_ragged_groups": dict(shape=(20, 6, 64), flow="tgv", kw=dict(tau=0.6, omega_bulk=1.0)),
    "unforced_minimum_depth": dict(shape=(16, 5, 128), flow="tgv_unforced", kw=dict(tau=0.53)),
    "walls_y_z_les_lid": dict(shape=(19, 9, 64), flow="channel",
                              kw=dict(tau=0.52, smagorinsky_cs=0.15, van_driest=(26.0, 8.0),
                                      bc=("periodic", "bounceback", "bounceback"),
                                      wall_velocity=[[[0, 0, 0], [0, 0, 0]], [[0.02, 0, 0.01], [-0.03, 0.0, 0.0]],
                                                     [[0.01, 0, 0], [0, 0.02, 0]]])),
}


@pytest.mark.parametrize("steps", [2, 7, 12])
@pytest.mark.parametrize("name", list(TWO_STEP_CASES))
def test_two_steps_per_pass_equal_single_steps_bitwise(cm, name, steps):
    """The plane-ring schedule runs the same kernel code on every cell: bitwise equal states."""
    case = dict(TWO_STEP_CASES[name], lattice="D3Q27")
    rho, u, F = _inputs(case)
    a, _ = _pair(cm, "D3Q27", case["shape"], "f32", rho, u, F, kernel="pair_two_steps", **case["kw"])
    b, _ = _pair(cm, "D3Q27", case["shape"], "f32", rho, u, F, kernel="pair", **case["kw"])
    assert a.step_kernel == "pair_two_steps" and b.step_kernel == "pair"
    a.step(steps)
    for _ in range(steps):
        b.step(1)
    assert torch.equal(a.get_state(), b.get_state())
    # and again after a force change (the captured passes are dropped)
    a.set_force((1e-5, -2e-5, 0.0))
    b.set_force((1e-5, -2e-5, 0.0))
    a.step(4)
    b.step(4)
    assert torch.equal(a.get_state(), b.get_state())
    a.close()
    b.close()


def test_two_steps_per_pass_against_the_oracle(cm):
    case = dict(TWO_STEP_CASES["walls_y_z_les_lid"], lattice="D3Q27")
    rho, u, F = _inputs(case)
    s, o = _pair(cm, "D3Q27", case["shape"], "f32", rho, u, F, kernel="pair_two_steps", **case["kw"])
    assert s.step_kernel == "pair_two_steps"
    s.step(20)
    o.step(20)
    _, ug = s.moments()
    _, uo = o.moments()
    assert H.rel_l2(ug, uo) < 1e-5
    s.close()


@pytest.mark.parametrize("kw", [dict(nz=15), dict(storage="bf16"), dict(nx=96), dict(bc=("periodic", "periodic", "halo")),
                                dict(attractor="factorized")])
def test_two_steps_requested_on_ineligible_config_is_rejected(cm, kw):
    args = dict(lattice="D3Q27", nx=64, ny=4, nz=16, storage="f32", kernel="pair_two_steps")
    args.update(kw)
    with pytest.raises(cm.CmlbmError) as e:
        cm.Solver(**args)
    assert e.value.code == cm.ERR_UNSUPPORTED


def test_host_fields_page_locked_and_pageable_agree(cm):
    """cmlbm_init / cmlbm_moments with CMLBM_HOST read and write page-locked buffers in place
    and stage pageable ones through the device: both routes give the same bits."""
    nz, ny, nx = 5, 7, 64
    rho, u = W.taylor_green(nx, ny, nz, u0=0.05, background=(0.01, 0.0, -0.02))
    states, fields = [], []
    for pinned in (False, True):
        s = cm.Solver(lattice="D3Q27", nx=nx, ny=ny, nz=nz, storage="f32", tau=0.6)
        if pinned:
            s.init(torch.tensor(rho).pin_memory(), torch.tensor(u).pin_memory())
        else:
            s.init(rho, u)
        states.append(s.get_state().clone())
        s.step(4)
        if pinned:
            out = (torch.empty((nz, ny, nx), dtype=torch.float64).pin_memory(),
                   torch.empty((3, nz, ny, nx), dtype=torch.float64).pin_memory())
            r, v = s.moments(host=True, out=out)
            fields.append((r.numpy().copy(), v.numpy().copy()))
        else:
            fields.append(s.moments(host=True))
        s.close()
    assert torch.equal(states[0].view(torch.uint8), states[1].view(torch.uint8))
    assert np.array_equal(fields[0][0], fields[1][0]) and np.array_equal(fields[0][1], fields[1][1])


def test_out_of_memory_is_reported_and_the_handle_recovers(cm, monkeypatch):
    """CMLBM_ERR_NOMEM through the allocation-limit test hook (no shared GPU is driven out of
    memory): a create that cannot allocate its state fails cleanly, and a handle whose staging
    allocation fails keeps working once memory is available."""
    monkeypatch.setenv("CMLBM_TEST_ALLOC_LIMIT", "100000")
    with pytest.raises(cm.CmlbmError) as e:
        cm.Solver(lattice="D3Q27", nx=32, ny=32, nz=32, storage="f32", tau=0.6)   # 3.5 MB per buffer
    assert e.value.code == cm.ERR_NOMEM
    s = cm.Solver(lattice="D3Q27", nx=8, ny=6, nz=4, storage="f32", tau=0.6)      # 21 kB per buffer
    rho = 1.0 + 0.01 * np.random.default_rng(1).standard_normal((4, 6, 8))
    monkeypatch.setenv("CMLBM_TEST_ALLOC_LIMIT", "1000")
    with pytest.raises(cm.CmlbmError) as e:
        s.init(rho, None)                        # pageable host data needs the 6 kB staging buffer
    assert e.value.code == cm.ERR_NOMEM
    monkeypatch.delenv("CMLBM_TEST_ALLOC_LIMIT")
    s.init(rho, None)
    s.step(3)
    red = s.reduce()
    assert abs(red[0] - rho.sum()) < 1e-6 * rho.sum()
    s.close()


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("walls", [False, True])
def test_pair_kernel_uniform_force_along_x(cm, storage, walls):
    """A uniform force along x only with the default unit higher-order rates takes the pair
    kernel's variant whose source recursion keeps only the x terms: one step element-wise and a
    trajectory against the oracle, with walls, eddy viscosity and van Driest damping (the channel
    configuration) and without."""
    shape = (6, 9, 64)
    nz, ny, nx = shape
    kw = dict(tau=0.53, omega_bulk=1.0, smagorinsky_cs=0.12)
    if walls:
        kw.update(bc=("periodic", "bounceback", "periodic"), van_driest=(26.0, 6.0),
                  wall_velocity=[[[0, 0, 0], [0, 0, 0]], [[0.01, 0, 0], [-0.02, 0, 0.01]], [[0, 0, 0], [0, 0, 0]]])
    rho, u, _ = W.channel(nx, ny, nz, u_tau=0.02, seed=9)
    F = (3e-5, 0.0, 0.0)
    s, o = _pair(cm, "D3Q27", shape, storage, rho, u, None, uniform=F, **kw)
    assert s.step_kernel == "pair"
    s0 = s.get_state()
    o.set_state(H.decode(s0, "D3Q27"))
    s.step(1)
    o.step(1)
    got = H.decode(s.get_state(), "D3Q27")
    w = H.lattice("D3Q27").w.view(-1, 1, 1, 1)
    d_got, d_ref = got / w - 1, o.s / w - 1
    tol = ONE_STEP_ATOL[storage] + ONE_STEP_RTOL[storage] * d_ref.abs()
    assert bool(((d_got - d_ref).abs() <= tol).all()), f"max |dd| = {(d_got - d_ref).abs().max().item():.3e}"
    if storage == "f32":
        s.step(20)
        o.step(20)
        assert H.rel_l2(s.moments()[1], o.moments()[1]) < 1e-5
    s.close()
