"""Slab decomposition along z on one GPU: K slab handles with face exchange against one handle.

The same step kernel runs on every cell either way, so the decomposed run must reproduce the
single-domain run bit for bit: the own planes of every slab's state and the moments, after
several steps, for periodic and wall-bounded boxes, LES, force fields and the other collision
forms, in every storage type. One case is also held against the oracle directly.
"""
import numpy as np
import pytest
import torch

import helpers as H
from oracle.collision import Params
from oracle.solver import OracleSim
from paper_1202_6074_gb300 import slab as SL

pytestmark = pytest.mark.gpu

NX, NY, NZ = 24, 10, 13
STEPS = 6


@pytest.fixture(scope="module")
def cm():
    import __graft_entry__ as G

    G.build()
    from paper_1202_6074_gb300 import cmlbm

    return cmlbm


def _fields(seed=3):
    g = np.random.default_rng(seed)
    rho = 1.0 + 0.01 * g.standard_normal((NZ, NY, NX))
    u = 0.03 * g.standard_normal((3, NZ, NY, NX))
    F = 1e-4 * g.standard_normal((3, NZ, NY, NX))
    return rho, u, F


CASES = {
    "periodic_field_f32": dict(storage="f32", tau=0.6, omega_bulk=1.0, field=True),
    "walls_les_bf16": dict(storage="bf16", tau=0.52, omega_bulk=1.0, smagorinsky_cs=0.15, van_driest=(26.0, 2.0),
                           xy=("periodic", "bounceback"), lid=0.04, uniform=(1e-5, 0.0, 0.0)),
    "xwalls_f16": dict(storage="f16", tau=0.55, xy=("bounceback", "periodic"), uniform=(0.0, 1e-5, 0.0)),
    "factorized_reduced_f64": dict(storage="f64", tau=0.7, omega_bulk=1.2, attractor="factorized",
                                   reduced_compressibility=True, xy=("periodic", "bounceback"),
                                   uniform=(0.0, 2e-5, 1e-5)),
}


def _solver_kw(c):
    kw = dict(lattice="D3Q27", nx=NX, ny=NY, storage=c["storage"], tau=c["tau"])
    for k in ("omega_bulk", "smagorinsky_cs", "van_driest", "attractor", "reduced_compressibility"):
        if k in c:
            kw[k] = c[k]
    if c.get("lid"):
        uw = [[[0.0] * 3 for _ in range(2)] for _ in range(3)]
        uw[1][1][0] = c["lid"]
        kw["wall_velocity"] = uw
    return kw


def _setup(s, c, rho, u, F, sl=slice(None)):
    if c.get("field"):
        s.set_force((0.0, 0.0, 0.0), torch.tensor(F[:, sl], device="cuda"))
    elif c.get("uniform"):
        s.set_force(c["uniform"])
    s.init(torch.tensor(rho[sl], device="cuda"), torch.tensor(u[:, sl], device="cuda"))


def _single(cm, c, rho, u, F):
    xy = c.get("xy", ("periodic", "periodic"))
    s = cm.Solver(nz=NZ, bc=(xy[0], xy[1], "periodic"), **_solver_kw(c))
    _setup(s, c, rho, u, F)
    return s


def _slabs(cm, c, rho, u, F, k):
    xy = c.get("xy", ("periodic", "periodic"))
    out = []
    for r in range(k):
        s, z0 = SL.cuda_slab(cm, NZ, r, k, bc=xy, **_solver_kw(c))
        _setup(s, c, rho, u, F, slice(z0, z0 + s.shape[0]))
        out.append(s)
    return out


@pytest.mark.parametrize("overlap", [False, True])
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("k", [1, 2, 3])
def test_slabs_reproduce_the_single_domain_bitwise(cm, name, k, overlap):
    """overlap: split steps (boundary planes on the handle's stream, interior planes on the
    library's own) with the face exchange issued while the interior runs."""
    c = CASES[name]
    rho, u, F = _fields()
    ref = _single(cm, c, rho, u, F)
    slabs = _slabs(cm, c, rho, u, F, k)
    assert slabs[0].state_shape[1] == slabs[0].shape[0] + 2
    ref.step(STEPS)
    run = SL.SlabRun(slabs, SL.LocalExchange(slabs), overlap=overlap)
    run.step(STEPS)
    torch.cuda.synchronize()
    s_ref = ref.get_state()
    own = torch.cat([s.get_state()[:, 1:-1] for s in slabs], dim=1)
    assert torch.equal(own.view(torch.uint8) if own.dtype != torch.float64 else own,
                       s_ref.view(torch.uint8) if s_ref.dtype != torch.float64 else s_ref)
    rho_r, u_r = ref.moments()
    rho_s = torch.cat([s.moments()[0] for s in slabs], dim=0)
    u_s = torch.cat([s.moments()[1] for s in slabs], dim=1)
    assert torch.equal(rho_s, rho_r) and torch.equal(u_s, u_r)
    red_r = ref.reduce()
    red_s = run.reduce()
    assert abs(red_s[0] - red_r[0]) <= 1e-12 * red_r[0]
    for a, b in zip(red_s[1:], red_r[1:]):
        assert abs(a - b) <= 1e-12 * red_r[0] * 0.05
    for s in slabs + [ref]:
        s.close()


def test_one_slab_is_its_own_neighbour_through_dist_exchange(cm):
    c = CASES["periodic_field_f32"]
    rho, u, F = _fields(5)
    ref = _single(cm, c, rho, u, F)
    (s,) = _slabs(cm, c, rho, u, F, 1)
    ex = SL.DistExchange(s)
    assert ex.world == 1
    ref.step(STEPS)
    SL.SlabRun([s], ex).step(STEPS)
    assert torch.equal(s.get_state()[:, 1:-1], ref.get_state())
    s.close()
    ref.close()


def test_host_staged_faces_equal_device_faces(cm):
    c = CASES["walls_les_bf16"]
    rho, u, F = _fields(6)
    slabs = _slabs(cm, c, rho, u, F, 2)
    slabs[0].step(2)
    for face in (SL.FACE_BOTTOM, SL.FACE_TOP):
        d = slabs[0].pack(face)
        hmsg = slabs[0].pack(face, host=True)
        torch.cuda.synchronize()
        assert hmsg.device.type == "cpu"
        assert torch.equal(d.cpu().view(torch.uint8), hmsg.view(torch.uint8))
        # the message is the 9 direction planes of the face's own plane (e_z = +1 up, -1 down)
        st = slabs[0].get_state()
        dirs = slice(18, 27) if face == SL.FACE_TOP else slice(0, 9)
        plane = st.shape[1] - 2 if face == SL.FACE_TOP else 1
        assert torch.equal(d.view(torch.uint8), st[dirs, plane].contiguous().view(torch.uint8))
        # unpack from host lands in the ghost plane on the other face of the neighbour
        slabs[1].unpack(1 - face, hmsg)
        torch.cuda.synchronize()
        st1 = slabs[1].get_state()
        gplane = 0 if face == SL.FACE_TOP else st1.shape[1] - 1
        assert torch.equal(st1[dirs, gplane].contiguous().view(torch.uint8), d.view(torch.uint8))
    for s in slabs:
        s.close()


def test_decomposed_run_against_the_oracle(cm):
    """Three FP64 slabs with walls, a moving lid and LES against the single-domain oracle."""
    c = dict(storage="f64", tau=0.52, omega_bulk=1.0, smagorinsky_cs=0.15, van_driest=(26.0, 2.0),
             xy=("periodic", "bounceback"), lid=0.04, uniform=(1e-5, 0.0, 0.0))
    rho, u, F = _fields(8)
    slabs = _slabs(cm, c, rho, u, F, 3)
    SL.SlabRun(slabs, SL.LocalExchange(slabs)).step(STEPS)
    uw = [[[0.0] * 3 for _ in range(2)] for _ in range(3)]
    uw[1][1][0] = 0.04
    o = OracleSim("D3Q27", NX, NY, NZ, Params(tau=0.52, omega_bulk=1.0, cs_smag=0.15),
                  bc=("periodic", "bounceback", "periodic"), wall_velocity=uw, van_driest=(26.0, 2.0))
    o.set_force((1e-5, 0.0, 0.0))
    o.init(torch.tensor(rho), torch.tensor(u))
    o.step(STEPS)
    rho_o, u_o = o.moments()
    u_s = torch.cat([s.moments()[1] for s in slabs], dim=1)
    rho_s = torch.cat([s.moments()[0] for s in slabs], dim=0)
    assert H.rel_l2(u_s, u_o) < 1e-11
    assert float((rho_s.cpu() - rho_o).abs().max()) < 1e-13
    for s in slabs:
        s.close()


def test_slab_only_calls_are_rejected(cm):
    s = cm.Solver(nx=8, ny=4, nz=4)
    with pytest.raises(cm.CmlbmError) as e:
        s.pack(SL.FACE_TOP)
    assert e.value.code == cm.ERR_INVALID
    s.close()
    s = cm.Solver(nx=8, ny=4, nz=4, bc=("periodic", "periodic", "halo"))
    assert s.state_bytes == 27 * 8 * 4 * 6 * 4
    assert int(s.lib.cmlbm_halo_bytes(s.h)) == 9 * 8 * 4 * 4
    with pytest.raises(cm.CmlbmError) as e:
        s.pack(7)
    assert e.value.code == cm.ERR_INVALID
    with pytest.raises(cm.CmlbmError) as e:
        s.turbulence_force(0.1)
    assert e.value.code == cm.ERR_UNSUPPORTED
    lam = torch.zeros((27, 4, 4, 8), dtype=torch.float32, device="cuda")
    dF = torch.zeros((3, 4, 4, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(cm.CmlbmError) as e:
        s.step_adjoint(s.get_state(), lam, lam.clone(), dF)
    assert e.value.code == cm.ERR_UNSUPPORTED
    s.close()


@pytest.mark.parametrize("storage,force", [("f32", 0.0), ("bf16", 0.0), ("f32", 1e-5)])
def test_slabs_with_the_two_cell_kernel(cm, storage, force):
    """The packed two-cells-per-thread step on slabs against the same kernel on one domain
    (unforced FP32: cells x, x + nx/2 per thread; 16-bit or forced: adjacent cells)."""
    nx, ny, nz = 64, 6, 9
    g = np.random.default_rng(11)
    rho = 1.0 + 0.01 * g.standard_normal((nz, ny, nx))
    u = 0.03 * g.standard_normal((3, nz, ny, nx))
    kw = dict(lattice="D3Q27", nx=nx, ny=ny, storage=storage, tau=0.53, omega_bulk=1.0, smagorinsky_cs=0.1,
              kernel="pair")
    ref = cm.Solver(nz=nz, bc=("periodic", "bounceback", "periodic"), **kw)
    ref.set_force((force, 0.0, 0.0))
    ref.init(torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"))
    slabs = []
    for r in range(2):
        s, z0 = SL.cuda_slab(cm, nz, r, 2, bc=("periodic", "bounceback"), **kw)
        s.set_force((force, 0.0, 0.0))
        sl = slice(z0, z0 + s.shape[0])
        s.init(torch.tensor(rho[sl], device="cuda"), torch.tensor(u[:, sl], device="cuda"))
        slabs.append(s)
    ref.step(STEPS)
    SL.SlabRun(slabs, SL.LocalExchange(slabs)).step(STEPS)
    own = torch.cat([s.get_state()[:, 1:-1] for s in slabs], dim=1)
    assert torch.equal(own.view(torch.uint8), ref.get_state().view(torch.uint8))
    for s in slabs + [ref]:
        s.close()


@pytest.mark.parametrize("storage", ["f32", "bf16", "f64"])
def test_split_step_equals_step_on_a_single_domain(cm, storage):
    """cmlbm_step_split on an ordinary handle: the same state as cmlbm_step, bit for bit, and the
    calls that follow it see the interior planes."""
    c = dict(storage=storage, tau=0.6, omega_bulk=1.0, field=True)
    rho, u, F = _fields(7)
    a = _single(cm, c, rho, u, F)
    b = _single(cm, c, rho, u, F)
    for _ in range(5):
        a.step_split()
    b.step(5)
    assert torch.equal(a.get_state().view(torch.uint8), b.get_state().view(torch.uint8))
    assert a.reduce() == b.reduce()
    a.step_split()
    ra, ua = a.moments()
    b.step(1)
    rb, ub = b.moments()
    assert torch.equal(ra, rb) and torch.equal(ua, ub)
    a.close()
    b.close()



def test_split_step_in_two_parts(cm):
    """The boundary and interior parts issued in two calls give the plain step's state; the
    parts must alternate, and a step or a state replacement between them is refused."""
    c = dict(storage="f32", tau=0.6, omega_bulk=1.0, field=True)
    rho, u, F = _fields(8)
    a = _single(cm, c, rho, u, F)
    b = _single(cm, c, rho, u, F)
    for _ in range(3):
        a.step_split(1)
        a.step_split(2)
    b.step(3)
    assert torch.equal(a.get_state(), b.get_state())
    with pytest.raises(cm.CmlbmError) as e:
        a.step_split(2)                       # an interior part without its boundary part
    assert e.value.code == cm.ERR_INVALID
    a.step_split(1)
    for bad in (lambda: a.step_split(1), lambda: a.step(1), lambda: a.set_state(b.get_state())):
        with pytest.raises(cm.CmlbmError) as e:
            bad()
        assert e.value.code == cm.ERR_INVALID
    a.step_split(2)
    b.step(1)
    assert torch.equal(a.get_state(), b.get_state())
    a.close()
    b.close()
