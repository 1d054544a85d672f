"""The allocation-free reduction (cmlbm_reduce_noalloc) against cmlbm_reduce.

It exists for callers that cannot allocate device memory, for example a host whose device
memory belongs to another allocator's pool, or a loop with a fixed memory budget. It works
without a handle, keeping its partial sums in a fixed device array inside the library. This
file sorts last so that a stop-at-first-failure run has executed every other test before it.
"""
import ctypes

import pytest
import torch

from paper_1202_6074_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# the same relative tolerance as the other FP64 reduction tests, taken relative to the size of
# the summands: momentum sums that cancel to ~0 are compared on the scale mass * rms velocity
RTOL = 1e-12


@pytest.fixture(scope="module")
def cm():
    import __graft_entry__ as G

    G.build()
    from paper_1202_6074_gb300 import cmlbm

    assert torch.cuda.is_available()
    return cmlbm


def _close(a, b):
    mass, ke = abs(b[0]), abs(b[4])
    u_rms = (2.0 * ke / mass) ** 0.5
    scale = [mass, mass * u_rms, mass * u_rms, mass * u_rms, ke]
    for k in range(5):
        assert abs(a[k] - b[k]) <= RTOL * max(abs(b[k]), scale[k]), (k, a[k], b[k])


@pytest.mark.parametrize("lattice,shape,storage,bc,field", [
    ("D3Q27", (37, 21, 19), "f32", ("periodic",) * 3, False),
    ("D3Q27", (37, 21, 19), "f64", ("periodic", "bounceback", "periodic"), True),
    ("D3Q27", (37, 21, 19), "bf16", ("bounceback", "periodic", "bounceback"), True),
    ("D3Q27", (37, 21, 19), "f16", ("bounceback", "bounceback", "periodic"), False),
    ("D2Q9", (97, 45, 1), "f64", ("periodic", "bounceback", "periodic"), True),
    # the largest grid the fixed scratch covers: 16384 blocks of 1024 cells fill every slot
    ("D3Q27", (256, 256, 256), "f32", ("periodic",) * 3, False),
])
def test_noalloc_matches_reduce_on_two_calls(cm, lattice, shape, storage, bc, field):
    nx, ny, nz = shape
    rho, u = W.taylor_green(nx, ny, nz, u0=0.04, background=(0.01, 0.0, -0.02 if lattice == "D3Q27" else 0.0))
    if lattice == "D2Q9":
        u[2] = 0.0
    uniform = (1e-5, -2e-5, 3e-6 if lattice == "D3Q27" else 0.0)
    walls = [[[0.01, 0, 0], [0, 0.02, 0]], [[0.03, 0, 0], [-0.01, 0, 0]], [[0, 0, 0.01], [0.02, 0, 0]]]
    s = cm.Solver(lattice=lattice, nx=nx, ny=ny, nz=nz, storage=storage, tau=0.6, bc=bc, wall_velocity=walls)
    F = None
    if field:
        F = torch.tensor(W.gaussian_force(nx, ny, nz, seed=3, std=1e-4), device="cuda")
        if lattice == "D2Q9":
            F[2] = 0.0
    s.set_force(uniform if not field else (0.0, 0.0, 0.0), F)
    s.init(torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"))
    Ff = None if F is None else F.to(s.real_dtype).contiguous()
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    for call in range(2):
        state = s.get_state()
        torch.cuda.synchronize()
        ref = s.reduce()
        cm.reduce_noalloc(s.cfg, state, out, uniform_force=uniform if not field else (0.0, 0.0, 0.0),
                          force_field=Ff)
        torch.cuda.synchronize()
        _close(out.cpu().tolist(), ref)
        s.step(3)
    s.close()


def test_noalloc_rejects_grids_over_the_limit(cm):
    cfg = cm.make_config(lattice="D3Q27", nx=257, ny=256, nz=256, storage="f32")
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    rc = cm.load().cmlbm_reduce_noalloc(ctypes.byref(cfg), cm._ptr(dummy), None, None, cm._ptr(out))
    assert rc == cm.ERR_INVALID
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
