"""Slab decomposition along z (the host side) against the single-domain oracle, on CPU.

Each slab is the oracle stand-in of tests/slab_oracle.py, so what is tested here is the
decomposition itself: the z-ranges, the faces each slab sends, the ghost planes they land in,
the periodic wrap, the initial ghosts and the FP64 reduction over slabs. Collisions are local
and the pulls are the same, so every own cell must match the single-domain run to rounding
(the oracle's torch reductions round differently on differently shaped tensors, by an ulp or
so; a wrong face or plane is off by O(u) = 1e-2).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle.collision import Params
from oracle.solver import OracleSim
from paper_1202_6074_gb300 import slab as SL
from slab_oracle import OracleSlab

NX, NY, NZ, STEPS = 6, 5, 7, 4
TOL = 1e-14


def _same(a, b):
    return float((a - b).abs().max()) <= TOL


def _case(name):
    g = np.random.default_rng(7)
    rho = 1.0 + 0.01 * g.standard_normal((NZ, NY, NX))
    u = 0.03 * g.standard_normal((3, NZ, NY, NX))
    F = 1e-4 * g.standard_normal((3, NZ, NY, NX))
    uw = [[[0.0] * 3 for _ in range(2)] for _ in range(3)]
    if name == "periodic_field":
        return dict(params=Params(tau=0.6, omega_bulk=1.0), bc_xy=("periodic", "periodic"), uw=uw, vd=None,
                    uniform=(0.0, 0.0, 0.0), field=F, rho=rho, u=u)
    if name == "walls_les":
        uw[1][1][0] = 0.04                                  # moving lid on the upper y wall
        u[:, :, 0, :] = 0.0
        u[:, :, -1, :] = 0.0
        return dict(params=Params(tau=0.52, omega_bulk=1.0, cs_smag=0.15), bc_xy=("bounceback", "bounceback"),
                    uw=uw, vd=(26.0, 2.0), uniform=(1e-5, 0.0, 0.0), field=None, rho=rho, u=u)
    if name == "factorized_reduced":
        return dict(params=Params(tau=0.7, omega_bulk=1.2, attractor="factorized", reduced_compressibility=True),
                    bc_xy=("periodic", "bounceback"), uw=uw, vd=None, uniform=(0.0, 2e-5, 1e-5), field=None,
                    rho=rho, u=u)
    raise KeyError(name)


def _single(c):
    o = OracleSim("D3Q27", NX, NY, NZ, c["params"], bc=c["bc_xy"] + ("periodic",), wall_velocity=c["uw"],
                  van_driest=c["vd"])
    o.set_force(c["uniform"], None if c["field"] is None else torch.tensor(c["field"]))
    o.init(torch.tensor(c["rho"]), torch.tensor(c["u"]))
    o.step(STEPS)
    rho, u = o.moments()
    return rho, u, o.reduce()


def _slab(c, z0, nzl):
    sl = slice(z0, z0 + nzl)
    e = OracleSlab(NX, NY, nzl, c["params"], c["bc_xy"], c["uw"], c["vd"], c["uniform"],
                   None if c["field"] is None else c["field"][:, sl])
    e.init(c["rho"][sl], c["u"][:, sl])
    return e


def test_split_is_balanced_and_covers():
    assert SL.split(7, 3) == [(0, 3), (3, 2), (5, 2)]
    assert SL.split(8, 1) == [(0, 8)]
    for nz in range(1, 20):
        for k in range(1, nz + 1):
            parts = SL.split(nz, k)
            assert sum(n for _, n in parts) == nz
            assert all(parts[r + 1][0] == parts[r][0] + parts[r][1] for r in range(k - 1))
            assert max(n for _, n in parts) - min(n for _, n in parts) <= 1
    with pytest.raises(ValueError):
        SL.split(2, 3)


@pytest.mark.parametrize("name", ["periodic_field", "walls_les", "factorized_reduced"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_local_exchange_matches_single_domain(name, k):
    c = _case(name)
    rho_ref, u_ref, red_ref = _single(c)
    engines = [_slab(c, z0, n) for z0, n in SL.split(NZ, k)]
    run = SL.SlabRun(engines, SL.LocalExchange(engines))
    run.step(STEPS)
    rho = torch.cat([e.moments()[0] for e in engines], dim=0)
    u = torch.cat([e.moments()[1] for e in engines], dim=1)
    assert _same(rho, rho_ref)
    assert _same(u, u_ref)
    red = run.reduce()
    scale = [abs(red_ref[0])] + [abs(red_ref[0]) * 0.05] * 3 + [abs(red_ref[4]) + 1e-30]
    for a, b, s in zip(red, red_ref, scale):
        assert abs(a - b) <= 1e-13 * s


def test_a_planted_exchange_mistake_is_caught():
    """Swapping the two faces (a plausible wiring slip) must break the match."""
    c = _case("periodic_field")
    rho_ref, _, _ = _single(c)

    class Swapped(SL.LocalExchange):
        def exchange(self):
            k = len(self.engines)
            tops = [e.pack(SL.FACE_TOP) for e in self.engines]
            bottoms = [e.pack(SL.FACE_BOTTOM) for e in self.engines]
            for r in range(k):
                self.engines[(r - 1) % k].unpack(SL.FACE_BOTTOM, tops[r])
                self.engines[(r + 1) % k].unpack(SL.FACE_TOP, bottoms[r])

    engines = [_slab(c, z0, n) for z0, n in SL.split(NZ, 3)]
    SL.SlabRun(engines, Swapped(engines)).step(STEPS)
    rho = torch.cat([e.moments()[0] for e in engines], dim=0)
    assert not torch.allclose(rho, rho_ref, rtol=0, atol=1e-12)


def test_dist_exchange_without_a_process_group_is_its_own_neighbour():
    c = _case("periodic_field")
    rho_ref, u_ref, _ = _single(c)
    e = _slab(c, 0, NZ)
    ex = SL.DistExchange(e)
    assert ex.world == 1
    SL.SlabRun([e], ex).step(STEPS)
    rho, u = e.moments()
    assert _same(rho, rho_ref) and _same(u, u_ref)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, name, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = _case(name)
        z0, nzl = SL.split(NZ, world)[rank]
        e = _slab(c, z0, nzl)
        run = SL.SlabRun([e], SL.DistExchange(e))
        run.step(STEPS)
        rho, u = e.moments()
        out[rank] = (z0, rho.numpy().tobytes(), u.numpy().tobytes(), nzl, run.reduce())
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(180)
@pytest.mark.parametrize("world,name", [(2, "periodic_field"), (3, "walls_les")])
def test_gloo_ranks_match_single_domain(world, name):
    c = _case(name)
    rho_ref, u_ref, red_ref = _single(c)
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, name, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(160)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    rho = torch.zeros_like(rho_ref)
    u = torch.zeros_like(u_ref)
    for r in range(world):
        z0, rb, ub, nzl, red = res[r]
        rho[z0:z0 + nzl] = torch.from_numpy(np.frombuffer(rb, dtype=np.float64).reshape(nzl, NY, NX).copy())
        u[:, z0:z0 + nzl] = torch.from_numpy(np.frombuffer(ub, dtype=np.float64).reshape(3, nzl, NY, NX).copy())
        # every rank holds the same all-reduced sums
        for a, b in zip(red, red_ref):
            assert abs(a - b) <= 1e-13 * max(abs(red_ref[0]), 1.0)
    assert _same(rho, rho_ref)
    assert _same(u, u_ref)
