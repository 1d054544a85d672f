"""A CPU stand-in for one z-slab, stepped by the FP64 oracle (test infrastructure).

It keeps the library's slab layout -- state [Q][nz + 2][ny][nx] with a ghost plane below and
above the slab's own planes -- and implements the engine interface of
``paper_1202_6074_gb300.slab`` (step, pack, unpack, reduce, moments) with the oracle's pull and
collision. Stepping the padded grid as if it were periodic in z changes nothing in the own
planes (their pulls never wrap); whatever lands in the ghost planes is overwritten by the next
exchange. Initialisation mirrors the library: the inverse pull of the own planes' pre-collision
field, with the entries that point into the ghost planes kept.
"""
import torch

from oracle import collision as C
from oracle import les as L
from oracle import stream as ST
from oracle.lattice import DT, get as get_lattice

FACE_BOTTOM, FACE_TOP = 0, 1


class OracleSlab:
    def __init__(self, nx, ny, nzl, params, bc_xy=("periodic", "periodic"), wall_velocity=None, van_driest=None,
                 uniform=(0.0, 0.0, 0.0), field=None):
        self.lat = get_lattice("D3Q27")
        self.p = params
        self.nzl = nzl
        self.pad = (nzl + 2, ny, nx)
        self.bc = (bc_xy[0], bc_xy[1], ST.PERIODIC)
        if wall_velocity is None:
            wall_velocity = [[[0.0] * 3 for _ in range(2)] for _ in range(3)]
        self.uw = wall_velocity
        F = torch.zeros((3,) + self.pad, dtype=DT)
        for d in range(3):
            F[d] += float(uniform[d])
        if field is not None:
            F[:, 1:-1] = torch.as_tensor(field, dtype=DT)
        self.F = F
        self.cs_eff = None
        if van_driest is not None and params.cs_smag > 0.0:
            self.cs_eff = L.van_driest_cs(params.cs_smag, ny, nzl + 2, nx, van_driest[0], van_driest[1], wall_axis=1)
        self.up = [i for i in range(self.lat.Q) if int(self.lat.e[i, 2]) == 1]
        self.down = [i for i in range(self.lat.Q) if int(self.lat.e[i, 2]) == -1]
        self.s = torch.zeros((self.lat.Q,) + self.pad, dtype=DT)

    def init(self, rho, u):
        rho = torch.as_tensor(rho, dtype=DT)
        u = torch.as_tensor(u, dtype=DT)
        if self.p.reduced_compressibility:     # as the single-domain oracle: centre on rho0 u / rho
            u = u * (self.p.rho0 / rho)
        fbar = torch.zeros((self.lat.Q,) + self.pad, dtype=DT)
        fbar[:, 1:-1] = C.equilibrium(rho, u, self.F[:, 1:-1], self.lat)
        self.s = ST.unstream(fbar, self.lat, self.bc, self.uw)

    def step(self, n=1):
        for _ in range(n):
            g = ST.pull(self.s, self.lat, self.bc, self.uw)
            self.s = C.collide(g, self.F, self.lat, self.p, self.cs_eff)

    def pack(self, face, host=False):
        if face == FACE_TOP:
            return self.s[self.up, self.nzl].clone()
        return self.s[self.down, 1].clone()

    def unpack(self, face, msg):
        msg = torch.as_tensor(msg, dtype=DT)
        if face == FACE_BOTTOM:
            self.s[self.up, 0] = msg
        else:
            self.s[self.down, self.nzl + 1] = msg

    def moments(self):
        g = ST.pull(self.s, self.lat, self.bc, self.uw)[:, 1:-1]
        return C.hydrodynamics(g, self.F[:, 1:-1], self.lat, self.p)

    def reduce(self):
        rho, u = self.moments()
        return [float(rho.sum()), float((rho * u[0]).sum()), float((rho * u[1]).sum()),
                float((rho * u[2]).sum()), float((0.5 * rho * (u * u).sum(0)).sum())]
