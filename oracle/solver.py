"""The oracle time loop: pull-stream, collide, diagnostics.

Test infrastructure (see the package docstring).

State convention (shared with the CUDA library's interface, not its code): ``s[i, z, y, x]``
holds the post-collision transformed population of cell (x, y, z) in direction i, as plain
float64 values f (the library stores d = f / w_i - 1 in its storage type). One step pulls
g = stream(s) and stores s <- collide(g).
"""
import torch

from .lattice import DT, get as get_lattice
from . import collision as C
from . import stream as ST
from . import les as L
from . import filtered as FL


STORAGE_DTYPES = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


def round_to_storage(s, w, storage):
    """The stored state of a library run in `storage`: each population as its deviation from the
    rest weight, d = f / w - 1, rounded to the nearest value of the storage type (ties to even;
    torch's conversion, a library primitive), then decoded f = w (1 + d) in float64. None or
    "f64" leaves s unchanged. Paper silent (storage formats are not in the paper)."""
    if storage in (None, "f64"):
        return s
    wv = w.view(-1, *([1] * (s.dim() - 1)))
    d = (s / wv - 1.0).to(STORAGE_DTYPES[storage]).to(DT)
    return wv * (1.0 + d)


class OracleSim:
    def __init__(self, lattice, nx, ny, nz=1, params=None, bc=("periodic",) * 3,
                 wall_velocity=None, van_driest=None, storage=None):
        """van_driest = (A_plus, u_tau / nu_0) damps C_s by the distance to the y walls.
        storage = "f32" | "bf16" | "f16" rounds the stored state after initialisation and after
        every step as a library run with that storage does (round_to_storage); None keeps FP64."""
        self.lat = get_lattice(lattice) if isinstance(lattice, str) else lattice
        if self.lat.d == 2 and nz != 1:
            raise ValueError("D2Q9 needs nz = 1")
        self.shape = (nz, ny, nx)
        self.p = params if params is not None else C.Params()
        self.bc = tuple(bc)
        if wall_velocity is None:
            wall_velocity = [[[0.0] * 3 for _ in range(2)] for _ in range(3)]
        self.uw = wall_velocity
        self.F = torch.zeros((3,) + self.shape, dtype=DT)
        self.cs_eff = None
        if van_driest is not None and self.p.cs_smag > 0.0:
            aplus, utau_nu = van_driest
            self.cs_eff = L.van_driest_cs(self.p.cs_smag, ny, nz, nx, aplus, utau_nu, wall_axis=1)
        self.s = torch.zeros((self.lat.Q,) + self.shape, dtype=DT)
        self.storage = storage

    # ---- set-up -------------------------------------------------------------------
    def set_force(self, uniform=(0.0, 0.0, 0.0), field=None):
        """Body force F (Eqs. densitycalculation, velocitycalculation): a uniform vector plus an optional [3, ...] field."""
        self.F_uniform = torch.zeros((3,) + self.shape, dtype=DT)
        for d in range(3):
            self.F_uniform[d] += float(uniform[d])
        if field is not None:
            self.F = torch.as_tensor(field, dtype=DT).reshape((3,) + self.shape).clone()
        else:
            self.F = self.F_uniform.clone()

    def init(self, rho=None, u=None):
        """Pre-collision field fbar = f^M(rho, u) - S/2 (paper silent on initialisation)."""
        rho = torch.ones(self.shape, dtype=DT) if rho is None else torch.as_tensor(rho, dtype=DT).reshape(self.shape)
        u = torch.zeros((3,) + self.shape, dtype=DT) if u is None else torch.as_tensor(u, dtype=DT).reshape((3,) + self.shape)
        if self.p.reduced_compressibility:
            # Sec. 12: the momentum is rho0 u, so the equilibrium is centred on rho0 u / rho
            u = u * (self.p.rho0 / rho)
        fbar = C.equilibrium(rho, u, self.F, self.lat)
        self.s = round_to_storage(ST.unstream(fbar, self.lat, self.bc, self.uw), self.lat.w, self.storage)

    def set_state(self, s):
        """Replace the stored post-collision populations (FP64)."""
        self.s = torch.as_tensor(s, dtype=DT).reshape((self.lat.Q,) + self.shape).clone()

    # ---- dynamics -----------------------------------------------------------------
    def pre_collision(self):
        """The streamed field fbar_alpha(x) = s_alpha(x - e_alpha) (Eq. cascadedstreaming1) with the boundaries."""
        return ST.pull(self.s, self.lat, self.bc, self.uw)

    def step(self, n=1):
        """n steps of stream and collide (procedure of Sec. 11)."""
        for _ in range(n):
            g = self.pre_collision()
            self.s = round_to_storage(C.collide(g, self.F, self.lat, self.p, self.cs_eff), self.lat.w, self.storage)

    def turbulence_force(self, cs):
        """Set F = rho a' from the Smagorinsky closure of the current resolved field (Sec. 14)."""
        if any(b != ST.PERIODIC for b in self.bc):
            raise ValueError("turbulence forcing needs periodic boundaries")
        rho, u = self.moments()
        base = getattr(self, "F_uniform", torch.zeros_like(self.F))
        self.F = rho * FL.turbulence_acceleration(u, cs, self.lat.d) + base

    def step_filtered(self, n, cs):
        """n steps of the filtered equation: closure force, then a step (Sec. 14 reading)."""
        for _ in range(n):
            self.turbulence_force(cs)
            self.step(1)

    # ---- diagnostics --------------------------------------------------------------
    def moments(self):
        """(rho, u) of the current pre-collision field (Eqs. densitycalculation, velocitycalculation)."""
        return C.hydrodynamics(self.pre_collision(), self.F, self.lat, self.p)

    def reduce(self):
        """[sum rho, sum rho u_x, sum rho u_y, sum rho u_z, sum rho |u|^2 / 2] (paper silent)."""
        rho, u = self.moments()
        return [float(rho.sum()), float((rho * u[0]).sum()), float((rho * u[1]).sum()),
                float((rho * u[2]).sum()), float((0.5 * rho * (u * u).sum(0)).sum())]


def collide_cells(g, F, lattice, params, cs_eff=None):
    """Collision of a batch of independent cells: g[Q, n], F[3, n] (no streaming)."""
    lat = get_lattice(lattice) if isinstance(lattice, str) else lattice
    return C.collide(g, F, lat, params, cs_eff)
