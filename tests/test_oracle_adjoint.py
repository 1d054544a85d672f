"""Pin of the oracle gradient dL/dF (autograd through the oracle) by central finite differences."""
import numpy as np
import pytest
import torch

from oracle import adjoint as A
from oracle.solver import OracleSim
from oracle.collision import Params
from paper_1202_6074_gb300 import workloads as W

DT = torch.float64


@pytest.mark.parametrize("lattice,shape,bc", [
    ("D3Q27", (5, 6, 4), ("periodic",) * 3),
    ("D2Q9", (1, 7, 6), ("periodic", "bounceback", "periodic")),
])
def test_oracle_gradient_matches_central_differences(lattice, shape, bc):
    nz, ny, nx = shape
    p = Params(tau=0.6, omega3=1.1, omega4=0.9)
    rho, u = W.random_solenoidal(nx, ny, nz, seed=2, u_rms=0.03)
    if lattice == "D2Q9":
        u[2] = 0
    F0 = W.gaussian_force(nx, ny, nz, seed=3, std=1e-3)
    if lattice == "D2Q9":
        F0[2] = 0
    target = torch.tensor(W.gaussian_force(nx, ny, nz, seed=4, std=1e-2))
    sim = OracleSim(lattice, nx, ny, nz, p, bc=bc)
    sim.set_force(field=torch.tensor(F0))
    sim.init(torch.tensor(rho), torch.tensor(u))
    s0 = sim.s.clone()
    args = (lattice, nx, ny, nz, p)
    kw = {"bc": bc}
    steps = 4
    L, g = A.loss_and_grad(args, s0, torch.tensor(F0), target, steps, kw)
    rng = np.random.default_rng(0)
    comps = 2 if lattice == "D2Q9" else 3
    for _ in range(8):
        idx = (int(rng.integers(comps)), int(rng.integers(nz)), int(rng.integers(ny)), int(rng.integers(nx)))
        h = 1e-5
        Fp = torch.tensor(F0)
        Fm = torch.tensor(F0)
        Fp[idx] += h
        Fm[idx] -= h
        with torch.no_grad():
            lp = float(A.velocity_loss(args, s0, Fp, target, steps, kw))
            lm = float(A.velocity_loss(args, s0, Fm, target, steps, kw))
        fd = (lp - lm) / (2 * h)
        assert abs(fd - float(g[idx])) <= 1e-4 * abs(fd) + 1e-12, (idx, fd, float(g[idx]))
