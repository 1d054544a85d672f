"""The oracle's pins catch plausible mistakes: each test plants one mistake in the oracle (on the
CPU, through monkeypatch) and runs the fast pin tests; at least one of them must fail.

The mistakes are the ones a restatement of the paper could plausibly make: a dropped or
sign-flipped F/2 in the velocity, a source without its sigma/2 feedback or with the wrong
factor, a wrong Maxwellian moment, central moments about the wrong velocity, a transposed
stream, swapped third/fourth-order rates, a wrong eddy-viscosity
constant, a flipped moving-wall term, an initial state without its -S/2 term, 3D factorized
attractors built over the wrong axes, divided by one power of rho too many, from the
pre-collision second-order moments, or non-zero where a factor vanishes, in the turbulence closure an eddy stress without its
factor 2, an unsymmetrised strain rate and a van Driest wall distance without the half cell,
reduced compressibility ignored in the velocity, the trace relaxed with the shear rate, a
storage emulation that truncates the deviations or rounds the populations themselves, a halved
moving-wall term, an inverse transform about zero velocity and a source with F instead of F/rho.
"""
import dataclasses
import inspect
import os

import pytest
import torch

import test_oracle_basis as TB
import test_oracle_collision as TC
import test_oracle_filtered as TFI
import test_oracle_flows as TF
import test_oracle_les as TL
import test_oracle_storage as TS
from oracle import collision as C
from oracle import filtered as FL
from oracle import les as L
from oracle import moments as M
from oracle import solver as SV
from oracle import stream as ST

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SLOW = {"test_poiseuille_exact_with_magic_parameter", "test_poiseuille_default_rates_wall_error_is_small",
        "test_couette_exact", "test_galilean_invariance_of_taylor_green_decay",
        "test_storage_error_scales_with_the_unit_roundoff"}


def _calls(module, include_slow=()):
    """(name, thunk) for every test function of a module, expanded over its parametrizations."""
    out = []
    for name, fn in inspect.getmembers(module, inspect.isfunction):
        if not name.startswith("test_") or (name in SLOW and name not in include_slow):
            continue
        params = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
        sig = inspect.signature(fn).parameters
        kw = {"golden_dir": GOLDEN} if "golden_dir" in sig else {}
        combos = [dict(kw)]
        for m in params:
            names = [s.strip() for s in m.args[0].split(",")] if isinstance(m.args[0], str) else list(m.args[0])
            new = []
            for c in combos:
                for v in m.args[1]:
                    vals = v if len(names) > 1 else (v,)
                    d = dict(c)
                    d.update(zip(names, vals))
                    new.append(d)
            combos = new
        for c in combos:
            out.append((f"{module.__name__}::{name}{c}", (lambda f=fn, c=c: f(**c))))
    return out


def _failures(include_slow=(), first=False):
    """Names of the pins that fail (only the first one with first=True)."""
    failed = []
    for mod in (TB, TC, TF, TL, TFI, TS):
        for name, thunk in _calls(mod, include_slow):
            try:
                thunk()
            except Exception:  # noqa: BLE001  (a pin that fails, however it fails)
                failed.append(name)
                if first:
                    return failed
    return failed


def test_the_pins_pass_without_a_mistake():
    assert _failures() == []


def _wrap(monkeypatch, module, name, make):
    orig = getattr(module, name)
    monkeypatch.setattr(module, name, make(orig))


def _source_without_feedback(kbar, rho, F, lat):
    """The hierarchical identity applied to kbar instead of kappa = kbar + sigma/2."""
    idx = {a: k for k, a in enumerate(lat.monomials)}
    sigma, kappa = [None] * len(idx), [None] * len(idx)
    for a in lat.monomials:
        k = idx[a]
        s = torch.zeros_like(rho)
        for d in range(3):
            if a[d] > 0:
                lower = list(a)
                lower[d] -= 1
                s = s + a[d] * (F[d] / rho) * kappa[idx[tuple(lower)]]
        sigma[k] = s
        n = sum(a)
        kappa[k] = rho if n == 0 else torch.zeros_like(rho) if n == 1 else kbar[k]
    return torch.stack(sigma), torch.stack(kappa)


MUTATIONS = {
    "velocity without F/2": lambda mp: _wrap(mp, C, "hydrodynamics",
                                             lambda f: lambda fbar, F, lat, p=None: f(fbar, 0 * F, lat, p)),
    "velocity with -F/2": lambda mp: _wrap(mp, C, "hydrodynamics",
                                           lambda f: lambda fbar, F, lat, p=None: f(fbar, -F, lat, p)),
    "source doubled": lambda mp: _wrap(mp, C, "source_central",
                                       lambda f: lambda kbar, rho, F, lat: (lambda s, k: (2 * s, k))(*f(kbar, rho, F, lat))),
    "source without sigma/2 feedback": lambda mp: mp.setattr(C, "source_central", _source_without_feedback),
    "fourth-order Maxwellian moment off": lambda mp: _wrap(
        mp, C, "maxwell_central",
        lambda f: lambda rho, lat: f(rho, lat) * torch.tensor(
            [1.05 if sum(a) == 4 else 1.0 for a in lat.monomials], dtype=rho.dtype).view(-1, *([1] * rho.dim()))),
    "central moments about -u": lambda mp: _wrap(mp, M, "central_moments", lambda f: lambda g, u, lat: f(g, -u, lat)),
    "stream transposed": lambda mp: mp.setattr(ST, "pull", lambda s, lat, bc, uw, _u=ST.unstream: _u(s, lat, bc, uw)),
    "third and fourth rates swapped": lambda mp: _wrap(
        mp, C, "collide",
        lambda f: lambda fbar, F, lat, p, cs_eff=None: f(fbar, F, lat, type(p)(**{**p.__dict__, "omega3": p.omega4,
                                                                                 "omega4": p.omega3}), cs_eff)),
    "eddy viscosity constant 18 instead of 18 sqrt 2": lambda mp: _wrap(
        mp, L, "tau_effective",
        lambda f: lambda tau0, cs, Pi, rho: f(tau0, cs / 2 ** 0.25, Pi, rho)),
    "moving-wall term flipped": lambda mp: _wrap(
        mp, ST, "_wall_terms",
        lambda f: lambda lat, i, shape, bc, uw, sign: (lambda m, w: (m, -w))(*f(lat, i, shape, bc, uw, sign))),
    "moving-wall term halved": lambda mp: _wrap(
        mp, ST, "_wall_terms",
        lambda f: lambda lat, i, shape, bc, uw, sign: (lambda m, w: (m, 0.5 * w))(*f(lat, i, shape, bc, uw, sign))),
    "initial state without -S/2": lambda mp: _wrap(mp, C, "equilibrium", lambda f: lambda rho, u, F, lat: f(rho, u, 0 * F, lat)),
    "inverse transform about zero velocity": lambda mp: _wrap(
        mp, M, "central_to_populations", lambda f: lambda kappa, u, lat: f(kappa, 0 * u, lat)),
    "source with F instead of F / rho": lambda mp: _wrap(
        mp, C, "source_central", lambda f: lambda kbar, rho, F, lat: f(kbar, rho, F * rho, lat)),
    "eddy stress without its factor 2": lambda mp: _wrap(
        mp, FL, "eddy_stress", lambda f: lambda u, cs, d: {k: 0.5 * v for k, v in f(u, cs, d).items()}),
    "strain rate not symmetrised": lambda mp: mp.setattr(
        FL, "strain_rate", lambda u, d: {(i, j): FL._d(u[j], i) for i in range(d) for j in range(d)}),
    "van Driest wall distance without the half cell": lambda mp: mp.setattr(L, "van_driest_cs", _vd_full_cells),
    "factorized (2,2,0) over the wrong axes": lambda mp: _wrap(mp, C, "_factorized_attractor",
                                                              _wrong_axes((2, 2, 0), (2, 0, 0), (0, 0, 2))),
    "factorized (2,0,2) over the wrong axes": lambda mp: _wrap(mp, C, "_factorized_attractor",
                                                              _wrong_axes((2, 0, 2), (2, 0, 0), (0, 2, 0))),
    "factorized products over rho^k instead of rho^(k-1)": lambda mp: _wrap(mp, C, "_factorized_attractor",
                                                                           _extra_rho),
    "factorized from the pre-collision second-order moments": lambda mp: _pre_collision_factors(mp),
    "factorized (2,1,1) with the wrong off-diagonal": lambda mp: _wrap(mp, C, "_factorized_attractor",
                                                                      _wrong_axes((2, 1, 1), (2, 0, 0), (1, 1, 0))),
    "factorized (1,2,1) with the wrong diagonal": lambda mp: _wrap(mp, C, "_factorized_attractor",
                                                                  _wrong_axes((1, 2, 1), (2, 0, 0), (1, 0, 1))),
    "reduced compressibility ignored (u = j / rho)": lambda mp: _wrap(mp, C, "hydrodynamics", _without_reduced),
    "trace relaxed with the shear rate": lambda mp: _wrap(mp, C, "collide", _bulk_as_shear),
    "stored deviations truncated instead of rounded": lambda mp: mp.setattr(SV, "round_to_storage", _truncated_storage),
    "stored populations rounded instead of their deviations": lambda mp: mp.setattr(SV, "round_to_storage",
                                                                                   _rounded_populations),
    "factorized (2,2,1) not zero": lambda mp: _wrap(mp, C, "_factorized_attractor",
                                                    _wrong_axes((2, 2, 1), (2, 0, 0), (0, 1, 1))),
}


def _without_reduced(f):
    """The velocity j / rho even where reduced compressibility asks for j / rho0."""
    def g(fbar, F, lat, p=None):
        if p is not None and p.reduced_compressibility:
            p = dataclasses.replace(p, reduced_compressibility=False)
        return f(fbar, F, lat, p)
    return g


def _bulk_as_shear(f):
    """The trace of the second-order moments relaxed with the shear rate, whatever omega_bulk says."""
    def g(fbar, F, lat, p, cs_eff=None):
        return f(fbar, F, lat, dataclasses.replace(p, omega_bulk=0.0), cs_eff)
    return g


def _truncated_storage(s, w, storage):
    """Deviations cut toward zero to the storage type's precision (the low bits of the float32
    pattern dropped) instead of rounded to nearest."""
    if storage in (None, "f64"):
        return s
    wv = w.view(-1, *([1] * (s.dim() - 1)))
    cut = {"bf16": 16, "f16": 13, "f32": 0}[storage]
    d = (s / wv - 1.0).to(torch.float32)
    d = (d.view(torch.int32) & -(1 << cut)).view(torch.float32).to(torch.float64)
    return wv * (1.0 + d)


def _rounded_populations(s, w, storage):
    """The populations f themselves rounded to the storage type instead of their deviations d."""
    if storage in (None, "f64"):
        return s
    return s.to(SV.STORAGE_DTYPES[storage]).to(torch.float64)


def _extra_rho(f):
    """Every factorized product of order >= 3 divided by rho once more."""
    def g(kM, post2, rho, lat):
        out = f(kM, post2, rho, lat)
        for k, a in enumerate(lat.monomials):
            if sum(a) >= 3:
                out[k] = out[k] / rho
        return out
    return g


def _pre_collision_factors(mp):
    """The factorized attractor built from the pre-collision second-order central moments (the
    collision's own central-moment transform is recorded and its values used in place of the
    relaxed ones)."""
    seen = {}
    orig_cm = M.central_moments

    def central_moments(f, u, lat):
        out = orig_cm(f, u, lat)
        seen["k"] = out
        return out

    orig_fa = C._factorized_attractor

    def factorized(kM, post2, rho, lat):
        pre = post2.clone()
        for k, a in enumerate(lat.monomials):
            if sum(a) == 2:
                pre[k] = seen["k"][k]
        return orig_fa(kM, pre, rho, lat)

    mp.setattr(M, "central_moments", central_moments)
    mp.setattr(C, "_factorized_attractor", factorized)


def _vd_full_cells(cs, ny, nz, nx, aplus, utau_over_nu, wall_axis=1):
    """van Driest damping with the wall distance counted in whole cells (y = j) instead of to
    the half-way wall (y = j + 1/2)."""
    n = (nx, ny, nz)[wall_axis]
    j = torch.arange(n, dtype=torch.float64)
    y = torch.minimum(j, n - 1.0 - j)
    c = cs * (1.0 - torch.exp(-(y * utau_over_nu) / aplus))
    shape = [1, 1, 1]
    shape[2 - wall_axis] = n
    full = [nz, ny, nx]
    return c.view(*shape).expand(*full).clone()


def _wrong_axes(target, m1, m2):
    """The factorized attractor of `target` built from the relaxed second-order moments m1, m2
    of the wrong pair of axes."""
    def make(f):
        def g(kM, post2, rho, lat):
            out = f(kM, post2, rho, lat)
            idx = {a: k for k, a in enumerate(lat.monomials)}
            if target in idx and m1 in idx and m2 in idx:
                out[idx[target]] = post2[idx[m1]] * post2[idx[m2]] / rho
            return out
        return g
    return make


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_a_planted_mistake_fails_a_pin(monkeypatch, name):
    MUTATIONS[name](monkeypatch)
    failed = _failures(first=True)
    if not failed:      # the slow closed-form flows are the last line
        failed = _failures(include_slow=SLOW, first=True)
    assert failed, f"no pin catches: {name}"
