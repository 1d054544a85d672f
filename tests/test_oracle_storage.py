"""Pins of the oracle's storage emulation (oracle/solver.py: round_to_storage).

A library run with 16-bit (or FP32) storage keeps each population as its deviation from the
rest weight, d = f / w - 1, rounded to nearest (ties to even) in the storage type after every
step. The oracle can apply the same rounding to its FP64 state, which separates what the
storage format costs in accuracy from what the kernels add.

  * The rounding itself is checked against brute force: every finite bit pattern of BF16
    (8 exponent bits, 7 fraction bits) and FP16 (5 exponent bits, 10 fraction bits) decoded
    by the IEEE-754 rule, the nearest one taken for each input, ties to the even pattern.
  * The format's effect on a Taylor-Green run: the velocity error against the FP64 run grows
    with the storage type's unit roundoff (FP16's 2^-11 against BF16's 2^-8, a ratio of 8),
    and BF16 alone exceeds 2e-3 on the fluctuation u - U of a flow with a background velocity U.
"""
import numpy as np
import pytest
import torch

import oracle.solver as SV
from oracle.collision import Params
from oracle.lattice import get as get_lattice
from paper_1202_6074_gb300 import workloads as W


def _all_values(exp_bits, frac_bits):
    """All finite values of a binary floating-point format, and whether each pattern is even."""
    bias = (1 << (exp_bits - 1)) - 1
    vals, even = [], []
    for bits in range(1 << (1 + exp_bits + frac_bits)):
        sign = bits >> (exp_bits + frac_bits)
        e = (bits >> frac_bits) & ((1 << exp_bits) - 1)
        m = bits & ((1 << frac_bits) - 1)
        if e == (1 << exp_bits) - 1:
            continue                                   # infinities and NaNs
        if e == 0:
            v = m * 2.0 ** (1 - bias - frac_bits)      # subnormals and zero
        else:
            v = (1.0 + m / 2.0 ** frac_bits) * 2.0 ** (e - bias)
        vals.append(-v if sign else v)
        even.append(m % 2 == 0)
    v = np.array(vals)
    order = np.argsort(v, kind="stable")
    return v[order], np.array(even)[order]


def _nearest_even(x, vals, even):
    out = np.empty_like(x)
    for k, xv in enumerate(x):
        dist = np.abs(vals - xv)
        best = np.flatnonzero(dist == dist.min())
        cand = vals[best]
        if len(np.unique(cand)) > 1:                   # a tie between two neighbours
            evens = best[even[best]]
            out[k] = vals[evens[0]]
        else:
            out[k] = cand[0]
    return out


FORMATS = {"bf16": (8, 7), "f16": (5, 10)}


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_round_to_storage_is_the_nearest_value_ties_to_even(storage):
    vals, even = _all_values(*FORMATS[storage])
    rng = np.random.default_rng(7)
    # deviations of the size the library stores, tiny ones, and the exact midpoints between
    # neighbours (all exactly representable in float32, so torch's path through float32 is exact)
    x = np.concatenate([
        rng.uniform(-0.6, 0.6, 300),
        rng.uniform(-1e-3, 1e-3, 100),
        np.sign(rng.standard_normal(60)) * 10.0 ** rng.uniform(-7, -2, 60),
    ]).astype(np.float32).astype(np.float64)
    k = rng.integers(0, len(vals) - 1, 200)
    mids = 0.5 * (vals[k] + vals[k + 1])
    mids = mids[(np.abs(mids) < 1.0) & (np.abs(mids) > 2.0 ** -20)]
    exact = vals[(np.abs(vals) < 1.0) & (np.abs(vals) > 2.0 ** -20)][::97]
    x = np.concatenate([x, mids, exact])
    want = _nearest_even(x, vals, even)
    w = torch.ones(1, dtype=torch.float64)
    got = SV.round_to_storage(torch.tensor(1.0 + x).view(1, -1), w, storage).view(-1).numpy() - 1.0
    # 1 + x is exact in float64 for every x above (at most 24 significant bits, |x| < 1)
    assert np.array_equal(got, want), np.flatnonzero(got != want)[:10]


def test_round_to_storage_fp64_and_none_are_identity():
    s = torch.rand(27, 3, 4, 5, dtype=torch.float64)
    w = get_lattice("D3Q27").w
    assert torch.equal(SV.round_to_storage(s, w, None), s)
    assert torch.equal(SV.round_to_storage(s, w, "f64"), s)


def _tgv_error(storage, background, n=10, steps=40):
    rho, u = W.taylor_green(n, n, n, u0=0.05, background=background)
    res = {}
    for st in (None, storage):
        o = SV.OracleSim("D3Q27", n, n, n, Params(tau=0.55), storage=st)
        o.init(torch.tensor(rho), torch.tensor(u))
        o.step(steps)
        res[st] = o.moments()[1]
    bg = torch.tensor(background, dtype=torch.float64).view(3, 1, 1, 1)
    a, b = res[storage] - bg, res[None] - bg
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_storage_error_scales_with_the_unit_roundoff():
    """The velocity error a storage type causes scales with its unit roundoff: FP16 (2^-11)
    against BF16 (2^-8) gives a ratio near 1/8. In a frame moving at U the fluctuation u - U is
    what the flow carries, while the stored deviations carry U too, so BF16 alone exceeds the
    2e-3 target there; FP16 stays well inside it."""
    bg = (0.05, 0.03, 0.0)
    e_bf16 = _tgv_error("bf16", bg)
    e_f16 = _tgv_error("f16", bg)
    e_f32 = _tgv_error("f32", bg)
    assert 0.06 < e_f16 / e_bf16 < 0.25, (e_f16, e_bf16)
    assert e_bf16 > 2e-3
    assert e_f16 < 2e-3
    assert e_f32 < 1e-5
