"""Failure reporting through the C ABI, tested without any GPU fault.

* Divergence: a NaN written into one stored population (host data, through cmlbm_set_state)
  must make cmlbm_reduce return CMLBM_ERR_DIVERGED, and the handle must work again once a clean
  state is set.
* A TMA-staged step whose bounded pipeline wait gives up stores 1 into the handle's device flag.
  The test hook CMLBM_TEST_PIPELINE_FAULT makes the library write that value itself after each
  batch of TMA-staged steps (no kernel is made to wait in vain); every call that returns results
  must then report CMLBM_ERR_CUDA once, and the handle must recover.
"""
import math

import pytest
import torch

from paper_1202_6074_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cm():
    import __graft_entry__ as G

    G.build()
    from paper_1202_6074_gb300 import cmlbm

    return cmlbm


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_reduce_reports_a_nan_population_as_divergence(cm, storage):
    n = 8
    rho, u = W.taylor_green(n, n, n, u0=0.03)
    s = cm.Solver(lattice="D3Q27", nx=n, ny=n, nz=n, storage=storage, tau=0.6)
    s.init(torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"))
    clean = s.get_state()
    ref = s.reduce()
    assert all(math.isfinite(v) for v in ref)

    bad = clean.clone()
    bad[13, 3, 4, 5] = float("nan")          # the rest population of one cell
    s.set_state(bad)
    with pytest.raises(cm.CmlbmError) as e:
        s.reduce()
    assert e.value.code == cm.ERR_DIVERGED
    # a step spreads the NaN; the reduction still reports it
    s.step(2)
    with pytest.raises(cm.CmlbmError) as e:
        s.reduce()
    assert e.value.code == cm.ERR_DIVERGED

    # the handle recovers with a clean state and gives the same sums as before
    s.set_state(clean)
    assert s.reduce() == ref
    s.step(3)
    assert all(math.isfinite(v) for v in s.reduce())
    s.close()


def test_infinite_population_is_divergence(cm):
    n = 6
    s = cm.Solver(lattice="D3Q27", nx=n, ny=n, nz=n, storage="f32", tau=0.6)
    st = s.get_state()
    st[5, 1, 2, 3] = float("inf")
    s.set_state(st)
    with pytest.raises(cm.CmlbmError) as e:
        s.reduce()
    assert e.value.code == cm.ERR_DIVERGED
    s.close()


def _tma_solver(cm):
    nx, ny, nz = 128, 6, 5
    rho, u = W.taylor_green(nx, ny, nz, u0=0.03)
    s = cm.Solver(lattice="D3Q27", nx=nx, ny=ny, nz=nz, storage="f32", tau=0.6, kernel="tma")
    assert s.step_kernel == "tma"
    s.init(torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"))
    return s


def test_pipeline_flag_is_reported_by_reduce(cm, monkeypatch):
    s = _tma_solver(cm)
    s.step(2)
    assert all(math.isfinite(v) for v in s.reduce())
    monkeypatch.setenv("CMLBM_TEST_PIPELINE_FAULT", "1")
    s.step(2)
    monkeypatch.delenv("CMLBM_TEST_PIPELINE_FAULT")
    with pytest.raises(cm.CmlbmError) as e:
        s.reduce()
    assert e.value.code == cm.ERR_CUDA
    assert "pipeline" in str(e.value)
    # reported once: the flag is cleared and the handle steps on
    s.step(1)
    assert all(math.isfinite(v) for v in s.reduce())
    s.close()


@pytest.mark.parametrize("call", ["step", "step_buffers", "moments", "moments_host", "get_state"])
def test_pipeline_flag_is_reported_by_every_result_call(cm, monkeypatch, call):
    s = _tma_solver(cm)
    monkeypatch.setenv("CMLBM_TEST_PIPELINE_FAULT", "1")
    s.step(1)
    monkeypatch.delenv("CMLBM_TEST_PIPELINE_FAULT")
    torch.cuda.synchronize()                 # the flag's copy to the host has landed
    fns = {
        "step": lambda: s.step(1),
        "step_buffers": lambda: s.step_buffers(s.new_state().zero_(), s.new_state()),
        "moments": lambda: s.moments(),
        "moments_host": lambda: s.moments(host=True),
        "get_state": lambda: s.get_state(),
    }
    with pytest.raises(cm.CmlbmError) as e:
        fns[call]()
    assert e.value.code == cm.ERR_CUDA
    # the next call goes through
    fns[call]()
    torch.cuda.synchronize()
    assert all(math.isfinite(v) for v in s.reduce())
    s.close()
