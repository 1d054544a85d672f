"""Benchmark of the cascaded central-moment stream-and-collide step (one JSON line on rank 0).

Workload (N=1): D3Q27 FP32 decaying Taylor-Green vortex on a 256^3 periodic box, u0 = 0.05,
Re = 1600 (tau from Re and L/(2 pi)), no eddy viscosity. A step is one launch of the fused
pull + collide + store kernel over all 16.8 M cells. The state (2 x 1.81 GB) is far larger
than the 129 MB L2, so no flush is needed between steps.

Also reported (same JSON line, "forms"): BF16 / FP16 storage of the same workload, the
512^3 forced LES (Smagorinsky) in FP32 / BF16 / FP16, the 1024x256x256 BF16 wall-bounded LES
channel, and the adjoint rollout on 128^3 when available.

--impl reference times the FP64 CPU oracle (the only baseline: the paper has no code).
Multi-GPU: the path is timed as independent replicas (one full workload per rank, "weak").
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

# end-to-end job: upload (rho, u), initialise, E2E_STEPS steps, download (rho, u) and the sums
E2E_STEPS = 50
BYTES_PER_CELL = {("D3Q27", "f32"): 216, ("D3Q27", "bf16"): 108, ("D3Q27", "f16"): 108, ("D3Q27", "f64"): 432,
                  ("D2Q9", "f64"): 144, ("D2Q9", "f32"): 72}
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.txt")
FALLBACK_HBM = 6800.0
# bulk-viscosity rate of the trace of the second-order moments: free in the paper ("adjusted to
# improve numerical stability"); at tau -> 1/2 a bulk rate equal to the shear rate is unstable
OMEGA_BULK = 1.0
HIT_TAU = 0.5005       # base relaxation time of the forced isotropic turbulence LES
FILTERED_BYTES_PER_CELL = 136 + 36 + 40 + 228
ADJOINT_SEGMENT_BYTES_PER_CELL = 3 * 108 + 12 + 24


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="edge of the cubic box")
    ap.add_argument("--no-forms", action="store_true", help="skip the secondary forms")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--form-steps", type=int, default=40)
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16"],
                    help="population storage of the timed step (f32 is the headline)")
    ap.add_argument("--no-cpu-samples", action="store_true",
                    help="skip the oracle timings on reduced samples of the other workloads (about 15 s "
                         "of host-core work)")
    ap.add_argument("--flow", default="tgv", choices=["tgv", "hit"],
                    help="timed workload: the Taylor-Green vortex (headline) or the forced isotropic "
                         "turbulence LES (force field, Cs = 0.1) on the same n^3 box")
    ap.add_argument("--only", default=None, choices=["channel", "hit", "tgv", "adjoint", "d2q9"],
                    help="run only this form (16-bit storage by --storage, shape by --shape) and print its "
                         "MLUPS; for profiling captures of one kernel variant")
    ap.add_argument("--shape", default=None, help="nx,ny,nz of the --only form")
    ap.add_argument("--kernel", default="auto", choices=["auto", "direct", "pair", "pair_two_steps", "tma"],
                    help="step kernel: the library's choice (auto), one cell per thread (direct), two cells "
                         "per thread in packed FP32 (pair), or rows staged by TMA (tma)")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------
# distributed plumbing (replicas)
# ------------------------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist

            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v):
        if not self.pg:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------
class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # nvidia-smi takes a moment to start: wait for its first sample so that the
            # samples cover the timed region
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------
# helpers
# ------------------------------------------------------------------------------------------
def peaks():
    try:
        with open(PEAKS) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM}, "fallback"


# sources the direct D3Q27 step kernel is compiled from (and the flags it is built with)
KERNEL_SOURCES = ("paper_1202_6074_gb300/csrc/cm_core.cuh", "paper_1202_6074_gb300/csrc/cm_kernels.cuh",
                  "paper_1202_6074_gb300/csrc/cm_pair.cuh", "paper_1202_6074_gb300/csrc/cm_launch.h",
                  "paper_1202_6074_gb300/csrc/inst_d3q27_f32.cu", "paper_1202_6074_gb300/csrc/inst_pair_f32.cu",
                  "paper_1202_6074_gb300/build.py")


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def measured_traffic(key):
    """DRAM bytes per cell from the committed ncu summary, when the kernels are unchanged since."""
    try:
        rows = {}
        with open(TRAFFIC) as fh:
            for line in fh:
                if line.strip() and not line.startswith("#"):
                    k, v = line.split("=", 1)
                    rows[k.strip()] = v.strip()
        if rows.get("source_hash") != kernel_source_hash():
            return None
        v = rows.get(key)
        return float(v) if v else None
    except (OSError, ValueError):
        return None


def tgv_tau(n, u0=0.05, re=1600.0):
    return 3.0 * u0 * (n / (2 * math.pi)) / re + 0.5


def time_steps(solver, steps, warmup, dist, stream):
    solver.step(warmup)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    l0 = solver.launch_count
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    solver.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    return ms, solver.launch_count - l0


# ------------------------------------------------------------------------------------------
# forms
# ------------------------------------------------------------------------------------------
def run_tgv(cm, n, storage, steps, warmup, dist, clocks=None, kernel="auto", flow="tgv", repeats=0, **form):
    from paper_1202_6074_gb300 import workloads as W

    stream = torch.cuda.current_stream()
    if flow == "hit":
        s = cm.Solver(lattice="D3Q27", nx=n, ny=n, nz=n, storage=storage, tau=HIT_TAU, smagorinsky_cs=0.1,
                      omega_bulk=OMEGA_BULK, kernel=kernel)
        F = W.hit_forcing(n, n, n, seed=1, xp=torch, device="cuda")
        s.set_force((0, 0, 0), F)
        del F
        s.init()
    else:
        s = cm.Solver(lattice="D3Q27", nx=n, ny=n, nz=n, storage=storage, tau=tgv_tau(n), omega_bulk=OMEGA_BULK,
                      kernel=kernel, **form)
        rho, u = W.taylor_green(n, n, n, u0=0.05, xp=torch, device="cuda")
        s.init(rho, u)
        del rho, u
    if clocks:
        clocks.start()
    ms, launches = time_steps(s, steps, warmup, dist, stream)
    rep = None
    if clocks and repeats:
        # beside the contractual region of exactly `steps` steps: `repeats` regions of at least
        # 200 steps each (a short region is dominated by launch and clock jitter)
        k = max(steps, 200)
        rep = [time_steps(s, k, 0, dist, stream)[0] / k for _ in range(repeats)]
    ck = clocks.stop() if clocks else None
    red = s.reduce()
    kernel_used = s.step_kernel
    s.close()
    if rep is not None:
        ck = dict(ck or {})
        ck["repeats_ms_per_step"] = rep
    return ms, launches, ck, red, kernel_used


def run_poiseuille(cm, steps=5000):
    """The D2Q9 FP64 body-force channel, 64 x 32, 5000 steps (2048 cells: launch bound; the
    library replays pairs of steps as CUDA graphs)."""
    stream = torch.cuda.current_stream()
    s = cm.Solver(lattice="D2Q9", nx=64, ny=32, nz=1, storage="f64", tau=0.8,
                  bc=("periodic", "bounceback", "periodic"))
    s.set_force((1e-6, 0.0, 0.0))
    s.init()
    ms, launches = time_steps(s, steps, 10, Dist0(), stream)
    red = s.reduce()
    s.close()
    sec = ms / 1e3
    return {"MLUPS": 64 * 32 * steps / sec / 1e6, "us_per_step": 1e6 * sec / steps, "steps": steps,
            "launches": int(launches), "mean_ux": red[1] / red[0]}


def _events_ms(fn, stream):
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def run_filtered(cm, n, steps):
    """Turbulence as forcing (the filtered equation) on the Taylor-Green flow: every step
    recomputes the closure force (three kernels) and then steps; FP32, n^3 periodic, factorized
    attractor and reduced compressibility as for the filtered form."""
    from paper_1202_6074_gb300 import workloads as W

    stream = torch.cuda.current_stream()
    s = cm.Solver(lattice="D3Q27", nx=n, ny=n, nz=n, storage="f32", tau=0.5005, omega_bulk=OMEGA_BULK,
                  attractor="factorized", reduced_compressibility=True)
    rho, u = W.taylor_green(n, n, n, u0=0.05, xp=torch, device="cuda")
    s.init(rho, u)
    del rho, u
    s.step_filtered(3, 0.1)
    l0 = s.launch_count
    ms = _events_ms(lambda: s.step_filtered(steps, 0.1), stream)
    launches = s.launch_count - l0
    s.close()
    mlups = n ** 3 * steps / (ms / 1e3) / 1e6
    # bytes per cell of one filtered step: (rho, u) pass 108 + 12 read, 16 written; eddy stress
    # 12 read, 24 written; closure force 24 + 4 read, 12 written; step 216 + 12
    bpc = FILTERED_BYTES_PER_CELL
    return {"MLUPS": mlups, "hbm_frac": bpc * mlups / 1e3 / peaks()[0]["hbm_gbs"], "bytes_per_cell": bpc,
            "steps": steps, "launches_per_step": launches / steps}


def run_slabs(cm, n, k, steps, overlap=True):
    """The Taylor-Green workload split into k z-slabs on this GPU, faces exchanged every step
    (in-process exchange): the cost of the decomposition against one domain. overlap: split steps,
    the exchange running while the interior planes are updated."""
    from paper_1202_6074_gb300 import slab as SL, workloads as W

    stream = torch.cuda.current_stream()
    rho, u = W.taylor_green(n, n, n, u0=0.05, xp=torch, device="cuda")
    slabs = []
    for r in range(k):
        s, z0 = SL.cuda_slab(cm, n, r, k, lattice="D3Q27", nx=n, ny=n, storage="f32", tau=tgv_tau(n),
                             omega_bulk=OMEGA_BULK)
        s.init(rho[z0:z0 + s.shape[0]].contiguous(), u[:, z0:z0 + s.shape[0]].contiguous())
        slabs.append(s)
    del rho, u
    run = SL.SlabRun(slabs, SL.LocalExchange(slabs), overlap=overlap)
    run.step(3)
    ms = _events_ms(lambda: run.step(steps), stream)
    red = run.reduce()
    for s in slabs:
        s.close()
    return {"MLUPS": n ** 3 * steps / (ms / 1e3) / 1e6, "slabs": k, "steps": steps, "overlap": overlap,
            "mass": red[0]}


def run_hit_les(cm, n, storage, steps, warmup, dist):
    from paper_1202_6074_gb300 import workloads as W

    s = cm.Solver(lattice="D3Q27", nx=n, ny=n, nz=n, storage=storage, tau=HIT_TAU, smagorinsky_cs=0.1,
                  omega_bulk=OMEGA_BULK)
    F = W.hit_forcing(n, n, n, seed=1, xp=torch, device="cuda")
    s.set_force((0, 0, 0), F)
    del F
    s.init()
    ms, launches = time_steps(s, steps, warmup, dist, torch.cuda.current_stream())
    s.close()
    return ms, launches


def run_channel(cm, storage, steps, warmup, dist, nx=1024, ny=256, nz=256):
    u_tau, h = 0.005, ny / 2
    nu0 = u_tau * h / 180.0
    s = cm.Solver(lattice="D3Q27", nx=nx, ny=ny, nz=nz, storage=storage, tau=3 * nu0 + 0.5, smagorinsky_cs=0.1,
                  van_driest=(26.0, u_tau / nu0), bc=("periodic", "bounceback", "periodic"), omega_bulk=OMEGA_BULK)
    s.set_force((u_tau * u_tau / h, 0.0, 0.0))
    # laminar-shape start scaled to the bulk speed, with seeded noise (device generator)
    y = (torch.arange(ny, device="cuda", dtype=torch.float64) + 0.5).view(1, ny, 1)
    shape = 6.0 * y * (ny - y) / ny ** 2
    ub = 15.7 * u_tau
    g = torch.Generator(device="cuda").manual_seed(5)
    u = 0.05 * 1.5 * ub * torch.randn((3, nz, ny, nx), generator=g, device="cuda", dtype=torch.float64) * (shape / 1.5)
    u[0] += ub * shape
    s.init(None, u)
    del u
    ms, launches = time_steps(s, steps, warmup, dist, torch.cuda.current_stream())
    s.close()
    return ms, launches


def e2e(cm, n, storage, steps, kernel="auto", repeats=5, dist=None):
    """Whole job through the C ABI with host buffers: upload (rho, u) from pinned memory, init,
    `steps` steps, download (rho, u) and the FP64 reductions; wall clock around all of it. The
    job is repeated `repeats` times (a new handle each time) and the median run is reported: the
    host link is shared with the machine's other GPUs, and a download occasionally stalls for
    tens of ms (every run is listed). With several ranks every rank runs its own job at the
    same time (a barrier before each run) and a run's value is the cells of all ranks over the
    slowest rank's wall clock."""
    dist = dist or Dist0()
    world = getattr(dist, "world", 1)
    from paper_1202_6074_gb300 import workloads as W

    rho, u = W.taylor_green(n, n, n, u0=0.05, xp=torch, device="cuda")
    rho_h = rho.cpu().pin_memory()
    u_h = u.cpu().pin_memory()
    del rho, u
    rho_o = torch.empty_like(rho_h).pin_memory()
    u_o = torch.empty_like(u_h).pin_memory()
    N = n ** 3
    runs = []
    for _ in range(repeats):
        s = cm.Solver(lattice="D3Q27", nx=n, ny=n, nz=n, storage=storage, tau=tgv_tau(n), omega_bulk=OMEGA_BULK,
                      kernel=kernel)
        lib = s.lib
        P = cm._ptr
        torch.cuda.synchronize()
        dist.barrier()
        t0 = time.perf_counter()
        s._check(lib.cmlbm_init(s.h, P(rho_h), P(u_h), cm.HOST))
        ta = time.perf_counter()
        s.step(steps)
        s._check(lib.cmlbm_moments(s.h, P(rho_o), P(u_o), cm.HOST))
        tb = time.perf_counter()
        red = s.reduce()
        t1 = time.perf_counter()
        s.close()
        assert math.isfinite(red[0])
        wall = dist.max(t1 - t0)
        # wall-clock split (this rank): upload + init, steps + moments download (the steps run
        # asynchronously until the download waits for them), reduction
        runs.append((world * N * steps / wall / 1e6,
                     {"init": 1e3 * (ta - t0), "steps_and_moments": 1e3 * (tb - ta), "reduce": 1e3 * (t1 - tb)}))
    best = sorted(runs, key=lambda r: r[0])[len(runs) // 2]
    return {"value": best[0], "unit": "MLUPS", "h2d_bytes_per_step": 32 * N / steps,
            "d2h_bytes_per_step": (32 * N + 40) / steps, "steps": steps, "split_ms": best[1],
            "runs_MLUPS": [r[0] for r in runs]}


def _oracle_mlups(n, steps):
    from oracle.solver import OracleSim
    from oracle.collision import Params
    from paper_1202_6074_gb300 import workloads as W

    rho, u = W.taylor_green(n, n, n, u0=0.05)
    o = OracleSim("D3Q27", n, n, n, Params(tau=tgv_tau(n), omega_bulk=OMEGA_BULK))
    o.init(torch.tensor(rho), torch.tensor(u))
    t0 = time.perf_counter()
    o.step(steps)
    t1 = time.perf_counter()
    return n ** 3 * steps / (t1 - t0) / 1e6, t1 - t0


def cpu_baseline(n=64, steps=50, n1=40, steps1=4):
    """The FP64 oracle on a bounded sample of the workload (a Taylor-Green box of n^3, about 10 s
    on 16 host cores), plus a smaller sample on one core."""
    import platform

    v, sec = _oracle_mlups(n, steps)
    threads = torch.get_num_threads()
    torch.set_num_threads(1)
    try:
        v1, sec1 = _oracle_mlups(n1, steps1)
    finally:
        torch.set_num_threads(threads)
    return {"value": v, "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": f"D3Q27 FP64 Taylor-Green {n}^3 x {steps} steps (same flow, smaller box)", "seconds": sec,
            "host": {"machine": platform.machine(), "cpus": os.cpu_count(), "affinity": len(os.sched_getaffinity(0))},
            "one_core": {"value": v1, "sample": f"{n1}^3 x {steps1} steps", "seconds": sec1}}


def cpu_samples():
    """The FP64 oracle on reduced samples of the other workloads (host cores, MLUPS each): the
    D2Q9 body-force channel (1000 of its 5000 steps), the forced isotropic LES and the wall-bounded
    channel LES on small boxes, and the adjoint (forward + reverse by automatic differentiation
    through the oracle) on a 16^3 box."""
    from oracle import adjoint as A
    from oracle.solver import OracleSim
    from oracle.collision import Params
    from paper_1202_6074_gb300 import workloads as W

    out = {}

    def timed(name, sample, cells, steps, fn):
        t0 = time.perf_counter()
        fn()
        sec = time.perf_counter() - t0
        out[name] = {"MLUPS": cells * steps / sec / 1e6, "sample": sample, "seconds": sec}

    o = OracleSim("D2Q9", 64, 32, 1, Params(tau=0.8), bc=("periodic", "bounceback", "periodic"))
    o.set_force((1e-6, 0.0, 0.0))
    o.init(None, None)
    timed("d2q9_poiseuille64x32", "64x32 x 1000 steps", 64 * 32, 1000, lambda: o.step(1000))

    n = 32
    o = OracleSim("D3Q27", n, n, n, Params(tau=HIT_TAU, cs_smag=0.1))
    o.set_force(field=torch.tensor(W.hit_forcing(n, n, n, seed=1)))
    o.init(None, None)
    timed("hit_les", f"{n}^3 x 10 steps, force field, Smagorinsky", n ** 3, 10, lambda: o.step(10))

    nx, ny, nz = 64, 32, 16
    rho, u, F = W.channel(nx, ny, nz, seed=5)
    o = OracleSim("D3Q27", nx, ny, nz, Params(tau=0.51067, cs_smag=0.1), bc=("periodic", "bounceback", "periodic"),
                  van_driest=(26.0, 0.005 / ((0.51067 - 0.5) / 3)))
    o.set_force((1.953e-7, 0.0, 0.0))
    o.init(torch.tensor(rho), torch.tensor(u))
    timed("channel_les", f"{nx}x{ny}x{nz} x 10 steps, walls, Smagorinsky + van Driest", nx * ny * nz, 10,
          lambda: o.step(10))

    n = 16
    p = Params(tau=0.6)
    rho, u0 = W.random_solenoidal(n, n, n, seed=2, u_rms=0.02)
    F = torch.tensor(W.gaussian_force(n, n, n, seed=3, std=1e-5))
    sim = OracleSim("D3Q27", n, n, n, p)
    sim.set_force(field=F)
    sim.init(torch.tensor(rho), torch.tensor(u0))
    s0 = sim.s.clone()
    target = torch.zeros((3, n, n, n), dtype=torch.float64)
    timed("adjoint", f"{n}^3 x 10 steps forward + reverse", n ** 3, 10,
          lambda: A.loss_and_grad(("D3Q27", n, n, n, p), s0, F, target, 10))
    return out


# ------------------------------------------------------------------------------------------
# arms
# ------------------------------------------------------------------------------------------
def workload_config(n, st, world, flow="tgv"):
    """The benchmark's workload description (shared by both arms)."""
    N = n ** 3
    half = BYTES_PER_CELL[("D3Q27", st)] / 2 * N
    if flow == "hit":
        name = (f"D3Q27 CM-LBM {st.upper()} forced isotropic turbulence {n}^3 periodic, shells |k| <= 2 "
                f"(seed 1), Smagorinsky Cs=0.1 (tau0={HIT_TAU}, bulk rate {OMEGA_BULK})")
    else:
        name = (f"D3Q27 CM-LBM {st.upper()} decaying Taylor-Green vortex {n}^3 periodic, u0=0.05, "
                f"Re=1600, no LES (tau={tgv_tau(n):.6f}, bulk rate {OMEGA_BULK})")
    return {"workload": name,
            "cells": N, "l2": "state 2 x %.2f GB %s 129 MB L2, no flush" % (half / 1e9, ">>" if half > 129e6 else "vs"),
            "parallelism": "replicas" if world > 1 else "single GPU"}


def reference_arm(args, dist):
    """The oracle as it stands, timed on the host cores: each step = one oracle step on a 32^3
    Taylor-Green sample of the 256^3 workload."""
    if dist.rank != 0:
        return
    from oracle.solver import OracleSim
    from oracle.collision import Params
    from paper_1202_6074_gb300 import workloads as W

    # sample edge sized so that warm-up + timed steps stay near a minute on the host cores
    # (about 0.4 M cell updates/s): n^3 (steps + warmup) <= 24e6, 8 <= n <= 32
    n = int(max(8, min(32, (24e6 / max(1, args.steps + args.warmup)) ** (1.0 / 3.0))))
    rho, u = W.taylor_green(n, n, n, u0=0.05)
    o = OracleSim("D3Q27", n, n, n, Params(tau=tgv_tau(args.n), omega_bulk=OMEGA_BULK))
    o.init(torch.tensor(rho), torch.tensor(u))
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    t1 = time.perf_counter()
    v = n ** 3 * args.steps / (t1 - t0) / 1e6
    sample = f"D3Q27 FP64 Taylor-Green {n}^3 per step (sample of the {args.n}^3 workload)"
    print(json.dumps({
        "impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * (t1 - t0) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.n, "f32", dist.world),
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": torch.get_num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def our_arm(args, dist):
    import __graft_entry__ as G

    G.build()
    from paper_1202_6074_gb300 import cmlbm as cm

    torch.cuda.set_device(dist.local)
    n = args.n
    N = n ** 3
    pk, pk_kind = peaks()
    clocks = Clocks(dist.local)
    st = args.storage
    hit = args.flow == "hit"
    ms, launches, ck, red, kname = run_tgv(cm, n, st, args.steps, args.warmup, dist, clocks, kernel=args.kernel,
                                           flow=args.flow, repeats=5)
    rep = (ck or {}).pop("repeats_ms_per_step", None)
    ms = dist.max(ms)
    per_launch_s = ms / 1e3 / args.steps
    value = dist.world * N * args.steps / (ms / 1e3) / 1e6
    bpc = BYTES_PER_CELL[("D3Q27", st)] + (12 if hit else 0)      # + the FP32 force field
    achieved = bpc * N / per_launch_s / 1e9
    traffic_pc = None if hit else measured_traffic(f"k_step_d3q27_{st}_periodic_{kname}")
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": st, "data": "synthetic",
        "config": workload_config(n, st, dist.world, args.flow),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "peak_kind": pk_kind,
                     "traffic": None if traffic_pc is None else traffic_pc * N,
                     "algorithmic_bytes_per_cell": bpc,
                     "kernel": {"tma": "k_step_tma", "pair": "k_step_pair", "direct": "k_step",
                                "pair_two_steps": "k_step_pair (two steps per pass)"}[kname]
                               + f"<D3Q27,{st},periodic{',LES,force field' if hit else ''}>"},
        "clocks": ck,
        "gpu_launches": int(launches),
        "repeats": None if not rep else {
            "steps_each": max(args.steps, 200), "ms_per_step": rep,
            "median_MLUPS": dist.world * N / (float(np.median(rep)) / 1e3) / 1e6,
            "note": "5 further timed regions of at least 200 steps after the contractual one (same handle)"},
        "diagnostics": {"mass": red[0], "kinetic_energy": red[4]},
    }
    # the end-to-end job is the Taylor-Green one (host fields rho, u in, rho, u out), on every rank
    torch.cuda.empty_cache()
    line["e2e"] = None if hit else e2e(cm, n, st, E2E_STEPS, kernel=args.kernel, dist=dist)
    if dist.rank == 0:
        forms = {}
        if not args.no_forms:
            fs = args.form_steps
            for st in ("bf16", "f16"):
                m, l, _, _, _ = run_tgv(cm, n, st, fs, 3, Dist0())
                sec = m / 1e3 / fs
                forms[f"tgv{n}_{st}"] = {"MLUPS": N / sec / 1e6, "hbm_frac": BYTES_PER_CELL[("D3Q27", st)] * N / sec / 1e9
                                         / pk["hbm_gbs"], "steps": fs}
            # the general collision forms (Secs. 12 and 13) on the same flow
            for name, form in (("factorized", dict(attractor="factorized")),
                               ("reduced", dict(reduced_compressibility=True, rho0=1.0))):
                for st in ("f32", "bf16"):
                    m, l, _, _, _ = run_tgv(cm, n, st, fs, 3, Dist0(), **form)
                    sec = m / 1e3 / fs
                    forms[f"tgv{n}_{name}_{st}"] = {"MLUPS": N / sec / 1e6, "hbm_frac": BYTES_PER_CELL[("D3Q27", st)] * N
                                                    / sec / 1e9 / pk["hbm_gbs"], "steps": fs}
            # 512^3, and 576^3 (27 N = 5.2e9 >= 2^32: the kernels with 64-bit element offsets)
            for nh, storages in ((512, ("f32", "bf16", "f16")), (576, ("bf16",))):
                for st in storages:
                    try:
                        m, l = run_hit_les(cm, nh, st, fs, 3, Dist0())
                        sec = m / 1e3 / fs
                        bpc_f = BYTES_PER_CELL[("D3Q27", st)] + 12
                        forms[f"hit{nh}_les_{st}"] = {"MLUPS": nh ** 3 / sec / 1e6,
                                                      "hbm_frac": bpc_f * nh ** 3 / sec / 1e9 / pk["hbm_gbs"],
                                                      "bytes_per_cell": bpc_f, "steps": fs,
                                                      "offsets": "64-bit" if 27 * nh ** 3 >= 2 ** 32 else "32-bit"}
                    except Exception as e:  # noqa: BLE001
                        forms[f"hit{nh}_les_{st}"] = {"error": str(e)[:200]}
                    torch.cuda.empty_cache()
            try:
                m, l = run_channel(cm, "bf16", fs, 3, Dist0())
                sec = m / 1e3 / fs
                nc = 1024 * 256 * 256
                forms["channel1024x256x256_les_bf16"] = {"MLUPS": nc / sec / 1e6, "hbm_frac": 108 * nc / sec / 1e9
                                                         / pk["hbm_gbs"], "steps": fs}
            except Exception as e:  # noqa: BLE001
                forms["channel1024x256x256_les_bf16"] = {"error": str(e)[:200]}
            torch.cuda.empty_cache()
            try:
                forms["filtered_hit256_f32"] = run_filtered(cm, 256, fs)
            except Exception as e:  # noqa: BLE001
                forms["filtered_hit256_f32"] = {"error": str(e)[:200]}
            for key, ov in (("slabs2_tgv256_f32", True), ("slabs2_serial_tgv256_f32", False)):
                try:
                    forms[key] = run_slabs(cm, n, 2, fs, overlap=ov)
                    forms[key]["vs_single_domain"] = forms[key]["MLUPS"] / value
                except Exception as e:  # noqa: BLE001
                    forms[key] = {"error": str(e)[:200]}
            torch.cuda.empty_cache()
            torch.cuda.empty_cache()
            try:
                forms["d2q9_poiseuille64x32_f64"] = run_poiseuille(cm)
            except Exception as e:  # noqa: BLE001
                forms["d2q9_poiseuille64x32_f64"] = {"error": str(e)[:200]}
            try:
                from paper_1202_6074_gb300 import rollout

                forms["adjoint128_f32"] = rollout.benchmark(cm, n=128, steps=500, segment=50)
            except Exception as e:  # noqa: BLE001
                forms["adjoint128_f32"] = {"error": str(e)[:200]}
        # the 16-bit and adjoint forms against the plain FP32 step of the same flow on this GPU
        if args.storage == "f32" and not hit:
            for k in (f"tgv{n}_bf16", f"tgv{n}_f16"):
                if "MLUPS" in forms.get(k, {}):
                    forms[k]["vs_fp32_step"] = forms[k]["MLUPS"] / value
        h32 = forms.get("hit512_les_f32", {}).get("MLUPS")
        for k in ("hit512_les_bf16", "hit512_les_f16"):
            if h32 and "MLUPS" in forms.get(k, {}):
                forms[k]["vs_fp32_step"] = forms[k]["MLUPS"] / h32
        adj = forms.get("adjoint128_f32", {})
        if "forward_MLUPS" in adj:
            adj["backward_vs_forward"] = adj["backward_MLUPS"] / adj["forward_MLUPS"]
            adj["fwd_plus_adjoint_vs_forward"] = adj["fwd_plus_adjoint_MLUPS"] / adj["forward_MLUPS"]
        if "adjoint_step_us" in adj:
            # a step inside a checkpoint segment: state, lambda in and out (27 x 4 B each), the
            # force field (12 B) and the FP32 segment accumulator read and written (24 B)
            adj["adjoint_step_bytes_per_cell"] = ADJOINT_SEGMENT_BYTES_PER_CELL
            adj["adjoint_step_frac_of_hbm"] = (adj["adjoint_step_MLUPS"] * ADJOINT_SEGMENT_BYTES_PER_CELL / 1e3
                                               / peaks()[0]["hbm_gbs"])
        line["forms"] = forms
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline()
            if not args.no_cpu_samples:
                line["cpu_baseline"]["other_workloads"] = cpu_samples()
        print(json.dumps(line))


class Dist0:
    """Rank-local timing for the secondary forms (no collective)."""

    world = 1

    def barrier(self):
        pass

    def max(self, v):
        return v


def only_form(args):
    """One form at a chosen shape (a profiling aid): --warmup steps, then --form-steps timed."""
    import __graft_entry__ as G

    G.build()
    from paper_1202_6074_gb300 import cmlbm as cm

    st = "bf16" if args.storage == "f32" and args.only == "channel" else args.storage
    if args.only == "adjoint":
        from paper_1202_6074_gb300 import rollout

        n = int((args.shape or "128").split(",")[0])
        out = rollout.benchmark(cm, n=n, steps=args.form_steps, segment=50)
        out["adjoint_step_frac_of_hbm"] = (out["adjoint_step_MLUPS"] * ADJOINT_SEGMENT_BYTES_PER_CELL / 1e3
                                           / peaks()[0]["hbm_gbs"])
        print(json.dumps({"form": "adjoint", "shape": [n, n, n], "storage": "f32", **out}))
        return
    if args.only == "d2q9":
        out = run_poiseuille(cm, steps=args.form_steps)
        print(json.dumps({"form": "d2q9", "shape": [64, 32, 1], "storage": "f64", **out}))
        return
    if args.only == "channel":
        nx, ny, nz = (int(v) for v in (args.shape or "1024,256,256").split(","))
        ms, _ = run_channel(cm, st, args.form_steps, args.warmup, Dist0(), nx=nx, ny=ny, nz=nz)
        bpc = BYTES_PER_CELL[("D3Q27", st)]
    elif args.only == "hit":
        nx, ny, nz = (int(v) for v in (args.shape or "512,512,512").split(","))
        assert nx == ny == nz, "the forced isotropic turbulence form runs on a cube"
        ms, _ = run_hit_les(cm, nx, st, args.form_steps, args.warmup, Dist0())
        bpc = BYTES_PER_CELL[("D3Q27", st)] + 12
    else:
        nx, ny, nz = (int(v) for v in (args.shape or "256,256,256").split(","))
        assert nx == ny == nz, "the Taylor-Green form runs on a cube"
        ms, _, _, _, _ = run_tgv(cm, nx, st, args.form_steps, args.warmup, Dist0())
        bpc = BYTES_PER_CELL[("D3Q27", st)]
    N = nx * ny * nz
    mlups = N * args.form_steps / (ms / 1e3) / 1e6
    print(json.dumps({"form": args.only, "shape": [nx, ny, nz], "storage": st, "steps": args.form_steps,
                      "MLUPS": mlups, "GBs": bpc * mlups / 1e3, "bytes_per_cell": bpc}))


def main():
    args = parse()
    if args.only:
        only_form(args)
        return
    dist = Dist()
    try:
        if args.impl == "reference":
            reference_arm(args, dist)
        else:
            our_arm(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
