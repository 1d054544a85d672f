"""Differentiable rollout: dL/dF of a loss on the final velocity, by the hand-written adjoint.

``velocity_after(solver, F, s0, steps, segment)`` returns u_T ([3, nz, ny, nx], float64) after
``steps`` stream-and-collide steps from the fixed state ``s0`` under the force field F, as a
torch.autograd.Function. Its backward runs the adjoint kernels of libcmlbm.so:

  forward   s_{t+1} = step(s_t, F); a checkpoint is kept every ``segment`` steps
  backward  lambda_T = pull^T (du_T/dg)^T dL/du_T           (cmlbm_adjoint_terminal)
            for each segment, last first: recompute its states from the checkpoint
            (cmlbm_step_buffers; the last segment's states are kept from the forward sweep),
            then lambda_t = J_t^T lambda_{t+1} and dL/dF += ... (cmlbm_step_adjoint_segment):
            the force gradient of a segment is summed in the arithmetic precision and added
            into the FP64 dL/dF once per segment.
Memory: ceil(steps / segment) checkpoints plus one segment of states, instead of all steps.
The initial state s0 is an input held fixed (its own dependence on F is not differentiated).
"""
import time

import torch

from . import cmlbm as _cm


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, solver, s0, steps, segment):
        solver.set_force((0.0, 0.0, 0.0), F.detach())
        nseg = (steps + segment - 1) // segment
        last = (nseg - 1) * segment          # first step of the last segment
        ckpts = [s0.detach().clone()]
        # the states of the last segment, s_last .. s_(steps-1), are written by the forward steps
        # into buffers that are kept for the backward sweep (which then need not recompute them)
        tail = [ckpts[0]] if last == 0 else []
        cur = ckpts[0]
        ping = [solver.new_state(), solver.new_state()]
        for t in range(steps):
            if t + 1 >= last and t + 1 > 0:
                nxt = solver.new_state()
            else:
                nxt = ping[t % 2]
            solver.step_buffers(cur, nxt)
            cur = nxt
            if t + 1 < last and (t + 1) % segment == 0:
                ckpts.append(cur.clone())
            if last <= t + 1 < steps:
                if t + 1 == last:
                    ckpts.append(cur)
                tail.append(cur)
        _, u = solver.moments(state=cur)
        ctx.solver, ctx.steps, ctx.segment = solver, steps, segment
        ctx.ckpts = ckpts
        ctx.tail = tail
        ctx.final = cur
        ctx.F = F.detach()
        return u

    @staticmethod
    def backward(ctx, gu):
        solver, steps, segment = ctx.solver, ctx.steps, ctx.segment
        solver.set_force((0.0, 0.0, 0.0), ctx.F)
        dev = solver.device
        shape = (solver.Q,) + solver.shape
        lam = torch.empty(shape, dtype=solver.real_dtype, device=dev)
        lam2 = torch.empty_like(lam)
        dLdF = torch.zeros((3,) + solver.shape, dtype=torch.float64, device=dev)
        # the force gradient of the steps of one segment is summed in the arithmetic precision and
        # folded into the FP64 dLdF at the segment's first step
        seg = torch.zeros((3,) + solver.shape, dtype=solver.real_dtype, device=dev)
        solver.adjoint_terminal(ctx.final, gu.detach().to(torch.float64).contiguous(), lam, dLdF)
        nseg = (steps + segment - 1) // segment
        buf = [None] * segment
        for k in reversed(range(nseg)):
            start, end = k * segment, min((k + 1) * segment, steps)
            if k == nseg - 1:
                states = ctx.tail
            else:
                buf[0] = ctx.ckpts[k]
                for t in range(start + 1, end):
                    j = t - start
                    if buf[j] is None or buf[j] is buf[0]:
                        buf[j] = solver.new_state()
                    solver.step_buffers(buf[j - 1], buf[j])
                states = buf
            for t in reversed(range(start, end)):
                solver.step_adjoint_segment(states[t - start], lam, lam2, seg, dLdF, fold=(t == start))
                lam, lam2 = lam2, lam
        ctx.tail = None
        return dLdF, None, None, None, None


def velocity_after(solver, F, s0, steps, segment=50):
    """u_T (float64 CUDA tensor [3, nz, ny, nx]) as a differentiable function of F."""
    if steps < 1:
        raise ValueError("steps must be >= 1")
    return _Rollout.apply(F, solver, s0, int(steps), int(max(1, segment)))


def benchmark(cm, n=128, steps=100, segment=50):
    """Forward rollout and its adjoint on the n^3 adjoint workload (FP32 storage)."""
    from . import workloads as W

    s = cm.Solver(lattice="D3Q27", nx=n, ny=n, nz=n, storage="f32", tau=0.6)
    rho, u0 = W.random_solenoidal(n, n, n, seed=2, u_rms=0.02)
    F = torch.tensor(W.gaussian_force(n, n, n, seed=3, std=1e-5), device="cuda")
    s.set_force((0, 0, 0), F)
    s.init(torch.tensor(rho, device="cuda"), torch.tensor(u0, device="cuda"))
    s0 = s.get_state()
    target = torch.zeros((3, n, n, n), dtype=torch.float64, device="cuda")
    Fp = F.clone().requires_grad_(True)
    # warm-up with one full segment, so that the caching allocator already holds the segment's
    # state buffers when the timed rollout runs (as in every iteration after the first of a loop)
    u = velocity_after(s, Fp, s0, segment + 1, segment)
    ((u - target) ** 2).sum(0).mean().backward()
    torch.cuda.synchronize()
    Fp.grad = None
    l0 = s.launch_count
    t0 = time.perf_counter()
    u = velocity_after(s, Fp, s0, steps, segment)
    loss = ((u - target) ** 2).sum(0).mean()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    N = n ** 3
    out = {"forward_MLUPS": N * steps / (t1 - t0) / 1e6, "backward_MLUPS": N * steps / (t2 - t1) / 1e6,
           "fwd_plus_adjoint_MLUPS": N * steps / (t2 - t0) / 1e6, "steps": steps, "segment": segment,
           "launches": s.launch_count - l0, "grad_norm": float(Fp.grad.norm())}
    # the adjoint step alone (CUDA events on the handle's stream, which is the current stream):
    # a step inside a segment (FP32 accumulator) and a folding step (FP32 into FP64)
    lam = torch.zeros((s.Q,) + s.shape, dtype=torch.float32, device="cuda")
    lam2 = torch.empty_like(lam)
    seg = torch.zeros((3,) + s.shape, dtype=torch.float32, device="cuda")
    dLdF = torch.zeros((3,) + s.shape, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for fold, key in ((False, "adjoint_step_us"), (True, "adjoint_fold_step_us")):
        for _ in range(3):
            s.step_adjoint_segment(s0, lam, lam2, seg, dLdF, fold)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        e0.record(stream)
        for _ in range(reps):
            s.step_adjoint_segment(s0, lam, lam2, seg, dLdF, fold)
        e1.record(stream)
        torch.cuda.synchronize()
        out[key] = e0.elapsed_time(e1) * 1e3 / reps
    out["adjoint_step_MLUPS"] = N / out["adjoint_step_us"]
    s.close()
    return out


__all__ = ["velocity_after", "benchmark", "_cm"]
