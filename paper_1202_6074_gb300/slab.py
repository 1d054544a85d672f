"""Slab decomposition of a periodic-in-z D3Q27 domain: the host side of the face exchange.

The paper has no parallel decomposition. What is split is the standard streaming step (Eq.
cascadedstreaming1): a cell pulls s_i(x - e_i), so a z-slab reads from outside itself only the
9 populations with e_z = +1 of the plane just below it and the 9 with e_z = -1 of the plane
just above. Each slab is a library handle created with bc[2] = "halo" (one ghost plane on each
side); after every step the slabs trade those planes:

    my top face    (e_z = +1 of my last plane)  -> ghost below of the slab above
    my bottom face (e_z = -1 of my first plane) -> ghost above of the slab below

with periodic wrap (the last slab's "above" is the first). The library's initialisation writes
valid ghosts itself, so the first step needs no exchange. Collisions are local, so the
decomposed run reproduces the single-domain run cell for cell.

An engine is anything with ``step(n)``, ``pack(face)``, ``unpack(face, msg)`` and ``reduce()``:
a ``cmlbm.Solver`` created with bc z = "halo" (the product), or a CPU stand-in in the tests.
Exchanges:
  * ``LocalExchange``: all slabs in this process (one GPU, or the CPU tests);
  * ``DistExchange``: one slab per rank of a torch.distributed group. Each rank posts two sends
    and two receives per step (tags distinguish the two faces for backends that use them;
    the posting order matches the pairs for backends that match in order). With one rank the
    slab is its own neighbour on both sides.
"""
import torch
import torch.distributed as dist

FACE_BOTTOM, FACE_TOP = 0, 1
_TAG_UP, _TAG_DOWN = 11, 12      # top face travels up, bottom face travels down


def split(nz, parts):
    """Balanced z-ranges [(z0, nz_local)] of `parts` slabs; the first nz % parts get a plane more."""
    if parts < 1 or nz < parts:
        raise ValueError(f"cannot split {nz} planes into {parts} slabs")
    base, extra = divmod(nz, parts)
    out, z0 = [], 0
    for r in range(parts):
        n = base + (1 if r < extra else 0)
        out.append((z0, n))
        z0 += n
    return out


class LocalExchange:
    """Face exchange among slabs held in this process, listed in increasing z."""

    def __init__(self, engines):
        self.engines = list(engines)

    def exchange(self):
        k = len(self.engines)
        tops = [e.pack(FACE_TOP) for e in self.engines]
        bottoms = [e.pack(FACE_BOTTOM) for e in self.engines]
        for r in range(k):
            self.engines[(r + 1) % k].unpack(FACE_BOTTOM, tops[r])
            self.engines[(r - 1) % k].unpack(FACE_TOP, bottoms[r])

    def allreduce(self, sums):
        return sums


class DistExchange:
    """Face exchange of this rank's slab with its neighbours in a torch.distributed group.

    host = True stages the messages through pinned host memory (for a CPU backend such as gloo
    driving GPU engines); otherwise messages stay where the engine's pack puts them.
    """

    def __init__(self, engine, group=None, host=False):
        self.engine = engine
        self.group = group
        self.host = host
        self.on = dist.is_available() and dist.is_initialized()
        self.rank = dist.get_rank(group) if self.on else 0
        self.world = dist.get_world_size(group) if self.on else 1

    def _peer(self, r):
        r %= self.world
        return dist.get_global_rank(self.group, r) if self.group is not None else r

    def exchange(self):
        e = self.engine
        kw = {"host": True} if self.host else {}
        top = e.pack(FACE_TOP, **kw)
        bottom = e.pack(FACE_BOTTOM, **kw)
        if self.world == 1:
            e.unpack(FACE_BOTTOM, top)
            e.unpack(FACE_TOP, bottom)
            return
        up, down = self._peer(self.rank + 1), self._peer(self.rank - 1)
        below = torch.empty_like(top)
        above = torch.empty_like(bottom)
        if top.is_cuda:
            # the packs were issued on the engine's stream; the backend reads on its own
            torch.cuda.current_stream(top.device).synchronize()
        ops = [dist.P2POp(dist.isend, top, up, self.group, _TAG_UP),
               dist.P2POp(dist.isend, bottom, down, self.group, _TAG_DOWN),
               dist.P2POp(dist.irecv, below, down, self.group, _TAG_UP),
               dist.P2POp(dist.irecv, above, up, self.group, _TAG_DOWN)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        e.unpack(FACE_BOTTOM, below)
        e.unpack(FACE_TOP, above)

    def allreduce(self, sums):
        if self.world == 1:
            return sums
        t = torch.tensor(sums, dtype=torch.float64)
        dist.all_reduce(t, group=self.group)
        return [float(v) for v in t]


class SlabRun:
    """Time loop of a decomposed domain: step every slab, then refresh the ghosts.

    overlap = True steps engines that offer ``step_split`` (the library's cmlbm_step_split) in
    two parts: the boundary planes, whose faces the exchange then packs, on the engine's stream,
    and the interior planes on a stream of their own, so that the exchange of a step runs while
    the interior of that step is computed. The results are the same bit for bit. The boundary
    planes and the exchange then run on a CUDA stream of the highest priority (the library's
    interior stream has the lowest), which the run creates: during step() the engines launch on
    it, and at its end the caller's stream waits for it and the engines return to the caller's
    stream.
    """

    def __init__(self, engines, exchange, overlap=False):
        self.engines = list(engines)
        self.exchange = exchange
        self.overlap = overlap
        self.stream = None
        self._split = [e for e in self.engines if hasattr(e, "step_split") and hasattr(e, "set_stream")]
        if overlap and torch.cuda.is_available() and self._split:
            _, highest = torch.cuda.Stream.priority_range()
            self.stream = torch.cuda.Stream(device=self._split[0].device, priority=highest)

    def step(self, n=1):
        if self.stream is None:
            return self._step(n)
        caller = torch.cuda.current_stream(self.stream.device)
        self.stream.wait_stream(caller)
        for e in self._split:
            e.set_stream(self.stream)
        try:
            with torch.cuda.stream(self.stream):
                self._step(n)
        finally:
            caller.wait_stream(self.stream)
            for e in self._split:
                e.set_stream(caller)

    def _step(self, n):
        for _ in range(n):
            if self.overlap:
                # every slab's boundary planes first, then the interiors: a kernel issued after a
                # large one waits for the large one's blocks to be dispatched
                for e in self.engines:
                    if hasattr(e, "step_split"):
                        e.step_split(1)
                for e in self.engines:
                    if hasattr(e, "step_split"):
                        e.step_split(2)
                    else:
                        e.step(1)
            else:
                for e in self.engines:
                    e.step(1)
            self.exchange.exchange()
        if self.overlap:
            # order each engine's stream after its last interior launch (a zero-step call joins
            # it), so that work the caller issues on those streams next sees the whole state
            for e in self.engines:
                if hasattr(e, "step_split"):
                    e.step(0)

    def reduce(self):
        """{sum rho, sum j (3), sum rho |u|^2 / 2} over the whole domain (FP64; j = sum fbar e + F/2)."""
        local = [0.0] * 5
        for e in self.engines:
            r = e.reduce()
            local = [a + b for a, b in zip(local, r)]
        return self.exchange.allreduce(local)


def cuda_slab(cm, nz, rank, world, bc=("periodic", "periodic"), **kw):
    """The library handle of slab `rank` of `world` along z of an nz-plane periodic domain.

    Returns (solver, z0): the solver owns planes z0 .. z0 + nz_local - 1 of the domain.
    """
    z0, nzl = split(nz, world)[rank]
    s = cm.Solver(nz=nzl, bc=(bc[0], bc[1], "halo"), **kw)
    return s, z0
