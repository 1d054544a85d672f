"""Thin ctypes binding of libcmlbm.so (argument marshalling only).

Every computation runs in the CUDA library; PyTorch supplies device memory (tensors) and
the stream. Importing this module loads the library and raises if it has not been built:
there is no CPU fallback.
"""
import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcmlbm.so")

OK, ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_UNSUPPORTED, ERR_DIVERGED = 0, -1, -2, -3, -4, -5
D2Q9, D3Q27 = 0, 1
F64, F32, BF16, F16 = 0, 1, 2, 3
PERIODIC, BOUNCEBACK, HALO = 0, 1, 2
DEVICE, HOST = 0, 1
FACE_BOTTOM, FACE_TOP = 0, 1

LATTICES = {"D2Q9": D2Q9, "D3Q27": D3Q27}
STORAGES = {"f64": F64, "f32": F32, "bf16": BF16, "f16": F16}
TORCH_STORAGE = {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16, F16: torch.float16}
BCS = {"periodic": PERIODIC, "bounceback": BOUNCEBACK, "halo": HALO}

# every symbol declared in include/cmlbm.h
SYMBOLS = ["cmlbm_config_default", "cmlbm_create", "cmlbm_destroy", "cmlbm_last_error", "cmlbm_set_stream",
           "cmlbm_set_force", "cmlbm_init", "cmlbm_step", "cmlbm_step_buffers", "cmlbm_moments",
           "cmlbm_moments_of", "cmlbm_reduce", "cmlbm_state_bytes", "cmlbm_get_state", "cmlbm_set_state",
           "cmlbm_adjoint_terminal", "cmlbm_step_adjoint", "cmlbm_launch_count", "cmlbm_reduce_noalloc",
           "cmlbm_turbulence_force", "cmlbm_step_filtered", "cmlbm_halo_bytes", "cmlbm_halo_pack",
           "cmlbm_halo_unpack", "cmlbm_step_kernel", "cmlbm_step_adjoint_segment", "cmlbm_step_split"]
KERNELS = {0: "auto", 1: "direct", 2: "tma", 3: "pair", 4: "pair_two_steps"}


class Config(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("storage", ctypes.c_int),
        ("bc", ctypes.c_int * 3),
        ("wall_velocity", ((ctypes.c_double * 3) * 2) * 3),
        ("tau", ctypes.c_double),
        ("omega_bulk", ctypes.c_double),
        ("omega_3", ctypes.c_double),
        ("omega_4", ctypes.c_double),
        ("smagorinsky_cs", ctypes.c_double),
        ("van_driest_aplus", ctypes.c_double),
        ("van_driest_utau_over_nu", ctypes.c_double),
        ("attractor", ctypes.c_int),
        ("reduced_compressibility", ctypes.c_int),
        ("rho0", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("device", ctypes.c_int),
        ("kernel", ctypes.c_int),
    ]


class CmlbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cmlbm error {code}: {msg}")
        self.code = code


_lib = None


def load():
    """Load libcmlbm.so (raises when it is missing: the product has no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1202_6074_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double), None
    sig = {
        "cmlbm_config_default": (I, [ctypes.POINTER(Config)]),
        "cmlbm_create": (I, [ctypes.POINTER(Config), ctypes.POINTER(P)]),
        "cmlbm_destroy": (V, [P]),
        "cmlbm_last_error": (ctypes.c_char_p, [P]),
        "cmlbm_set_stream": (I, [P, P]),
        "cmlbm_set_force": (I, [P, D, P, I]),
        "cmlbm_init": (I, [P, P, P, I]),
        "cmlbm_step": (I, [P, I]),
        "cmlbm_step_split": (I, [P, I]),
        "cmlbm_step_buffers": (I, [P, P, P]),
        "cmlbm_moments": (I, [P, P, P, I]),
        "cmlbm_moments_of": (I, [P, P, P, P]),
        "cmlbm_reduce": (I, [P, D]),
        "cmlbm_state_bytes": (ctypes.c_size_t, [P]),
        "cmlbm_get_state": (I, [P, P, ctypes.c_size_t, I]),
        "cmlbm_set_state": (I, [P, P, ctypes.c_size_t, I]),
        "cmlbm_adjoint_terminal": (I, [P, P, P, P, P, P]),
        "cmlbm_step_adjoint": (I, [P, P, P, P, P]),
        "cmlbm_step_adjoint_segment": (I, [P, P, P, P, P, P, I]),
        "cmlbm_launch_count": (ctypes.c_longlong, [P]),
        "cmlbm_reduce_noalloc": (I, [ctypes.POINTER(Config), P, D, P, P]),
        "cmlbm_turbulence_force": (I, [P, ctypes.c_double]),
        "cmlbm_step_filtered": (I, [P, I, ctypes.c_double]),
        "cmlbm_halo_bytes": (ctypes.c_size_t, [P]),
        "cmlbm_halo_pack": (I, [P, I, P, I]),
        "cmlbm_halo_unpack": (I, [P, I, P, I]),
        "cmlbm_step_kernel": (I, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    raise TypeError(type(t))


def _as_vec3(v):
    arr = (ctypes.c_double * 3)()
    for d in range(3):
        arr[d] = float(v[d]) if v is not None else 0.0
    return arr


def make_config(lattice="D3Q27", nx=32, ny=32, nz=32, storage="f32", bc=("periodic",) * 3, wall_velocity=None,
                tau=0.8, omega_bulk=0.0, omega_3=1.0, omega_4=1.0, smagorinsky_cs=0.0, van_driest=None,
                attractor="maxwell", reduced_compressibility=False, rho0=1.0, device=0, stream=None, kernel="auto"):
    lib = load()
    c = Config()
    lib.cmlbm_config_default(ctypes.byref(c))
    c.lattice = LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
    c.nx, c.ny, c.nz = int(nx), int(ny), int(nz)
    c.storage = STORAGES[storage] if isinstance(storage, str) else int(storage)
    for a in range(3):
        c.bc[a] = BCS[bc[a]] if isinstance(bc[a], str) else int(bc[a])
    if wall_velocity is not None:
        for a in range(3):
            for s in range(2):
                for d in range(3):
                    c.wall_velocity[a][s][d] = float(wall_velocity[a][s][d])
    c.tau = float(tau)
    c.omega_bulk = float(omega_bulk)
    c.omega_3 = float(omega_3)
    c.omega_4 = float(omega_4)
    c.smagorinsky_cs = float(smagorinsky_cs)
    if van_driest is not None:
        c.van_driest_aplus, c.van_driest_utau_over_nu = float(van_driest[0]), float(van_driest[1])
    c.attractor = {"maxwell": 0, "factorized": 1}[attractor] if isinstance(attractor, str) else int(attractor)
    c.reduced_compressibility = int(bool(reduced_compressibility))
    c.rho0 = float(rho0)
    c.device = int(device)
    c.stream = stream
    c.kernel = ({"auto": 0, "direct": 1, "tma": 2, "pair": 3, "pair_two_steps": 4}[kernel] if isinstance(kernel, str)
                else int(kernel))
    return c


class Solver:
    """One lattice on one GPU (owns a cmlbm handle). Fields are torch tensors.

    Device inputs are CUDA float64 tensors: rho [nz, ny, nx], u and F [3, nz, ny, nx].
    Host inputs (numpy float64 arrays) are copied by the library itself.
    """

    def __init__(self, **kw):
        self.lib = load()
        if "device" not in kw and torch.cuda.is_available():
            kw["device"] = torch.cuda.current_device()
        if kw.get("stream") is None and torch.cuda.is_available():
            kw["stream"] = ctypes.c_void_p(torch.cuda.current_stream(kw.get("device", 0)).cuda_stream)
        self.cfg = make_config(**kw)
        h = ctypes.c_void_p()
        rc = self.lib.cmlbm_create(ctypes.byref(self.cfg), ctypes.byref(h))
        if rc != OK:
            raise CmlbmError(rc, self.lib.cmlbm_last_error(None).decode())
        self.h = h
        self.Q = 27 if self.cfg.lattice == D3Q27 else 9
        self.shape = (self.cfg.nz, self.cfg.ny, self.cfg.nx)
        self.N = self.cfg.nx * self.cfg.ny * self.cfg.nz
        self.slab = self.cfg.bc[2] == HALO
        # a slab's state buffers carry a ghost plane below and above its own planes
        self.state_shape = (self.Q, self.cfg.nz + (2 if self.slab else 0), self.cfg.ny, self.cfg.nx)
        self.device = torch.device("cuda", self.cfg.device)
        self.state_dtype = TORCH_STORAGE[self.cfg.storage]
        self.real_dtype = torch.float64 if self.cfg.storage == F64 else torch.float32

    # ---- plumbing ---------------------------------------------------------------------
    def _check(self, rc):
        if rc != OK:
            raise CmlbmError(rc, self.lib.cmlbm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.cmlbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream=None):
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._check(self.lib.cmlbm_set_stream(self.h, ctypes.c_void_p(s.cuda_stream)))

    @property
    def launch_count(self):
        return int(self.lib.cmlbm_launch_count(self.h))

    @property
    def step_kernel(self):
        """"direct", "pair" or "tma": the step kernel this handle runs."""
        return KERNELS[int(self.lib.cmlbm_step_kernel(self.h))]

    # ---- API --------------------------------------------------------------------------
    def set_force(self, uniform=(0.0, 0.0, 0.0), field=None):
        where = HOST if isinstance(field, np.ndarray) else DEVICE
        if isinstance(field, np.ndarray):
            field = np.ascontiguousarray(field, dtype=np.float64)
        elif field is not None:
            field = field.to(self.device, torch.float64).contiguous()
        self._field_keepalive = field
        self._check(self.lib.cmlbm_set_force(self.h, _as_vec3(uniform), _ptr(field), where))

    def init(self, rho=None, u=None):
        """Equilibrium initial state from FP64 fields: CUDA tensors, or host data (numpy arrays
        or CPU tensors; page-locked CPU tensors are read in place by the init kernel)."""
        def on_host(t):
            return isinstance(t, np.ndarray) or (isinstance(t, torch.Tensor) and t.device.type == "cpu")
        host = on_host(rho) or on_host(u)
        if host:
            def prep(t):
                if t is None:
                    return None
                if isinstance(t, torch.Tensor) and t.dtype == torch.float64 and t.is_contiguous():
                    return t
                return np.ascontiguousarray(t.numpy() if isinstance(t, torch.Tensor) else t, dtype=np.float64)
            rho, u = prep(rho), prep(u)
        else:
            rho = None if rho is None else rho.to(self.device, torch.float64).contiguous()
            u = None if u is None else u.to(self.device, torch.float64).contiguous()
        self._check(self.lib.cmlbm_init(self.h, _ptr(rho), _ptr(u), HOST if host else DEVICE))
        self._init_keepalive = (rho, u)

    def step(self, n=1):
        self._check(self.lib.cmlbm_step(self.h, int(n)))

    def step_split(self, parts=3):
        """One step with the boundary planes on the handle's stream and the interior on the
        library's own (cmlbm_step_split): a face exchange issued next overlaps the interior.
        parts = 1 (boundary) and then 2 (interior) issue the two parts in two calls."""
        self._check(self.lib.cmlbm_step_split(self.h, int(parts)))

    def turbulence_force(self, cs):
        """Set the force field to rho a' from the Smagorinsky closure (filtered equation)."""
        self._check(self.lib.cmlbm_turbulence_force(self.h, float(cs)))

    def step_filtered(self, n, cs):
        self._check(self.lib.cmlbm_step_filtered(self.h, int(n), float(cs)))

    def step_buffers(self, src, dst):
        self._check(self.lib.cmlbm_step_buffers(self.h, _ptr(src), _ptr(dst)))

    def moments(self, state=None, host=False, out=None):
        """(rho [nz,ny,nx], u [3,nz,ny,nx]) as float64; CUDA tensors, or host data when host=True
        (new numpy arrays, or the caller's `out` = (rho, u) float64 host buffers; page-locked CPU
        tensors are written in place by the moments kernel)."""
        if host:
            if out is None:
                rho = np.empty(self.shape)
                u = np.empty((3,) + self.shape)
            else:
                rho, u = out
            self._check(self.lib.cmlbm_moments(self.h, _ptr(rho), _ptr(u), HOST))
            return rho, u
        rho = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        u = torch.empty((3,) + self.shape, dtype=torch.float64, device=self.device)
        if state is None:
            self._check(self.lib.cmlbm_moments(self.h, _ptr(rho), _ptr(u), DEVICE))
        else:
            self._check(self.lib.cmlbm_moments_of(self.h, _ptr(state), _ptr(rho), _ptr(u)))
        return rho, u

    def reduce(self):
        out = (ctypes.c_double * 5)()
        self._check(self.lib.cmlbm_reduce(self.h, out))
        return [out[k] for k in range(5)]

    @property
    def state_bytes(self):
        return int(self.lib.cmlbm_state_bytes(self.h))

    def new_state(self):
        return torch.empty(self.state_shape, dtype=self.state_dtype, device=self.device)

    # ---- slab faces -------------------------------------------------------------------
    def new_face(self, host=False):
        """A face message buffer [9, ny, nx] in the storage type (pinned host memory if host)."""
        shape = (9, self.cfg.ny, self.cfg.nx)
        if host:
            return torch.empty(shape, dtype=self.state_dtype, pin_memory=torch.cuda.is_available())
        return torch.empty(shape, dtype=self.state_dtype, device=self.device)

    def pack(self, face, out=None, host=False):
        """The 9 populations leaving through `face` (FACE_TOP: e_z = +1, FACE_BOTTOM: e_z = -1)."""
        out = self.new_face(host) if out is None else out
        self._check(self.lib.cmlbm_halo_pack(self.h, int(face), _ptr(out), HOST if out.device.type == "cpu" else DEVICE))
        return out

    def unpack(self, face, msg):
        """Write a neighbour's message into the ghost plane on `face` of the current state."""
        if msg.device.type != "cpu":
            msg = msg.to(self.device, self.state_dtype).contiguous()
        else:
            msg = msg.to(self.state_dtype).contiguous()
        self._check(self.lib.cmlbm_halo_unpack(self.h, int(face), _ptr(msg),
                                               HOST if msg.device.type == "cpu" else DEVICE))
        self._face_keepalive = msg

    def get_state(self, out=None):
        out = self.new_state() if out is None else out
        nbytes = out.numel() * out.element_size()
        self._check(self.lib.cmlbm_get_state(self.h, _ptr(out), nbytes, DEVICE))
        return out

    def set_state(self, s):
        s = s.to(self.device, self.state_dtype).contiguous()
        nbytes = s.numel() * s.element_size()
        self._check(self.lib.cmlbm_set_state(self.h, _ptr(s), nbytes, DEVICE))
        torch.cuda.current_stream(self.device).synchronize()

    # ---- adjoint ----------------------------------------------------------------------
    def adjoint_terminal(self, state, dLdu, lam, dLdF, dLdrho=None):
        self._check(self.lib.cmlbm_adjoint_terminal(self.h, _ptr(state), _ptr(dLdu), _ptr(dLdrho), _ptr(lam),
                                                    _ptr(dLdF)))

    def step_adjoint(self, state, lam_in, lam_out, dLdF):
        self._check(self.lib.cmlbm_step_adjoint(self.h, _ptr(state), _ptr(lam_in), _ptr(lam_out), _ptr(dLdF)))

    def step_adjoint_segment(self, state, lam_in, lam_out, seg, dLdF, fold):
        """One step back with the force gradient added into the segment accumulator seg (arithmetic
        type, [3, nz, ny, nx]); with fold, seg is then added into the FP64 dLdF and zeroed."""
        self._check(self.lib.cmlbm_step_adjoint_segment(self.h, _ptr(state), _ptr(lam_in), _ptr(lam_out), _ptr(seg),
                                                        _ptr(dLdF), 1 if fold else 0))


def reduce_noalloc(cfg, state, out, uniform_force=(0.0, 0.0, 0.0), force_field=None):
    """cmlbm_reduce_noalloc: FP64 sums of a state buffer into the device tensor out[5] without
    a handle or any allocation (the call is asynchronous on cfg.stream)."""
    lib = load()
    rc = lib.cmlbm_reduce_noalloc(ctypes.byref(cfg), _ptr(state), _as_vec3(uniform_force), _ptr(force_field),
                                  _ptr(out))
    if rc != OK:
        raise CmlbmError(rc, "cmlbm_reduce_noalloc rejected the call (see include/cmlbm.h)")


def rest_weights(lattice):
    """Rest weights in the library's direction order (products of the 1D weights 1/6, 2/3, 1/6)."""
    w1 = {-1: 1.0 / 6.0, 0: 2.0 / 3.0, 1: 1.0 / 6.0}
    return np.array([w1[ex] * w1[ey] * (w1[ez] if lattice == "D3Q27" else 1.0)
                     for (ex, ey, ez) in velocities(lattice)])


def velocities(lattice):
    if lattice == "D2Q9":
        return [(0, 0, 0), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0), (1, 1, 0), (-1, 1, 0), (-1, -1, 0),
                (1, -1, 0)]
    return [((i % 3) - 1, (i // 3) % 3 - 1, i // 9 - 1) for i in range(27)]
