"""Thin ctypes binding over the libspe C ABI (include/spe.h).

Argument marshalling only: every step of the solver runs in libspe's CUDA kernels.  PyTorch
supplies device memory (the grid's workspace is a torch uint8 tensor) and the CUDA stream.
There is no fallback: if libspe.so is missing or no GPU is present, creating a grid raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspe.so")

# status codes and flags (mirror include/spe.h)
SPE_OK, SPE_EINVAL, SPE_ENOMEM, SPE_ECUDA, SPE_ECFL, SPE_ENONFINITE, SPE_ETIMEOUT, SPE_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
SPE_HOST, SPE_DEVICE = 0, 1
SPE_GRAVITY_OFF = 1 << 0
SPE_NO_CFL_CHECK = 1 << 1
SPE_ASYNC = 1 << 2
SPE_PROFILE = 1 << 3
SPE_NO_GRAPH = 1 << 4
SPE_STATIC_POTENTIAL = 1 << 5
SPE_PREC_SPLIT16 = 1 << 6
SPE_NO_TMA = 1 << 7

SUPPORTED_N = (4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024)

# every entry point include/spe.h declares
EXPORTED = (
    "spe_workspace_bytes", "spe_create_grid", "spe_destroy", "spe_set_ic", "spe_add_particles",
    "spe_clear_particles", "spe_step", "spe_suggest_dt", "spe_density", "spe_potential", "spe_energy",
    "spe_last_mass", "spe_mass_async", "spe_get_psi", "spe_get_particles", "spe_particle_count", "spe_sync", "spe_settle",
    "spe_launch_count", "spe_profile_read", "spe_strerror", "spe_field_energy_noalloc",
    "spe_set_static_potential", "spe_virial", "spe_autotune", "spe_set_schedule", "spe_get_schedule",
    "spe_get_schedule_half",
    "spe_batch_create", "spe_batch_grid",
    "spe_batch_autotune", "spe_batch_step", "spe_batch_settle", "spe_batch_launch_count", "spe_batch_destroy",
    "spe_batch_set_persistent", "spe_batch_get_persistent", "spe_pair_norms",
    # include/spe_fno.h
    "spe_fno_param_count", "spe_fno_create", "spe_fno_destroy", "spe_fno_set_params", "spe_fno_get_params",
    "spe_fno_get_grads", "spe_fno_forward", "spe_fno_backward", "spe_fno_adam", "spe_fno_sync",
    "spe_fno_profile_read", "spe_fno_launch_count",
    "spe_surrogate_create", "spe_surrogate_destroy", "spe_surrogate_advance", "spe_surrogate_launch_count",
)

# include/spe_fno.h
SPE_FNO_WIDTH, SPE_FNO_HIDDEN = 32, 64
SPE_FNO_TRAIN = 1 << 0
SPE_FNO_ACT_FP32 = 1 << 1
SPE_FNO_NO_GRAPH = 1 << 2
SPE_FNO_PROFILE = 1 << 3


class SpeError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: {strerror(status)} (status {status})")
        self.status = status


class spe_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
        ("hbar_over_m", ctypes.c_double), ("G", ctypes.c_double), ("kappa", ctypes.c_double),
        ("max_particles", ctypes.c_size_t), ("flags", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
        ("absorb_alpha", ctypes.c_double), ("absorb_nb", ctypes.c_int),
    ]


class spe_virial_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("K", "Q", "V", "E", "virial")]


class spe_energy_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("mass", "kinetic", "potential", "interaction", "star_kinetic", "total", "max_abs_phi")]


class spe_fno_config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("layers", ctypes.c_int), ("modes", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("flags", ctypes.c_int), ("inv_A", ctypes.c_double),
                ("sigma", ctypes.c_double), ("cuda_stream", ctypes.c_void_p)]


class spe_judge_config(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("max_mass_drift", "max_energy_drift", "max_rel_l2")]


class spe_judge_result(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_int), ("spot_checked", ctypes.c_int), ("used_proposal", ctypes.c_int),
                ("mass_drift", ctypes.c_double), ("energy_drift", ctypes.c_double), ("rel_l2", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libspe.so (built by __graft_entry__.build() / paper_2606_25026_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libspe.so not built at {path}; run paper_2606_25026_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, S, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_double
    fp = ctypes.c_void_p
    sig = {
        "spe_workspace_bytes": (I, [ctypes.POINTER(spe_config), ctypes.POINTER(S)]),
        "spe_create_grid": (I, [ctypes.POINTER(spe_config), P, S, ctypes.POINTER(P)]),
        "spe_destroy": (I, [P]),
        "spe_set_ic": (I, [P, P, S, I]),
        "spe_add_particles": (I, [P, S, fp, fp, fp, I]),
        "spe_clear_particles": (I, [P]),
        "spe_step": (I, [P, I, D]),
        "spe_suggest_dt": (I, [P, D, ctypes.POINTER(D)]),
        "spe_density": (I, [P, fp, I]),
        "spe_potential": (I, [P, fp, I]),
        "spe_energy": (I, [P, ctypes.POINTER(spe_energy_t)]),
        "spe_last_mass": (I, [P, ctypes.POINTER(D)]),
        "spe_mass_async": (I, [P, P]),
        "spe_get_psi": (I, [P, P, I]),
        "spe_get_particles": (I, [P, fp, fp, I]),
        "spe_particle_count": (I, [P, ctypes.POINTER(S)]),
        "spe_sync": (I, [P]),
        "spe_settle": (I, [P]),
        "spe_launch_count": (I, [P, ctypes.POINTER(ctypes.c_ulonglong), I]),
        "spe_profile_read": (I, [P, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_ulonglong),
                                 ctypes.POINTER(D), I]),
        "spe_strerror": (ctypes.c_char_p, [I]),
        "spe_field_energy_noalloc": (I, [P, S, D, D, ctypes.POINTER(D), I, P]),
        "spe_set_static_potential": (I, [P, fp, I]),
        "spe_virial": (I, [P, ctypes.POINTER(spe_virial_t)]),
        "spe_autotune": (I, [P, ctypes.POINTER(I)]),
        "spe_set_schedule": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "spe_get_schedule": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "spe_get_schedule_half": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "spe_batch_create": (I, [ctypes.POINTER(spe_config), I, ctypes.POINTER(P)]),
        "spe_batch_grid": (I, [P, I, ctypes.POINTER(P)]),
        "spe_batch_autotune": (I, [P]),
        "spe_batch_step": (I, [P, I, ctypes.POINTER(D)]),
        "spe_batch_settle": (I, [P]),
        "spe_batch_launch_count": (I, [P, ctypes.POINTER(ctypes.c_ulonglong)]),
        "spe_batch_set_persistent": (I, [P, I, ctypes.c_longlong]),
        "spe_pair_norms": (I, [P, P, S, I, P, P]),
        "spe_batch_get_persistent": (I, [P, ctypes.POINTER(I)]),
        "spe_batch_destroy": (I, [P]),
        "spe_fno_param_count": (I, [ctypes.POINTER(spe_fno_config), ctypes.POINTER(S)]),
        "spe_fno_create": (I, [ctypes.POINTER(spe_fno_config), ctypes.POINTER(P)]),
        "spe_fno_destroy": (I, [P]),
        "spe_fno_set_params": (I, [P, fp, S, I]),
        "spe_fno_get_params": (I, [P, fp, S, I]),
        "spe_fno_get_grads": (I, [P, fp, S, I]),
        "spe_fno_forward": (I, [P, P, P, P, I]),
        "spe_fno_backward": (I, [P, P, ctypes.POINTER(D)]),
        "spe_fno_adam": (I, [P, D, D, D, D]),
        "spe_fno_sync": (I, [P]),
        "spe_fno_profile_read": (I, [P, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_ulonglong),
                                     ctypes.POINTER(D), I]),
        "spe_fno_launch_count": (I, [P, ctypes.POINTER(ctypes.c_ulonglong), I]),
        "spe_surrogate_create": (I, [ctypes.POINTER(spe_config), P, ctypes.POINTER(spe_judge_config),
                                     ctypes.POINTER(P)]),
        "spe_surrogate_destroy": (I, [P]),
        "spe_surrogate_advance": (I, [P, P, I, D, I, ctypes.POINTER(spe_judge_result)]),
        "spe_surrogate_launch_count": (I, [P, ctypes.POINTER(ctypes.c_ulonglong), I]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def strerror(status: int) -> str:
    try:
        return load_library().spe_strerror(int(status)).decode()
    except ImportError:
        return f"status {status}"


def _check(status, what):
    if status != SPE_OK:
        raise SpeError(status, what)


def _ptr_where(a):
    """(pointer, where, keepalive) for a numpy array or a torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return a.data_ptr(), (SPE_DEVICE if a.is_cuda else SPE_HOST), a
    except ImportError:
        pass
    a = np.ascontiguousarray(a)
    return a.ctypes.data, SPE_HOST, a


class Grid:
    """One periodic grid on the current CUDA device.  Methods map one to one onto the C ABI:
    create_grid (the constructor), set_ic, add_particles, clear_particles, step, suggest_dt,
    density, potential, energy, last_mass, get_psi, get_particles, particle_count, sync,
    launch_count, profile_read, destroy."""

    def __init__(self, nx, ny=None, nz=None, L=1.0, hbar_over_m=1.0, G=1.0, kappa=0.0, max_particles=0,
                 flags=0, stream=None, device=None, absorb_alpha=0.0, absorb_nb=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libspe needs a CUDA device; there is no CPU fallback")
        self._lib = load_library()
        ny = nx if ny is None else ny
        nz = nx if nz is None else nz
        if np.isscalar(L):
            L = (float(L),) * 3
        self.shape = (nz, ny, nx)
        self.ncells = nx * ny * nz
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.cfg = spe_config(nx, ny, nz, *(float(v) for v in L), float(hbar_over_m), float(G), float(kappa),
                              int(max_particles), int(flags), ctypes.c_void_p(self.stream.cuda_stream),
                              float(absorb_alpha), int(absorb_nb))
        nbytes = ctypes.c_size_t()
        _check(self._lib.spe_workspace_bytes(ctypes.byref(self.cfg), ctypes.byref(nbytes)), "spe_workspace_bytes")
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        _check(self._lib.spe_create_grid(ctypes.byref(self.cfg), ctypes.c_void_p(self.workspace.data_ptr()),
                                         nbytes.value, ctypes.byref(h)), "spe_create_grid")
        self._h = h

    # -- lifetime
    def destroy(self):
        if getattr(self, "_batch_member", False):
            self._h = None      # the batch owns its members
            return
        if getattr(self, "_h", None):
            self._lib.spe_destroy(self._h)
            self._h = None
            self.workspace = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    # -- state in
    def set_ic(self, psi):
        """psi: complex64 (nz, ny, nx) numpy array (host) or torch tensor (host or device)."""
        import torch
        if isinstance(psi, torch.Tensor):
            if psi.dtype != torch.complex64:
                raise TypeError("psi must be complex64")
            ptr, where, keep = _ptr_where(psi.contiguous())
        else:
            ptr, where, keep = _ptr_where(np.ascontiguousarray(psi, dtype=np.complex64))
        _check(self._lib.spe_set_ic(self._h, ctypes.c_void_p(ptr), self.ncells, where), "spe_set_ic")

    def add_particles(self, pos, vel, mass):
        import torch
        if isinstance(pos, torch.Tensor):
            pos, vel, mass = (t.contiguous().float() for t in (pos, vel, mass))
        else:
            pos = np.ascontiguousarray(pos, dtype=np.float32).reshape(-1, 3)
            vel = np.ascontiguousarray(vel, dtype=np.float32).reshape(-1, 3)
            mass = np.ascontiguousarray(mass, dtype=np.float32).reshape(-1)
        n = int(mass.shape[0])
        pp, where, k1 = _ptr_where(pos)
        vp, w2, k2 = _ptr_where(vel)
        mp, w3, k3 = _ptr_where(mass)
        if not (where == w2 == w3):
            raise ValueError("pos, vel and mass must live in the same memory")
        _check(self._lib.spe_add_particles(self._h, n, ctypes.c_void_p(pp), ctypes.c_void_p(vp),
                                           ctypes.c_void_p(mp), where), "spe_add_particles")

    def clear_particles(self):
        _check(self._lib.spe_clear_particles(self._h), "spe_clear_particles")

    # -- stepping
    def step(self, nsteps, dt):
        _check(self._lib.spe_step(self._h, int(nsteps), float(dt)), "spe_step")

    def suggest_dt(self, safety=0.9):
        out = ctypes.c_double()
        _check(self._lib.spe_suggest_dt(self._h, float(safety), ctypes.byref(out)), "spe_suggest_dt")
        return out.value

    def sync(self):
        _check(self._lib.spe_sync(self._h), "spe_sync")

    def settle(self):
        """Queue the closing half kick the last step() deferred (no wait)."""
        _check(self._lib.spe_settle(self._h), "spe_settle")

    # -- state out
    def _field_out(self, fn, what, out, dtype_np, dtype_t):
        import torch
        if out is None:
            out = np.empty(self.shape, dtype=dtype_np)
        if isinstance(out, torch.Tensor):
            if out.dtype != dtype_t or not out.is_contiguous() or out.numel() != self.ncells:
                raise ValueError(f"{what}: output tensor must be contiguous {dtype_t} of {self.ncells} elements")
        ptr, where, keep = _ptr_where(out)
        _check(fn(self._h, ctypes.c_void_p(ptr), where), what)
        return out

    def get_psi(self, out=None):
        import torch
        return self._field_out(self._lib.spe_get_psi, "spe_get_psi", out, np.complex64, torch.complex64)

    def density(self, out=None):
        import torch
        return self._field_out(self._lib.spe_density, "spe_density", out, np.float32, torch.float32)

    def potential(self, out=None):
        import torch
        return self._field_out(self._lib.spe_potential, "spe_potential", out, np.float32, torch.float32)

    def energy(self) -> dict:
        e = spe_energy_t()
        _check(self._lib.spe_energy(self._h, ctypes.byref(e)), "spe_energy")
        return {n: getattr(e, n) for n, _ in spe_energy_t._fields_}

    def set_static_potential(self, phi_b):
        """Static external potential (nz, ny, nx) float32, numpy or torch; None removes it."""
        if phi_b is None:
            _check(self._lib.spe_set_static_potential(self._h, None, SPE_HOST), "spe_set_static_potential")
            return
        import torch
        if not isinstance(phi_b, torch.Tensor):
            phi_b = np.ascontiguousarray(phi_b, dtype=np.float32)
        ptr, where, keep = _ptr_where(phi_b)
        _check(self._lib.spe_set_static_potential(self._h, ctypes.c_void_p(ptr), where), "spe_set_static_potential")

    def autotune(self):
        """Pick the strided passes' tile widths and radix schedules by timing (see spe_autotune);
        returns the (y, z) widths."""
        out = (ctypes.c_int * 2)()
        _check(self._lib.spe_autotune(self._h, out), "spe_autotune")
        return out[0], out[1]

    def set_schedule(self, tiles=(0, 0), plans=(0, 0)):
        """Pin the y and z passes' tile widths (0 = default) and radix schedules (0/1)."""
        t = (ctypes.c_int * 2)(*[int(v) for v in tiles])
        p = (ctypes.c_int * 2)(*[int(v) for v in plans])
        _check(self._lib.spe_set_schedule(self._h, t, p), "spe_set_schedule")

    def schedule(self):
        """((y tile, z tile), (y plan, z plan)) in use."""
        t = (ctypes.c_int * 2)()
        p = (ctypes.c_int * 2)()
        _check(self._lib.spe_get_schedule(self._h, t, p), "spe_get_schedule")
        return (t[0], t[1]), (p[0], p[1])

    def schedule_half(self):
        """((y tile, z tile), (y plan, z plan)) of the half spectrum's passes (rho, Poisson, Phi)."""
        t = (ctypes.c_int * 2)()
        p = (ctypes.c_int * 2)()
        _check(self._lib.spe_get_schedule_half(self._h, t, p), "spe_get_schedule_half")
        return (t[0], t[1]), (p[0], p[1])

    def virial(self) -> dict:
        v = spe_virial_t()
        _check(self._lib.spe_virial(self._h, ctypes.byref(v)), "spe_virial")
        return {n: getattr(v, n) for n, _ in spe_virial_t._fields_}

    def last_mass(self) -> float:
        out = ctypes.c_double()
        _check(self._lib.spe_last_mass(self._h, ctypes.byref(out)), "spe_last_mass")
        return out.value

    def mass_async(self, dst):
        """Queue a copy of the last step's mass into dst (a float64 tensor element: pinned host or
        CUDA memory) on the grid's stream; no wait."""
        import torch
        if not isinstance(dst, torch.Tensor) or dst.dtype != torch.float64 or dst.numel() < 1:
            raise ValueError("mass_async needs a float64 tensor")
        if not dst.is_cuda and not dst.is_pinned():
            raise ValueError("mass_async needs pinned host or device memory")
        _check(self._lib.spe_mass_async(self._h, ctypes.c_void_p(dst.data_ptr())), "spe_mass_async")

    def particle_count(self) -> int:
        out = ctypes.c_size_t()
        _check(self._lib.spe_particle_count(self._h, ctypes.byref(out)), "spe_particle_count")
        return out.value

    def get_particles(self):
        n = self.particle_count()
        pos = np.empty((n, 3), np.float32)
        vel = np.empty((n, 3), np.float32)
        if n:
            _check(self._lib.spe_get_particles(self._h, pos.ctypes.data, vel.ctypes.data, SPE_HOST),
                   "spe_get_particles")
        return pos, vel

    # -- accounting
    def launch_count(self, reset=False) -> int:
        out = ctypes.c_ulonglong()
        _check(self._lib.spe_launch_count(self._h, ctypes.byref(out), int(bool(reset))), "spe_launch_count")
        return out.value

    def profile_read(self) -> dict:
        cap = 32
        names = (ctypes.c_char_p * cap)()
        launches = (ctypes.c_ulonglong * cap)()
        ms = (ctypes.c_double * cap)()
        k = self._lib.spe_profile_read(self._h, names, launches, ms, cap)
        if k < 0:
            raise SpeError(k, "spe_profile_read")
        return {names[i].decode(): (launches[i], ms[i]) for i in range(k)}


def create_grid(*args, **kwargs) -> Grid:
    return Grid(*args, **kwargs)


def pair_norms(a, b, stream=None):
    """Per-sample (sum |a - b|^2, sum |b|^2) of two (S, ...) complex64 CUDA tensors, through
    spe_pair_norms (FP64, fixed order); returns two numpy arrays of length S."""
    import torch
    lib = load_library()
    for t in (a, b):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex64 and t.is_contiguous()):
            raise TypeError("a and b must be contiguous complex64 CUDA tensors")
    if a.shape != b.shape:
        raise ValueError("a and b differ in shape")
    S = a.shape[0]
    out = torch.empty((S, 2), dtype=torch.float64, device=a.device)
    st = (stream or torch.cuda.current_stream(a.device)).cuda_stream
    _check(lib.spe_pair_norms(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), a[0].numel(), S,
                              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st)), "spe_pair_norms")
    h = out.cpu().numpy()
    return h[:, 0].copy(), h[:, 1].copy()


def field_energy_noalloc(psi, cell_volume, kappa=0.0, stream=None):
    """(mass, interaction) of a complex64 CUDA tensor through spe_field_energy_noalloc: the
    library allocates nothing for it (its scratch is a fixed array inside libspe)."""
    import torch
    lib = load_library()
    if not (isinstance(psi, torch.Tensor) and psi.is_cuda and psi.dtype == torch.complex64 and psi.is_contiguous()):
        raise TypeError("psi must be a contiguous complex64 CUDA tensor")
    out = (ctypes.c_double * 2)()
    st = (stream or torch.cuda.current_stream(psi.device)).cuda_stream
    _check(lib.spe_field_energy_noalloc(ctypes.c_void_p(psi.data_ptr()), psi.numel(), float(cell_volume),
                                        float(kappa), out, SPE_HOST, ctypes.c_void_p(st)),
           "spe_field_energy_noalloc")
    return out[0], out[1]


class Batch:
    """Independent grids stepped together (spe_batch_*).  ``configs``: list of dicts with the
    Grid keyword arguments nx, ny, nz, L, hbar_over_m, G, kappa, max_particles, flags,
    absorb_alpha, absorb_nb.  ``members[i]`` behaves like a Grid (set_ic, add_particles, get_psi,
    energy, ...) but belongs to the batch."""

    def __init__(self, configs, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libspe needs a CUDA device; there is no CPU fallback")
        self._lib = load_library()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        n = len(configs)
        arr = (spe_config * n)()
        shapes = []
        for i, c in enumerate(configs):
            nx = c["nx"]
            ny = c.get("ny", nx)
            nz = c.get("nz", nx)
            L = c.get("L", 1.0)
            if np.isscalar(L):
                L = (float(L),) * 3
            arr[i] = spe_config(nx, ny, nz, *(float(v) for v in L), float(c.get("hbar_over_m", 1.0)),
                                float(c.get("G", 1.0)), float(c.get("kappa", 0.0)), int(c.get("max_particles", 0)),
                                int(c.get("flags", 0)), ctypes.c_void_p(self.stream.cuda_stream),
                                float(c.get("absorb_alpha", 0.0)), int(c.get("absorb_nb", 0)))
            shapes.append((nz, ny, nx))
        h = ctypes.c_void_p()
        _check(self._lib.spe_batch_create(arr, n, ctypes.byref(h)), "spe_batch_create")
        self._h = h
        self.members = []
        for i in range(n):
            gh = ctypes.c_void_p()
            _check(self._lib.spe_batch_grid(self._h, i, ctypes.byref(gh)), "spe_batch_grid")
            m = Grid.__new__(Grid)
            m._lib, m._h, m._batch_member = self._lib, gh, True
            m.shape = shapes[i]
            m.ncells = shapes[i][0] * shapes[i][1] * shapes[i][2]
            m.workspace = None
            m.stream = self.stream
            self.members.append(m)

    def autotune(self):
        _check(self._lib.spe_batch_autotune(self._h), "spe_batch_autotune")

    def step(self, nsteps, dts):
        d = (ctypes.c_double * len(self.members))(*[float(v) for v in dts])
        _check(self._lib.spe_batch_step(self._h, int(nsteps), d), "spe_batch_step")

    def settle(self):
        """Queue every member's deferred closing half kick on the batch stream (no wait)."""
        _check(self._lib.spe_batch_settle(self._h), "spe_batch_settle")

    def launch_count(self) -> int:
        out = ctypes.c_ulonglong()
        _check(self._lib.spe_batch_launch_count(self._h, ctypes.byref(out)), "spe_batch_launch_count")
        return out.value

    def set_persistent(self, on=True, wait_limit=-1):
        """One persistent launch per step (on) or the graph of per-member branches (off);
        wait_limit: polls of a grid-wide barrier before it gives up (-1 = default)."""
        _check(self._lib.spe_batch_set_persistent(self._h, int(bool(on)), int(wait_limit)),
               "spe_batch_set_persistent")

    def persistent(self) -> bool:
        """True when the next step runs as one persistent launch."""
        out = ctypes.c_int()
        _check(self._lib.spe_batch_get_persistent(self._h, ctypes.byref(out)), "spe_batch_get_persistent")
        return bool(out.value)

    def step_status(self, nsteps, dts) -> int:
        """spe_batch_step's status code, without raising."""
        d = (ctypes.c_double * len(self.members))(*[float(v) for v in dts])
        return int(self._lib.spe_batch_step(self._h, int(nsteps), d))

    def destroy(self):
        if getattr(self, "_h", None):
            for m in self.members:
                m._h = None
            self._lib.spe_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass



class Fno:
    """The FNO surrogate network (include/spe_fno.h) on the current CUDA device: create, set/get
    the flat parameter vector, forward, backward, Adam.  Fields are complex64 torch tensors on the
    device, shaped (batch, n, n, n) or (n, n, n)."""

    def __init__(self, n=64, layers=4, modes=16, max_batch=1, train=False, act_fp32=False, inv_A=1.0,
                 sigma=1.0, stream=None, graph=True, profile=False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libspe needs a CUDA device; there is no CPU fallback")
        self._lib = load_library()
        self.n, self.layers, self.modes, self.max_batch = int(n), int(layers), int(modes), int(max_batch)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        flags = ((SPE_FNO_TRAIN if train else 0) | (SPE_FNO_ACT_FP32 if act_fp32 else 0)
                 | (0 if graph else SPE_FNO_NO_GRAPH) | (SPE_FNO_PROFILE if profile else 0))
        self.cfg = spe_fno_config(self.n, self.layers, self.modes, self.max_batch, flags, float(inv_A),
                                  float(sigma), ctypes.c_void_p(self.stream.cuda_stream))
        cnt = ctypes.c_size_t()
        _check(self._lib.spe_fno_param_count(ctypes.byref(self.cfg), ctypes.byref(cnt)), "spe_fno_param_count")
        self.param_count = cnt.value
        h = ctypes.c_void_p()
        _check(self._lib.spe_fno_create(ctypes.byref(self.cfg), ctypes.byref(h)), "spe_fno_create")
        self._h = h
        self._keep = None

    def destroy(self):
        if getattr(self, "_h", None):
            self._lib.spe_fno_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def set_params(self, params):
        import torch
        if isinstance(params, torch.Tensor):
            params = params.contiguous().float()
            ptr, where, keep = _ptr_where(params)
        else:
            ptr, where, keep = _ptr_where(np.ascontiguousarray(params, dtype=np.float32))
        _check(self._lib.spe_fno_set_params(self._h, ctypes.c_void_p(ptr), self.param_count, where),
               "spe_fno_set_params")
        if where == SPE_DEVICE:
            self.stream.synchronize()

    def _vec_out(self, fn, what):
        out = np.empty(self.param_count, dtype=np.float32)
        _check(fn(self._h, ctypes.c_void_p(out.ctypes.data), self.param_count, SPE_HOST), what)
        return out

    def get_params(self) -> np.ndarray:
        return self._vec_out(self._lib.spe_fno_get_params, "spe_fno_get_params")

    def grads(self) -> np.ndarray:
        return self._vec_out(self._lib.spe_fno_get_grads, "spe_fno_get_grads")

    @staticmethod
    def _dev(t, what):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex64 and t.is_contiguous()):
            raise TypeError(f"{what} must be a contiguous complex64 CUDA tensor")
        return t

    def forward(self, psi, psi_b, out=None):
        """Proposal for (psi, psi_b); in training mode keeps the activations for backward()."""
        import torch
        psi, psi_b = self._dev(psi, "psi"), self._dev(psi_b, "psi_b")
        batch = psi.shape[0] if psi.dim() == 4 else 1
        if out is None:
            out = torch.empty_like(psi_b)
        self._dev(out, "out")
        _check(self._lib.spe_fno_forward(self._h, ctypes.c_void_p(psi.data_ptr()),
                                          ctypes.c_void_p(psi_b.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                          int(batch)), "spe_fno_forward")
        self._keep = (psi, psi_b, out)
        return out

    def backward(self, target, want_loss=True):
        target = self._dev(target, "target")
        loss = ctypes.c_double()
        _check(self._lib.spe_fno_backward(self._h, ctypes.c_void_p(target.data_ptr()),
                                           ctypes.byref(loss) if want_loss else None), "spe_fno_backward")
        return loss.value if want_loss else None

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(self._lib.spe_fno_adam(self._h, float(lr), float(beta1), float(beta2), float(eps)), "spe_fno_adam")

    def sync(self):
        _check(self._lib.spe_fno_sync(self._h), "spe_fno_sync")

    def profile_read(self) -> dict:
        """{kernel kind: (launches, summed CUDA-event ms)} since the last read (profile mode)."""
        cap = 32
        names = (ctypes.c_char_p * cap)()
        launches = (ctypes.c_ulonglong * cap)()
        ms = (ctypes.c_double * cap)()
        n = self._lib.spe_fno_profile_read(self._h, names, launches, ms, cap)
        if n < 0:
            _check(n, "spe_fno_profile_read")
        return {names[i].decode(): (launches[i], ms[i]) for i in range(min(n, cap)) if launches[i]}

    def launch_count(self, reset=False) -> int:
        out = ctypes.c_ulonglong()
        _check(self._lib.spe_fno_launch_count(self._h, ctypes.byref(out), int(bool(reset))), "spe_fno_launch_count")
        return out.value


class Surrogate:
    """The judge (include/spe_fno.h): advance(grid, K, dt) moves the grid K steps by the network's
    proposal when the mass and energy drifts pass, by the solver otherwise; spot_check=True runs
    the solver as well and measures the proposal's relative L2 error."""

    def __init__(self, grid: Grid, fno: Fno, max_mass_drift=1e-4, max_energy_drift=1e-3, max_rel_l2=1e-3):
        self._lib = load_library()
        self.fno = fno
        self.jc = spe_judge_config(float(max_mass_drift), float(max_energy_drift), float(max_rel_l2))
        h = ctypes.c_void_p()
        _check(self._lib.spe_surrogate_create(ctypes.byref(grid.cfg), fno._h, ctypes.byref(self.jc),
                                              ctypes.byref(h)), "spe_surrogate_create")
        self._h = h

    def destroy(self):
        if getattr(self, "_h", None):
            self._lib.spe_surrogate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def launch_count(self, reset=False) -> int:
        out = ctypes.c_ulonglong()
        _check(self._lib.spe_surrogate_launch_count(self._h, ctypes.byref(out), int(bool(reset))),
               "spe_surrogate_launch_count")
        return out.value

    def advance(self, grid: Grid, K: int, dt: float, spot_check=False) -> dict:
        r = spe_judge_result()
        _check(self._lib.spe_surrogate_advance(self._h, grid._h, int(K), float(dt), int(bool(spot_check)),
                                               ctypes.byref(r)), "spe_surrogate_advance")
        return {k: getattr(r, k) for k, _ in spe_judge_result._fields_}
