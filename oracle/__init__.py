"""Plain FP64 CPU oracle of the Schroedinger-Poisson split step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference
legs may import this package.  The product path (``paper_2606_25026_gb300``) never does.

The arithmetic lives in ``spe_oracle.c`` (own recursive FFT, own CIC, the kick-drift-kick
order of Sec. 3.1 Eq. (SPE_solver_KDK) / Algorithm 1 of Meng & Dong 2026).  This module only
compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spe_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (-O3, OpenMP).  Portable flags only (x86 and Arm)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    S = ctypes.c_size_t
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_create.restype = P
    lib.oracle_create.argtypes = [I, I, I, D, D, D, D, D, D]
    lib.oracle_destroy.argtypes = [P]
    lib.oracle_set_psi.argtypes = [P, dp]
    lib.oracle_get_psi.argtypes = [P, dp]
    lib.oracle_set_particles.argtypes = [P, S, dp, dp, dp]
    lib.oracle_get_particles.argtypes = [P, dp, dp]
    lib.oracle_set_phi.argtypes = [P, dp]
    lib.oracle_accel.argtypes = [P, dp]
    lib.oracle_deposit.argtypes = [P, dp]
    lib.oracle_step.argtypes = [P, I, D]
    lib.oracle_potential.argtypes = [P, dp]
    lib.oracle_density.argtypes = [P, dp]
    lib.oracle_energy.argtypes = [P, dp]
    lib.oracle_suggest_dt.restype = D
    lib.oracle_suggest_dt.argtypes = [P, D]
    lib.oracle_fft1.argtypes = [I, dp, I]
    lib.oracle_fft3.argtypes = [I, I, I, dp, I]
    lib.oracle_threads.restype = I
    lib.oracle_set_absorb.argtypes = [P, D, I]
    lib.oracle_set_static_phi.argtypes = [P, ctypes.c_void_p]
    lib.oracle_virial.argtypes = [P, dp]
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def threads() -> int:
    """OpenMP threads the oracle runs with."""
    return int(_load().oracle_threads())


def fft1(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """1D transform, forward (sign=-1) unnormalised, inverse (sign=+1) divided by n."""
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    _load().oracle_fft1(a.size, _dptr(a.view(np.float64)), int(sign))
    return a


def fft3(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """3D transform of a (nz, ny, nx) array (x fastest), conventions as fft1 per axis."""
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    nz, ny, nx = a.shape
    _load().oracle_fft3(nx, ny, nz, _dptr(a.view(np.float64)), int(sign))
    return a


ENERGY_FIELDS = ("mass", "kinetic", "potential", "interaction", "star_kinetic", "total", "max_abs_phi")


class Oracle:
    """FP64 state of one periodic grid: psi (nz, ny, nx) complex128 plus star particles."""

    def __init__(self, nx, ny, nz, L=(1.0, 1.0, 1.0), hbar_over_m=1.0, G=1.0, kappa=0.0):
        if np.isscalar(L):
            L = (float(L),) * 3
        self.shape = (nz, ny, nx)
        self.L = tuple(float(v) for v in L)
        self._lib = _load()
        self._h = self._lib.oracle_create(nx, ny, nz, *self.L, float(hbar_over_m), float(G), float(kappa))
        self.np = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_destroy(h)
            self._h = None

    def set_ic(self, psi: np.ndarray):
        a = np.ascontiguousarray(psi, dtype=np.complex128).reshape(self.shape)
        self._lib.oracle_set_psi(self._h, _dptr(a.view(np.float64)))

    def get_psi(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.complex128)
        self._lib.oracle_get_psi(self._h, _dptr(out.view(np.float64)))
        return out

    def set_particles(self, pos, vel, mass):
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3)
        mass = np.ascontiguousarray(mass, dtype=np.float64).reshape(-1)
        self.np = mass.size
        self._lib.oracle_set_particles(self._h, self.np, _dptr(pos), _dptr(vel), _dptr(mass))

    def get_particles(self):
        pos = np.empty((self.np, 3))
        vel = np.empty((self.np, 3))
        if self.np:
            self._lib.oracle_get_particles(self._h, _dptr(pos), _dptr(vel))
        return pos, vel

    def set_phi(self, phi: np.ndarray):
        a = np.ascontiguousarray(phi, dtype=np.float64).reshape(self.shape)
        self._lib.oracle_set_phi(self._h, _dptr(a))

    def accel(self) -> np.ndarray:
        g = np.empty((self.np, 3))
        if self.np:
            self._lib.oracle_accel(self._h, _dptr(g))
        return g

    def deposit(self) -> np.ndarray:
        out = np.empty(self.shape)
        self._lib.oracle_deposit(self._h, _dptr(out))
        return out

    def step(self, nsteps: int, dt: float):
        self._lib.oracle_step(self._h, int(nsteps), float(dt))

    def potential(self) -> np.ndarray:
        out = np.empty(self.shape)
        self._lib.oracle_potential(self._h, _dptr(out))
        return out

    def density(self) -> np.ndarray:
        out = np.empty(self.shape)
        self._lib.oracle_density(self._h, _dptr(out))
        return out

    def energy(self) -> dict:
        out = np.empty(7)
        self._lib.oracle_energy(self._h, _dptr(out))
        return dict(zip(ENERGY_FIELDS, out.tolist()))

    def set_absorb(self, alpha: float, nb: int):
        """Absorbing layer of Sec. 3.1 after every step (alpha = 0 switches it off)."""
        self._lib.oracle_set_absorb(self._h, float(alpha), int(nb))

    def set_static_phi(self, phi_b):
        """Static external potential added to Phi_total (None removes it)."""
        if phi_b is None:
            self._lib.oracle_set_static_phi(self._h, None)
        else:
            a = np.ascontiguousarray(phi_b, dtype=np.float64).reshape(self.shape)
            self._lib.oracle_set_static_phi(self._h, a.ctypes.data)

    def virial(self) -> dict:
        """The paper's overall energy terms K, Q, V (Sec. 3.6), their sum and 2K + 2Q + V."""
        out = np.empty(5)
        self._lib.oracle_virial(self._h, _dptr(out))
        return dict(zip(("K", "Q", "V", "E", "virial"), out.tolist()))

    def suggest_dt(self, safety: float = 0.9) -> float:
        return float(self._lib.oracle_suggest_dt(self._h, float(safety)))
