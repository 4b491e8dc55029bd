"""CPU-side checks of the C ABI: the library builds, loads, and exports every entry point that
include/*.h declares; the host-only calls (workspace sizing, status strings) behave.  No call here
launches device work."""
import ctypes
import glob
import os
import re

import pytest

from paper_2606_25026_gb300 import build as spe_build
from paper_2606_25026_gb300 import spe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"^SPE_API\s+[\w\s\*]*?\b(spe_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    path = spe_build.build()
    return spe.load_library(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    # the binding wraps exactly the declared set
    assert set(spe.EXPORTED) == set(names)


def test_workspace_bytes_and_validation(lib):
    cfg = spe.spe_config(256, 256, 256, 1.0, 1.0, 1.0, 1.0, 1.0, 0.0, 1_000_000, 0, None)
    nb = ctypes.c_size_t()
    assert lib.spe_workspace_bytes(ctypes.byref(cfg), ctypes.byref(nb)) == spe.SPE_OK
    n3 = 256 ** 3
    # psi (8 B) + half spectrum (~4 B) + phi (4 B) + fixed-point deposit (8 B) per cell, + particles
    assert nb.value >= n3 * (8 + 4 + 4 + 8) + 7 * 4 * 1_000_000
    assert nb.value < n3 * 26 + 64 * 2 ** 20
    for bad in (dict(nx=100), dict(ny=1), dict(Lx=0.0), dict(hbar_over_m=-1.0), dict(nz=2048)):
        c = spe.spe_config(32, 32, 32, 1.0, 1.0, 1.0, 1.0, 1.0, 0.0, 0, 0, None)
        for k, v in bad.items():
            setattr(c, k, v)
        assert lib.spe_workspace_bytes(ctypes.byref(c), ctypes.byref(nb)) == spe.SPE_EINVAL, bad


def test_supported_sizes_match_header():
    h = open(os.path.join(ROOT, "include", "spe.h")).read()
    m = re.search(r"each in \{([\d,]+)\}", h)
    assert tuple(int(v) for v in m.group(1).split(",")) == spe.SUPPORTED_N


def test_strerror(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert lib.spe_strerror(code)
    assert b"CFL" in lib.spe_strerror(spe.SPE_ECFL)
