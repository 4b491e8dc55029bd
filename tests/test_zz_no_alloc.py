"""spe_field_energy_noalloc: the field-energy reduction for callers that may not allocate.

Callers inside another framework's memory pool, or with a fixed device-memory budget, cannot call
cudaMalloc where they want a diagnostic.  This entry point takes their device field and returns the
same mass and self-interaction energy as spe_energy, with its scratch in a fixed array inside the
library.  The test calls it through the C ABI twice in a row (the shared scratch keeps the previous
call's contents, so the second call checks that nothing stale leaks in) and compares both results
with spe_energy on a grid holding the same field and with an FP64 sum of |psi|^2 and |psi|^4 on
the host, within the energy tolerances of the other GPU tests; a flat field of 300001 values (more
than the 1024 blocks x 256 threads of one sweep, and odd) runs the grid-stride loop.  It lives in
its own file, collected last, so that a run stopping at the first failure has already run every
other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2606_25026_gb300 import inputs

pytestmark = pytest.mark.gpu

MASS_TOL = 1e-6
ENERGY_TOL = 1e-5


@pytest.fixture(scope="module")
def spe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_25026_gb300 import build
    build.build()
    from paper_2606_25026_gb300 import spe as mod
    mod.load_library()
    return mod


def test_noalloc_matches_energy_two_calls(spe):
    import torch
    n, L, kappa = 64, 1.0, 0.7
    psi = inputs.soliton_halo(n, psi_mass=1.0, seed=77).astype(np.complex64)
    g = spe.Grid(n, L=L, G=1.0, kappa=kappa)
    g.set_ic(psi)
    ref = g.energy()
    lib = spe.load_library()
    dv = (L / n) ** 3
    d_psi = torch.from_numpy(psi).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = (ctypes.c_double * 2)()
        st = lib.spe_field_energy_noalloc(ctypes.c_void_p(d_psi.data_ptr()), d_psi.numel(), dv, kappa, out,
                                          spe.SPE_HOST, ctypes.c_void_p(stream))
        assert st == spe.SPE_OK, (call, st)
        assert abs(out[0] - ref["mass"]) <= MASS_TOL * abs(ref["mass"]), (call, out[0], ref["mass"])
        assert abs(out[1] - ref["interaction"]) <= ENERGY_TOL * abs(ref["interaction"]), \
            (call, out[1], ref["interaction"])
    # device-side output, also twice
    d_out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for call in range(2):
        st = lib.spe_field_energy_noalloc(ctypes.c_void_p(d_psi.data_ptr()), d_psi.numel(), dv, kappa,
                                          ctypes.cast(ctypes.c_void_p(d_out.data_ptr()),
                                                      ctypes.POINTER(ctypes.c_double)),
                                          spe.SPE_DEVICE, ctypes.c_void_p(stream))
        assert st == spe.SPE_OK
        got = d_out.cpu().numpy()
        assert abs(got[0] - ref["mass"]) <= MASS_TOL * abs(ref["mass"])
        assert abs(got[1] - ref["interaction"]) <= ENERGY_TOL * abs(ref["interaction"])


def host_sums(psi, dv, kappa):
    """FP64 host reference: (dv sum |psi|^2, kappa / 2 dv sum |psi|^4)."""
    a2 = np.abs(psi.astype(np.complex128).ravel()) ** 2
    return float(a2.sum() * dv), float(0.5 * kappa * (a2 * a2).sum() * dv)


def call_noalloc(spe, lib, d_psi, dv, kappa, stream):
    out = (ctypes.c_double * 2)()
    st = lib.spe_field_energy_noalloc(ctypes.c_void_p(d_psi.data_ptr()), d_psi.numel(), dv, kappa, out,
                                      spe.SPE_HOST, ctypes.c_void_p(stream))
    return st, (out[0], out[1])


def test_noalloc_matches_host_fp64_sum(spe):
    import torch
    n, L, kappa = 64, 1.0, 0.7
    psi = inputs.soliton_halo(n, psi_mass=1.0, seed=77).astype(np.complex64)
    dv = (L / n) ** 3
    ref = host_sums(psi, dv, kappa)
    lib = spe.load_library()
    d_psi = torch.from_numpy(psi).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        st, got = call_noalloc(spe, lib, d_psi, dv, kappa, stream)
        assert st == spe.SPE_OK, (call, st)
        assert abs(got[0] - ref[0]) <= MASS_TOL * abs(ref[0]), (call, got, ref)
        assert abs(got[1] - ref[1]) <= ENERGY_TOL * abs(ref[1]), (call, got, ref)


def test_noalloc_grid_stride_loop_on_a_flat_odd_field(spe):
    """300001 values: more than one sweep of the 1024 x 256 threads, and not a multiple of 256."""
    import torch
    rng = np.random.default_rng(78)
    m = 300001
    psi = (rng.standard_normal(m) + 1j * rng.standard_normal(m)).astype(np.complex64)
    dv, kappa = 1.0 / m, -1.3
    ref = host_sums(psi, dv, kappa)
    lib = spe.load_library()
    d_psi = torch.from_numpy(psi).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        st, got = call_noalloc(spe, lib, d_psi, dv, kappa, stream)
        assert st == spe.SPE_OK, (call, st)
        assert abs(got[0] - ref[0]) <= MASS_TOL * abs(ref[0]), (call, got, ref)
        assert abs(got[1] - ref[1]) <= ENERGY_TOL * abs(ref[1]), (call, got, ref)
    # a 128^3 field, also beyond one sweep, against spe_energy
    n = 128
    psi3 = inputs.soliton_halo(n, psi_mass=1.0, seed=79).astype(np.complex64)
    g = spe.Grid(n, L=1.0, G=1.0, kappa=kappa)
    g.set_ic(psi3)
    e = g.energy()
    g.destroy()
    st, got = call_noalloc(spe, lib, torch.from_numpy(psi3).cuda(), 1.0 / n ** 3, kappa, stream)
    assert st == spe.SPE_OK
    assert abs(got[0] - e["mass"]) <= MASS_TOL * abs(e["mass"])
    assert abs(got[1] - e["interaction"]) <= ENERGY_TOL * abs(e["interaction"])


def test_noalloc_rejects_misaligned_pointers(spe):
    """Checked on the host before any launch: nothing reaches the GPU."""
    lib = spe.load_library()
    out = (ctypes.c_double * 2)()
    assert lib.spe_field_energy_noalloc(ctypes.c_void_p(0x1004), 16, 1.0, 0.0, out, spe.SPE_HOST, None) == \
        spe.SPE_EINVAL
    dev_out = ctypes.cast(ctypes.c_void_p(0x2004), ctypes.POINTER(ctypes.c_double))
    assert lib.spe_field_energy_noalloc(ctypes.c_void_p(0x1000), 16, 1.0, 0.0, dev_out, spe.SPE_DEVICE, None) == \
        spe.SPE_EINVAL


def test_noalloc_rejects_bad_sizes(spe):
    lib = spe.load_library()
    out = (ctypes.c_double * 2)()
    too_many = (1 << 30) + 1
    assert lib.spe_field_energy_noalloc(ctypes.c_void_p(16), too_many, 1.0, 0.0, out, spe.SPE_HOST, None) == \
        spe.SPE_EINVAL
    assert lib.spe_field_energy_noalloc(ctypes.c_void_p(16), 0, 1.0, 0.0, out, spe.SPE_HOST, None) == spe.SPE_EINVAL
