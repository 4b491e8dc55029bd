"""spe_field_energy_noalloc: the field-energy reduction for callers that may not allocate.

Callers inside another framework's memory pool, or with a fixed device-memory budget, cannot call
cudaMalloc where they want a diagnostic.  This entry point takes their device field and returns the
same mass and self-interaction energy as spe_energy, with its scratch in a fixed array inside the
library.  The test calls it through the C ABI twice in a row (the shared scratch keeps the previous
call's contents, so the second call checks that nothing stale leaks in) and compares both results
with spe_energy on a grid holding the same field, within the energy tolerances of the other GPU
tests.  It lives in its own file, collected last, so that a run stopping at the first failure has
already run every other test.
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


def test_noalloc_rejects_bad_sizes(spe):
    lib = spe.load_library()
    out = (ctypes.c_double * 2)()
    too_many = (1 << 30) + 1
    assert lib.spe_field_energy_noalloc(ctypes.c_void_p(16), too_many, 1.0, 0.0, out, spe.SPE_HOST, None) == \
        spe.SPE_EINVAL
    assert lib.spe_field_energy_noalloc(ctypes.c_void_p(16), 0, 1.0, 0.0, out, spe.SPE_HOST, None) == spe.SPE_EINVAL
