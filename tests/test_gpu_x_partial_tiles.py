"""x passes on partial row tiles, at the lengths where their rows arrive by bulk copies.

The fused x passes work on tiles of 16 consecutive rows (y + ny z). At x lengths of 256 and more the
density pass stages its psi rows with one bulk copy per row; at 384, 512 and 768 the kick pass stages
the half-spectrum rows of Phi that way too (and its psi rows at every length whose last radix is at
most 8). A grid with ny nz not a multiple of 16 ends in a tile with fewer live rows: only those are
copied, the mbarrier expects only their bytes, and the rows past the end are zeros in shared memory.
Each case here has ny nz = 24 (one full tile and one of 8 rows) and runs gravity and the
self-interaction for several steps in two calls against the FP64 oracle (Sec. 3.1, Algorithm 1).
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

PSI_TOL = 1e-5   # relative L2, as for every other psi parity case


@pytest.fixture(scope="module")
def spe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_25026_gb300 import build
    build.build()
    oracle.build()
    from paper_2606_25026_gb300 import spe as mod
    mod.load_library()
    return mod


@pytest.mark.parametrize("nx", [256, 384, 512, 768])
def test_partial_row_tile_matches_oracle(spe, nx):
    nz, ny = 4, 6
    rng = np.random.default_rng(nx + 7)
    shape = (nz, ny, nx)
    psi = ((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * 0.3 + 1.0).astype(np.complex64)
    L = (1.0, 0.7, 1.3)
    dt = 0.15 * min(L[0] / nx, L[1] / ny, L[2] / nz) ** 2
    g = spe.Grid(nx, ny, nz, L=L, G=0.8, kappa=0.2)
    g.set_ic(psi)
    o = oracle.Oracle(nx, ny, nz, L, G=0.8, kappa=0.2)
    o.set_ic(psi.astype(np.complex128))
    for _ in range(2):
        g.step(3, dt)
        o.step(3, dt)
    got, ref = g.get_psi(), o.get_psi()
    err = float(np.linalg.norm((got - ref).ravel()) / np.linalg.norm(ref.ravel()))
    assert err <= PSI_TOL, (nx, err)
    # the mass after the partial tile's rows: the density pass reduces it over live rows only
    assert abs(g.last_mass() - o.energy()["mass"]) <= 1e-6 * o.energy()["mass"]
