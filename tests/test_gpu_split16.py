"""Split-FP16 tensor-core DFT stages (SPE_PREC_SPLIT16) against the FP64 oracle and the FP32 path.

Axes of 256 or 512 points run every radix-16 stage as a tcgen05 GEMM with hi + lo fp16 operands and
FP32 accumulation; the other axes stay FP32.  Each stage keeps ~2^-22 relative accuracy (the lo x lo
product is dropped), so a few steps stay within the FP32 parity bar of 1e-5 rel-L2."""
import numpy as np
import pytest

import oracle
from paper_2606_25026_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("shape", [(8, 8, 256), (8, 256, 8), (256, 8, 8), (8, 8, 512), (512, 8, 8), (8, 512, 8)])
def test_split16_axes_match_oracle(spe, shape):
    nz, ny, nx = shape
    rng = np.random.default_rng(sum(shape))
    psi = ((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * 0.3 + 1.0).astype(np.complex64)
    L = (1.0, 0.8, 1.2)
    dx = min(L[0] / nx, L[1] / ny, L[2] / nz)
    dt = 0.15 * dx * dx
    res = {}
    for flags in (0, spe.SPE_PREC_SPLIT16):
        g = spe.Grid(nx, ny, nz, L=L, G=0.8, kappa=0.2, flags=flags)
        g.set_ic(psi)
        for _ in range(2):
            g.step(3, dt)
        res[flags] = g.get_psi()
    o = oracle.Oracle(nx, ny, nz, L, G=0.8, kappa=0.2)
    o.set_ic(psi.astype(np.complex128))
    for _ in range(2):
        o.step(3, dt)
    ref = o.get_psi()
    e32, e16 = rel_l2(res[0], ref), rel_l2(res[spe.SPE_PREC_SPLIT16], ref)
    print(f"{shape}: FP32 {e32:.2e}  split16 {e16:.2e}")
    assert e16 <= 1e-5, (e32, e16)
    assert not np.array_equal(res[0], res[spe.SPE_PREC_SPLIT16])   # the tensor path really ran
