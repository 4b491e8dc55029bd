"""GPU parity of the paper variants against the oracle: the absorbing layer (Sec. 3.1), a static
external potential (Sec. 3.2.2, static particle mode) and the K/Q/V energy terms (Sec. 3.6).
Tolerances as in test_gpu_parity.py (rel-L2 psi <= 1e-5, positions <= 1e-5 of the box)."""
import math

import numpy as np
import pytest

import oracle
from paper_2606_25026_gb300 import inputs

pytestmark = pytest.mark.gpu

PSI_TOL = 1e-5


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


def f64(a):
    return np.asarray(a).astype(np.complex64).astype(np.complex128) if np.iscomplexobj(a) else \
        np.asarray(a).astype(np.float32).astype(np.float64)


def coords(n, L=1.0):
    return -0.5 * L + (L / n) * np.arange(n)


def test_absorbing_layer_parity(spe):
    n, alpha, nb = 64, 10.0, 50
    x = coords(n)
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    psi = (np.exp(-((xx - 0.3) ** 2 + y ** 2 + z ** 2) / (4 * 0.05 ** 2)) * np.exp(1j * 2 * np.pi * 6 * xx)
           + 0.3 * np.exp(-((xx + 0.1) ** 2 + (y - 0.35) ** 2 + z ** 2) / (4 * 0.06 ** 2)))
    dt = inputs.kinetic_dt(n)
    g = spe.Grid(n, G=1.0, absorb_alpha=alpha, absorb_nb=nb)
    g.set_ic(psi.astype(np.complex64))
    o = oracle.Oracle(n, n, n, 1.0, G=1.0)
    o.set_absorb(alpha, nb)
    o.set_ic(f64(psi))
    m0 = o.energy()["mass"]
    for _ in range(3):
        g.step(40, dt)
        o.step(40, dt)
    assert rel_l2(g.get_psi(), o.get_psi()) <= PSI_TOL
    mg, mo = g.energy()["mass"], o.energy()["mass"]
    assert mo < m0 * (1 - 1e-4)          # the layer removed mass
    assert abs(mg - mo) <= 1e-6 * mo


def test_static_potential_with_stars_parity(spe):
    n = 64
    psi, pos, vel, mass, dt, _ = inputs.make_workload("halo256_stars1e6", n=n, n_star=8000)
    x = coords(n)
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    phib = (40.0 * np.cos(2 * np.pi * xx) + 25.0 * np.sin(4 * np.pi * y) * np.cos(2 * np.pi * z)).astype(np.float32)
    g = spe.Grid(n, G=1.0, max_particles=len(mass), flags=spe.SPE_STATIC_POTENTIAL)
    g.set_ic(psi)
    g.add_particles(pos, vel, mass)
    g.set_static_potential(phib)
    o = oracle.Oracle(n, n, n, 1.0, G=1.0)
    o.set_ic(f64(psi))
    o.set_particles(f64(pos), f64(vel), f64(mass))
    o.set_static_phi(phib.astype(np.float64))
    for _ in range(2):
        g.step(8, dt)
        o.step(8, dt)
    assert rel_l2(g.get_psi(), o.get_psi()) <= PSI_TOL
    gp, _ = g.get_particles()
    op, _ = o.get_particles()
    d = (gp - op + 0.5) % 1.0 - 0.5
    assert np.abs(d).max() <= 1e-5
    phg, pho = g.potential(), o.potential()
    assert np.abs(phg - pho).max() <= 1e-5 * np.abs(pho).max()
    eg, eo = g.energy(), o.energy()
    assert eg["potential"] == pytest.approx(eo["potential"], rel=1e-5)
    assert eg["total"] == pytest.approx(eo["total"], rel=1e-5)


def test_constant_static_potential_phase_gpu(spe):
    n, eta, c = 32, 0.6, 3.7
    psi = inputs.gaussian_packets(n, seed=5).astype(np.complex64)
    g = spe.Grid(n, G=0.0, hbar_over_m=eta, flags=spe.SPE_STATIC_POTENTIAL)
    g.set_ic(psi)
    g.set_static_potential(np.full((n, n, n), c, np.float32))
    h = spe.Grid(n, G=0.0, hbar_over_m=eta)
    h.set_ic(psi)
    dt, steps = 1e-4, 12
    g.step(steps, dt)
    h.step(steps, dt)
    assert rel_l2(g.get_psi(), h.get_psi() * np.exp(-1j * c * dt * steps / eta)) <= 1e-6


def test_virial_terms_parity(spe):
    n = 64
    psi, _, _, _, dt, _ = inputs.make_workload("halo256_stars1e6", n=n, n_star=0)
    g = spe.Grid(n, G=1.0, hbar_over_m=0.9)
    g.set_ic(psi)
    o = oracle.Oracle(n, n, n, 1.0, G=1.0, hbar_over_m=0.9)
    o.set_ic(f64(psi))
    vg, vo = g.virial(), o.virial()
    for k in ("K", "Q", "V", "E", "virial"):
        assert vg[k] == pytest.approx(vo[k], rel=1e-5), (k, vg[k], vo[k])
    g.step(10, dt)
    o.step(10, dt)
    vg, vo = g.virial(), o.virial()
    for k in ("K", "Q", "V"):
        assert vg[k] == pytest.approx(vo[k], rel=1e-5), (k, vg[k], vo[k])


def test_static_potential_needs_flag(spe):
    g = spe.Grid(16, G=1.0)
    with pytest.raises(spe.SpeError) as e:
        g.set_static_potential(np.zeros((16, 16, 16), np.float32))
    assert e.value.status == spe.SPE_ESTATE
