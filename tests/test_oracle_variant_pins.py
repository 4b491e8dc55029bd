"""Pins of the oracle's paper variants: the absorbing layer (Sec. 3.1), a static external potential
(Sec. 3.2.2, static particle mode) and the overall energy terms K, Q, V (Sec. 3.6).

Each is checked against special cases with closed forms, not against a retyped formula: the layer
is exactly 1 in the interior and exp(-alpha dt) / exp(-3 alpha dt) on a face / corner node; a
constant static potential is a pure global phase; the energy terms of a plane wave and of a real
sinusoidal field follow from the exact action of the central difference on sinusoids.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import Oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def coords(n, L):
    return -0.5 * L + (L / n) * np.arange(n)


def test_absorbing_layer_special_values():
    g = json.load(open(os.path.join(GOLDEN, "absorbing_mask_sec3_1.json")))
    alpha, nb = g["alpha"], g["N_b"]
    n, dt = 64, 1e-3
    o = Oracle(n, n, n, 1.0, G=0.0)
    o.set_absorb(alpha, nb)
    psi0 = np.full((n, n, n), 0.7 + 0.2j)
    o.set_ic(psi0)
    o.step(1, dt)   # uniform field, no potential: kick and drift leave it unchanged
    r = (o.get_psi() / psi0).real
    c = n // 2
    assert r[c, c, c] == pytest.approx(1.0, abs=1e-14)                     # interior
    assert r[c, c, 0] == pytest.approx(math.exp(-alpha * dt), rel=1e-12)    # face node x = -L/2
    assert r[0, 0, 0] == pytest.approx(math.exp(-3 * alpha * dt), rel=1e-12)  # corner node
    assert np.all(r <= 1.0 + 1e-15)
    # alpha = 0 is the plain step
    o2 = Oracle(n, n, n, 1.0, G=0.0)
    o2.set_absorb(0.0, nb)
    o2.set_ic(psi0)
    o2.step(1, dt)
    assert np.abs(o2.get_psi() - psi0).max() < 1e-14


def test_absorbing_layer_removes_outgoing_mass():
    n = 32
    x = coords(n, 1.0)
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    psi = np.exp(-((xx - 0.3) ** 2 + y ** 2 + z ** 2) / (4 * 0.05 ** 2)) * np.exp(1j * 2 * np.pi * 4 * xx)
    dt = 2e-4
    masses = []
    for alpha in (0.0, 10.0):
        o = Oracle(n, n, n, 1.0, G=0.0)
        o.set_absorb(alpha, 50)
        o.set_ic(psi)
        m0 = o.energy()["mass"]
        o.step(60, dt)
        masses.append(o.energy()["mass"] / m0)
    assert masses[0] == pytest.approx(1.0, abs=1e-13)
    assert masses[1] < 0.999


def test_constant_static_potential_is_a_global_phase():
    n, eta, c = 16, 0.6, 3.7
    rng = np.random.default_rng(21)
    psi = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    o = Oracle(n, n, n, 1.0, hbar_over_m=eta, G=0.0)
    o.set_ic(psi)
    o.set_static_phi(np.full((n, n, n), c))
    free = Oracle(n, n, n, 1.0, hbar_over_m=eta, G=0.0)
    free.set_ic(psi)
    dt, steps = 1e-4, 9
    o.step(steps, dt)
    free.step(steps, dt)
    assert np.abs(o.get_psi() - free.get_psi() * np.exp(-1j * c * dt * steps / eta)).max() < 1e-12
    e = o.energy()
    assert e["potential"] == pytest.approx(c * e["mass"], rel=1e-12)


def test_energy_terms_of_plane_wave():
    """sqrt(rho0) e^{i k x}: the central difference gives Im(conj psi D psi) = rho0 sin(k dx)/dx,
    so K = rho0 (eta sin(k dx)/dx)^2 V / 2, Q = 0, V = 0 (uniform density, Phi = 0)."""
    n, L, eta, rho0 = 32, 1.0, 0.8, 1.7
    x = coords(n, L)
    k = 2 * np.pi * 5 / L
    dx = L / n
    psi = np.broadcast_to(math.sqrt(rho0) * np.exp(1j * k * x), (n, n, n))
    o = Oracle(n, n, n, L, hbar_over_m=eta, G=1.0)
    o.set_ic(psi)
    v = o.virial()
    assert v["K"] == pytest.approx(0.5 * rho0 * (eta * math.sin(k * dx) / dx) ** 2 * L ** 3, rel=1e-12)
    assert abs(v["Q"]) < 1e-20 and abs(v["V"]) < 1e-12


def test_energy_terms_of_real_sinusoid():
    """psi = 1 + a cos(kx) (real, positive): K = 0; Q = eta^2 a^2 (sin(k dx)/dx)^2 V / 2;
    rho = (1 + a^2/2) + 2a cos(kx) + (a^2/2) cos(2kx) gives Phi exactly, and
    V = -4 pi G V_box (2 a^2 / k^2 + a^4 / (32 k^2))."""
    n, L, eta, a, G = 32, 1.0, 1.3, 0.4, 2.0
    x = coords(n, L)
    k = 2 * np.pi * 3 / L
    dx = L / n
    psi = np.broadcast_to((1.0 + a * np.cos(k * x)).astype(complex), (n, n, n))
    o = Oracle(n, n, n, L, hbar_over_m=eta, G=G)
    o.set_ic(psi)
    v = o.virial()
    assert abs(v["K"]) < 1e-20
    assert v["Q"] == pytest.approx(eta ** 2 * a ** 2 * 0.5 * (math.sin(k * dx) / dx) ** 2 * L ** 3, rel=1e-12)
    assert v["V"] == pytest.approx(-4 * math.pi * G * L ** 3 * (2 * a ** 2 / k ** 2 + a ** 4 / (32 * k ** 2)),
                                   rel=1e-12)
    assert v["E"] == pytest.approx(v["K"] + v["Q"] + v["V"], rel=1e-14)
