"""Seeded synthetic initial conditions shared by the CUDA path's tests/benchmark and the oracle.

This module holds input synthesis only -- none of the split-step arithmetic.  The paper's own
workload (the Crater II halo, Sec. 4) needs an observational model that is not available, so
these seeded families stand in for it:

* ``gaussian_packets``: a sum of Gaussian wave packets with integer-mode momenta (periodic);
* ``soliton_halo``: a central soliton rho_c / (1 + 0.091 (r/r_c)^2)^8 plus a random-phase
  granular halo under an NFW-like envelope;
* ``plummer``: star particles from a Plummer sphere, velocities by the Aarseth-Henon-Wielen
  (1974) rejection method in the sphere's own potential.

Grid convention: node i of an axis of n points and length L sits at x_i = -L/2 + i L/n;
arrays are indexed [z, y, x] with x fastest.  The random-field filter below uses numpy's FFT
as an input-synthesis tool; it is not part of either solver.
"""
from __future__ import annotations

import math

import numpy as np

SOLITON_SHAPE_INTEGRAL = None  # filled lazily: 4 pi int_0^inf x^2 (1 + 0.091 x^2)^-8 dx


def axis_coords(n: int, L: float) -> np.ndarray:
    return -0.5 * L + (L / n) * np.arange(n)


def _mesh(n, L):
    nx, ny, nz = n
    Lx, Ly, Lz = L
    z, y, x = np.meshgrid(axis_coords(nz, Lz), axis_coords(ny, Ly), axis_coords(nx, Lx), indexing="ij")
    return x, y, z


def _min_image(d, L):
    return d - L * np.round(d / L)


def _norm3(n):
    if np.isscalar(n):
        return (int(n),) * 3
    return tuple(int(v) for v in n)


def _normL(L):
    if np.isscalar(L):
        return (float(L),) * 3
    return tuple(float(v) for v in L)


def gaussian_packets(n, L=1.0, n_packets=8, sigma=0.05, max_mode=8, mass=1.0, seed=1235,
                     dtype=np.complex128) -> np.ndarray:
    """Sum of ``n_packets`` Gaussian packets exp(-|r-c|^2/(4 sigma^2)) exp(i k.r), sigma the
    density standard deviation (minimum-image distance), centres uniform in the box, momenta
    k = 2 pi m / L with integer vectors |m| <= max_mode so each packet is periodic.  Every
    packet carries equal mass; the sum is rescaled to total mass ``mass``."""
    n = _norm3(n)
    L = _normL(L)
    rng = np.random.default_rng(seed)
    x, y, z = _mesh(n, L)
    dv = (L[0] / n[0]) * (L[1] / n[1]) * (L[2] / n[2])
    psi = np.zeros(x.shape, dtype=np.complex128)
    for _ in range(n_packets):
        c = (rng.random(3) - 0.5) * np.array(L)
        while True:
            m = rng.integers(-max_mode, max_mode + 1, size=3)
            if np.dot(m, m) <= max_mode * max_mode:
                break
        k = 2.0 * np.pi * m / np.array(L)
        r2 = _min_image(x - c[0], L[0]) ** 2 + _min_image(y - c[1], L[1]) ** 2 + _min_image(z - c[2], L[2]) ** 2
        p = np.exp(-r2 / (4.0 * sigma * sigma)) * np.exp(1j * (k[0] * x + k[1] * y + k[2] * z))
        p /= math.sqrt(np.sum(np.abs(p) ** 2) * dv)
        psi += p * math.sqrt(1.0 / n_packets)
    psi *= math.sqrt(mass / (np.sum(np.abs(psi) ** 2) * dv))
    return psi.astype(dtype)


def soliton_shape_integral() -> float:
    """4 pi int_0^inf x^2 (1 + a x^2)^-8 dx with a = 0.091, in closed form:
    4 pi a^{-3/2} Gamma(3/2) Gamma(13/2) / (2 Gamma(8))  (= 11.5865...)."""
    a = 0.091
    return 4.0 * math.pi * a ** -1.5 * math.gamma(1.5) * math.gamma(6.5) / (2.0 * math.gamma(8.0))


def soliton_halo(n, L=1.0, r_c=0.05, psi_mass=0.95, soliton_fraction=0.3, r_s=0.1, r_trunc=0.45,
                 k_filter_modes=16, seed=1236, dtype=np.complex64) -> np.ndarray:
    """Central soliton plus a granular halo.

    * soliton: rho_sol = rho_c / (1 + 0.091 (r/r_c)^2)^8, rho_c = M_sol / (I r_c^3) with I the
      shape integral, M_sol = soliton_fraction * psi_mass (r_c, r_s, r_trunc in units of L);
    * halo: sqrt(rho_env(r)) times a unit-variance complex Gaussian random field (seeded),
      Gaussian-filtered at k_f = 2 pi k_filter_modes / L; rho_env ~ 1/((r/r_s)(1 + r/r_s)^2)
      with r softened to max(r, dx) and tapered smoothly to zero around r_trunc;
    * psi = sqrt(rho_sol) + psi_halo, rescaled so sum |psi|^2 dV = psi_mass.
    """
    n = _norm3(n)
    L = _normL(L)
    Lm = min(L)
    rng = np.random.default_rng(seed)
    x, y, z = _mesh(n, L)
    dx = min(L[i] / n[i] for i in range(3))
    dv = (L[0] / n[0]) * (L[1] / n[1]) * (L[2] / n[2])
    r = np.sqrt(x * x + y * y + z * z)
    del x, y, z
    rc = r_c * Lm
    m_sol = soliton_fraction * psi_mass
    rho_c = m_sol / (soliton_shape_integral() * rc ** 3)
    amp_sol = np.sqrt(rho_c / (1.0 + 0.091 * (r / rc) ** 2) ** 8)
    # halo random field
    shape = amp_sol.shape
    g = (rng.standard_normal(shape, dtype=np.float32) + 1j * rng.standard_normal(shape, dtype=np.float32))
    g = g.astype(np.complex64)
    gk = np.fft.fftn(g)
    kf = 2.0 * np.pi * k_filter_modes / Lm
    kz = 2.0 * np.pi * np.fft.fftfreq(n[2], d=L[2] / n[2])
    ky = 2.0 * np.pi * np.fft.fftfreq(n[1], d=L[1] / n[1])
    kx = 2.0 * np.pi * np.fft.fftfreq(n[0], d=L[0] / n[0])
    filt = (np.exp(-kz[:, None, None] ** 2 / (2 * kf * kf)) * np.exp(-ky[None, :, None] ** 2 / (2 * kf * kf))
            * np.exp(-kx[None, None, :] ** 2 / (2 * kf * kf))).astype(np.float32)
    gk *= filt
    del filt
    g = np.fft.ifftn(gk).astype(np.complex64)
    del gk
    g /= np.sqrt(np.mean(np.abs(g) ** 2))
    rs = r_s * Lm
    rr = np.maximum(r, dx) / rs
    env = 1.0 / (rr * (1.0 + rr) ** 2)
    env *= 0.5 * (1.0 - np.tanh((r - r_trunc * Lm) / (0.02 * Lm)))
    m_halo = psi_mass - m_sol
    env *= m_halo / (np.sum(env) * dv)
    psi = amp_sol.astype(np.complex64) + (np.sqrt(env).astype(np.float32) * g)
    del g, env, amp_sol, r, rr
    mass = float(np.sum(np.abs(psi.astype(np.complex128)) ** 2) * dv)
    psi *= np.float32(math.sqrt(psi_mass / mass))
    return psi.astype(dtype)


def plummer(n_star, a=0.03, total_mass=0.05, L=1.0, r_max=0.45, G=1.0, seed=1237):
    """Plummer sphere centred in the box: positions by the inverse mass profile
    r = a / sqrt(X^{-2/3} - 1) (rejected beyond r_max*L), speeds q v_esc with q drawn from
    q^2 (1 - q^2)^{7/2} by rejection, v_esc = sqrt(2 G M / a) (1 + r^2/a^2)^{-1/4}, isotropic
    directions, equal masses.  a and r_max are in units of L (the smallest side).
    Returns (pos (n,3), vel (n,3), mass (n,)) in float64."""
    L = _normL(L)
    Lm = min(L)
    a = a * Lm
    rng = np.random.default_rng(seed)
    n = int(n_star)
    if n == 0:
        return np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0)
    r = np.empty(n)
    filled = 0
    while filled < n:
        X = rng.random(2 * (n - filled) + 16)
        X = X[X > 1e-12]
        rr = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        rr = rr[rr < r_max * Lm]
        take = min(n - filled, rr.size)
        r[filled:filled + take] = rr[:take]
        filled += take

    def iso(m):
        u = rng.random(m) * 2.0 - 1.0
        ph = rng.random(m) * 2.0 * np.pi
        s = np.sqrt(1.0 - u * u)
        return np.stack([s * np.cos(ph), s * np.sin(ph), u], axis=1)

    pos = r[:, None] * iso(n)
    q = np.empty(n)
    filled = 0
    while filled < n:
        m = 2 * (n - filled) + 16
        x4 = rng.random(m)
        x5 = rng.random(m)
        ok = 0.1 * x5 < x4 * x4 * (1.0 - x4 * x4) ** 3.5
        qq = x4[ok]
        take = min(n - filled, qq.size)
        q[filled:filled + take] = qq[:take]
        filled += take
    vesc = np.sqrt(2.0 * G * total_mass / a) * (1.0 + r * r / (a * a)) ** -0.25
    vel = (q * vesc)[:, None] * iso(n)
    mass = np.full(n, total_mass / n)
    # wrap into [-L/2, L/2)
    for ax in range(3):
        pos[:, ax] -= L[ax] * np.floor((pos[:, ax] + 0.5 * L[ax]) / L[ax])
    return pos, vel, mass


def uniform_particles(n_star, L=1.0, total_mass=0.05, vmax=0.0, seed=1238):
    """Particles uniform in the box with uniform random velocities in [-vmax, vmax]^3."""
    L = np.array(_normL(L))
    rng = np.random.default_rng(seed)
    pos = (rng.random((n_star, 3)) - 0.5) * L
    vel = (rng.random((n_star, 3)) * 2.0 - 1.0) * vmax
    mass = np.full(n_star, total_mass / max(n_star, 1))
    return pos, vel, mass


def kinetic_dt(n, L=1.0, hbar_over_m=1.0, safety=0.9):
    """The kinetic term of the Sec. 3.5 CFL bound times ``safety``: 0.5 * 4/(3 pi) dx^2 / eta."""
    n = _norm3(n)
    L = _normL(L)
    dx = min(L[i] / n[i] for i in range(3))
    return safety * 0.5 * 4.0 / (3.0 * math.pi) * dx * dx / hbar_over_m


# Workload table: the configurations the tests and the benchmark run (grid, steps, ICs).
WORKLOADS = {
    "packets32": dict(n=32, steps=100, ic="gaussian_packets", n_star=0, dt=0.2 * (1.0 / 32) ** 2),
    "halo256_stars1e6": dict(n=256, steps=1000, ic="soliton_halo", n_star=1_000_000, dt=None),
    "halo512": dict(n=512, steps=200, ic="soliton_halo", n_star=0, dt=None),
}


def make_workload(name, seed_offset=0, n=None, n_star=None):
    """Build (psi (complex64), pos, vel, mass, dt, steps) for a named workload.  ``n`` and
    ``n_star`` override the sizes for reduced-size parity cases of the same family."""
    w = dict(WORKLOADS[name])
    if n is not None:
        w["n"] = n
    if n_star is not None:
        w["n_star"] = n_star
    N = w["n"]
    if w["ic"] == "gaussian_packets":
        psi = gaussian_packets(N, seed=1235 + seed_offset).astype(np.complex64)
        psi_mass = 1.0
    else:
        psi_mass = 0.95 if w["n_star"] else 1.0
        psi = soliton_halo(N, psi_mass=psi_mass, seed=1236 + seed_offset)
    if w["n_star"]:
        pos, vel, mass = plummer(w["n_star"], total_mass=1.0 - psi_mass, seed=1237 + seed_offset)
    else:
        pos = vel = np.zeros((0, 3))
        mass = np.zeros(0)
    dt = w["dt"] if w["dt"] is not None else kinetic_dt(N)
    return psi, pos, vel, mass, dt, w["steps"]


def ensemble(count=64, sizes=(64, 96, 128, 192), rc_range=(0.03, 0.08), max_stars=100_000, seed=1239):
    """Independent halos of uneven sizes: per member a seeded grid size from ``sizes``, soliton core
    radius r_c uniform in ``rc_range`` (units of L), a star count uniform in [0, max_stars] (Plummer,
    5% of the mass when present), the soliton + granular halo field, and the kinetic CFL dt of its
    grid.  Returns a list of dicts (n, psi, pos, vel, mass, dt, r_c)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        rc = float(rng.uniform(*rc_range))
        nstar = int(rng.integers(0, max_stars + 1))
        psi_mass = 0.95 if nstar else 1.0
        psi = soliton_halo(n, r_c=rc, psi_mass=psi_mass, seed=seed * 1000 + i)
        if nstar:
            pos, vel, mass = plummer(nstar, total_mass=1.0 - psi_mass, seed=seed * 1000 + 500 + i)
        else:
            pos = vel = np.zeros((0, 3))
            mass = np.zeros(0)
        out.append(dict(n=n, psi=psi, pos=pos, vel=vel, mass=mass, dt=kinetic_dt(n), r_c=rc))
    return out


def fno_param_shapes(layers=4, modes=16, width=32, hidden=64, in_ch=4, out_ch=2):
    """[(name, shape)] of the FNO surrogate's flat parameter vector, in order: P, p, then per
    layer W, b, R (modes^3 x C_in x C_out x (re, im)), then Q1, q1, Q2, q2."""
    out = [("P", (width, in_ch)), ("p", (width,))]
    for l in range(layers):
        out += [(f"W{l}", (width, width)), (f"b{l}", (width,)), (f"R{l}", (modes ** 3, width, width, 2))]
    out += [("Q1", (hidden, width)), ("q1", (hidden,)), ("Q2", (out_ch, hidden)), ("q2", (out_ch,))]
    return out


def fno_init_params(layers=4, modes=16, seed=0, out_gain=0.1, width=32, hidden=64, in_ch=4, out_ch=2):
    """Seeded initial parameters of the FNO surrogate (float32): uniform(-1/sqrt(fan_in),
    1/sqrt(fan_in)) for the pointwise maps, spectral weights uniform in [0, 1/(C C)) per real
    component, and the last projection shrunk by out_gain so the untrained proposal stays close
    to the coarse step."""
    rng = np.random.default_rng(seed)
    fan = {"P": in_ch, "p": in_ch, "Q1": width, "q1": width, "Q2": hidden, "q2": hidden}
    parts = []
    for name, shape in fno_param_shapes(layers, modes, width, hidden, in_ch, out_ch):
        if name.startswith("R"):
            a = rng.random(shape) / (width * width)
        else:
            bound = 1.0 / math.sqrt(fan.get(name, width))
            a = rng.uniform(-bound, bound, shape)
            if name in ("Q2", "q2"):
                a = a * out_gain
        parts.append(a.ravel())
    return np.concatenate(parts).astype(np.float32)
