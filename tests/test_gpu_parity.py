"""GPU path (libspe through its C ABI) against the FP64 oracle, element by element.

Tolerances (FP32 path vs FP64 oracle):
  * psi: relative L2 error <= 1e-5;
  * particle positions: <= 1e-5 of the box (periodic distance);
  * potential / density: max error <= 1e-5 of the field's max magnitude;
  * energies: relative 1e-5 (mass 1e-6).
The FP32 error budget behind 1e-5: each 1D pass rounds at ~eps32 * log2(N) ~ 1e-6 per step of
four 3D transforms, accumulating like a random walk over the steps these cases run.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_25026_gb300 import inputs

pytestmark = pytest.mark.gpu

PSI_TOL = 1e-5
POS_TOL = 1e-5


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


def c64(a):
    return np.ascontiguousarray(a, dtype=np.complex64)


def as_oracle(a):
    """The exact values the FP32 path was given, in FP64."""
    return np.asarray(a).astype(np.complex64).astype(np.complex128) if np.iscomplexobj(a) else \
        np.asarray(a).astype(np.float32).astype(np.float64)


def run_pair(spe, shape, psi, steps, dt, L=1.0, eta=1.0, G=1.0, kappa=0.0, parts=None, calls=1, flags=0):
    nz, ny, nx = shape
    g = spe.Grid(nx, ny, nz, L=L, hbar_over_m=eta, G=G, kappa=kappa,
                 max_particles=0 if parts is None else len(parts[2]), flags=flags)
    g.set_ic(c64(psi))
    o = oracle.Oracle(nx, ny, nz, L, hbar_over_m=eta, G=G, kappa=kappa)
    o.set_ic(as_oracle(psi))
    if parts is not None:
        pos, vel, mass = parts
        g.add_particles(pos, vel, mass)
        o.set_particles(as_oracle(pos), as_oracle(vel), as_oracle(mass))
    for _ in range(calls):
        g.step(steps, dt)
        o.step(steps, dt)
    return g, o


def periodic_err(a, b, L):
    L = np.asarray(L, dtype=float) * np.ones(3)
    d = (a - b + 0.5 * L) % L - 0.5 * L
    return float(np.abs(d).max() / L.min())


# --------------------------------------------------------------------------- closed forms on the GPU


def test_free_gaussian_gpu_matches_closed_form_and_oracle(spe):
    n, s0, eta = 64, 0.05, 0.7
    x = -0.5 + np.arange(n) / n
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    k0 = 2 * np.pi * np.array([2.0, -1.0, 3.0])
    c = np.array([-0.1, 0.05, 0.0])
    psi = (2 * np.pi * s0 ** 2) ** -0.75 * np.exp(
        -((xx - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (4 * s0 ** 2)
    ) * np.exp(1j * (k0[0] * xx + k0[1] * y + k0[2] * z))
    dt = 0.002
    g, o = run_pair(spe, (n, n, n), psi, 6, dt, eta=eta, G=0.0, flags=spe.SPE_NO_CFL_CHECK)
    assert rel_l2(g.get_psi(), o.get_psi()) <= PSI_TOL


def test_plane_wave_phase_exact(spe):
    nx, ny, nz, L = 32, 16, 8, (2.0, 1.0, 1.0)
    x = -0.5 * L[0] + L[0] * np.arange(nx) / nx
    eta, kappa, rho0 = 0.5, 3.0, 2.0
    k0 = 2 * np.pi * 3 / L[0]
    psi = np.broadcast_to(math.sqrt(rho0) * np.exp(1j * k0 * x), (nz, ny, nx))
    dt, steps = 1e-3, 20
    g = spe.Grid(nx, ny, nz, L=L, hbar_over_m=eta, G=1.3, kappa=kappa)
    g.set_ic(c64(psi))
    g.step(steps, dt)
    ref = psi * np.exp(-1j * (eta * k0 ** 2 / 2 + kappa * rho0 / eta) * dt * steps)
    assert rel_l2(g.get_psi(), ref) < 2e-6


def test_poisson_sinusoid_gpu(spe):
    nx, ny, nz, L = 48, 32, 16, (1.5, 1.0, 0.5)
    G, rho0, A = 2.5, 3.0, 0.7
    m = np.array([2, -1, 1])
    kv = 2 * np.pi * m / np.array(L)
    ax = [-0.5 * L[i] + L[i] * np.arange(nn) / nn for i, nn in enumerate((nx, ny, nz))]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    ph = kv[0] * x + kv[1] * y + kv[2] * z
    g = spe.Grid(nx, ny, nz, L=L, G=G)
    g.set_ic(c64(np.sqrt(rho0 + A * np.cos(ph))))
    phi = g.potential()
    ref = -4 * np.pi * G * A * np.cos(ph) / np.dot(kv, kv)
    assert np.abs(phi - ref).max() <= 1e-5 * np.abs(ref).max()


# --------------------------------------------------------------------------- parity with the oracle


def test_packets32_full_run_parity(spe):
    """32^3 periodic grid, 8 Gaussian packets, dt = 0.2 dx^2, 100 steps, G = 1."""
    psi, _, _, _, dt, steps = inputs.make_workload("packets32")
    g, o = run_pair(spe, psi.shape, psi, steps, dt)
    err = rel_l2(g.get_psi(), o.get_psi())
    assert err <= PSI_TOL, err
    eg, eo = g.energy(), o.energy()
    assert abs(eg["mass"] - eo["mass"]) <= 1e-6 * eo["mass"]
    for k in ("kinetic", "potential", "total"):
        assert abs(eg[k] - eo[k]) <= 1e-5 * abs(eo["kinetic"]), (k, eg[k], eo[k])


def test_packets32_thousand_steps(spe):
    """The same 32^3 packets for 1000 steps (the step count of the 256^3 workload): FP32 rounding
    must not accumulate coherently from step to step."""
    psi, _, _, _, dt, _ = inputs.make_workload("packets32")
    g, o = run_pair(spe, psi.shape, psi, 250, dt, calls=4)
    err = rel_l2(g.get_psi(), o.get_psi())
    print(f"packets32 x1000 rel-L2 {err:.3e}")
    assert err <= PSI_TOL, err


SIZES = [4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024]


@pytest.mark.parametrize("N", SIZES)
def test_every_transform_length_on_every_axis(spe, N):
    """Each supported length along x, y and z in turn (other axes short), random psi, gravity and
    self-interaction on, several steps: exercises every FFT plan, the ragged column tiles of the
    half spectrum and partial row tiles."""
    rng = np.random.default_rng(N)
    other = 8 if N >= 256 else 12
    for shape in ((other, other, N), (other, N, other), (N, other, other)):
        nz, ny, nx = shape
        psi = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * 0.3 + 1.0
        L = (1.0, 0.7, 1.3)
        dx = min(L[0] / nx, L[1] / ny, L[2] / nz)
        dt = 0.15 * dx * dx
        g, o = run_pair(spe, shape, psi, 3, dt, L=L, G=0.8, kappa=0.2, calls=2)
        err = rel_l2(g.get_psi(), o.get_psi())
        assert err <= PSI_TOL, (shape, err)


def test_halo_with_stars_parity(spe):
    """Soliton + granular halo with Plummer stars (the 256^3 workload's family) at 64^3 and 2e4
    stars, 20 steps in two calls."""
    psi, pos, vel, mass, dt, _ = inputs.make_workload("halo256_stars1e6", n=64, n_star=20000)
    g, o = run_pair(spe, psi.shape, psi, 10, dt, parts=(pos, vel, mass), calls=2)
    err = rel_l2(g.get_psi(), o.get_psi())
    assert err <= PSI_TOL, err
    gp, gv = g.get_particles()
    op, ov = o.get_particles()
    assert periodic_err(gp, op, 1.0) <= POS_TOL
    assert np.abs(gv - ov).max() <= 1e-4 * np.abs(ov).max()
    rho_g, rho_o = g.density(), o.density()
    assert np.abs(rho_g - rho_o).max() <= 1e-5 * rho_o.max()
    phi_g, phi_o = g.potential(), o.potential()
    assert np.abs(phi_g - phi_o).max() <= 1e-5 * np.abs(phi_o).max()
    eg, eo = g.energy(), o.energy()
    for k in ("mass", "kinetic", "potential", "star_kinetic", "total", "max_abs_phi"):
        assert abs(eg[k] - eo[k]) <= 1e-5 * max(abs(eo[k]), abs(eo["potential"])), (k, eg[k], eo[k])
    assert g.suggest_dt() == pytest.approx(o.suggest_dt(), rel=1e-5)


def test_full_size_256_with_1e6_stars_parity(spe):
    """The benchmark workload at full size (256^3, 1e6 stars) in the benchmark's launch
    configuration, 3 steps against the oracle."""
    psi, pos, vel, mass, dt, _ = inputs.make_workload("halo256_stars1e6")
    g, o = run_pair(spe, psi.shape, psi, 3, dt, parts=(pos, vel, mass))
    err = rel_l2(g.get_psi(), o.get_psi())
    assert err <= PSI_TOL, err
    gp, _ = g.get_particles()
    op, _ = o.get_particles()
    assert periodic_err(gp, op, 1.0) <= POS_TOL


def test_fast_stars_sweeping_rows_parity(spe):
    """Stars spread over the whole box and moving ~0.7 cells per step across y and z rows: the
    density pass must read every row that got deposit (rows are marked by the star kernel and
    cleared by the density pass), also after energy() deposited and cleared on its own."""
    n = 32
    rng = np.random.default_rng(91)
    psi = inputs.gaussian_packets(n, seed=92).astype(np.complex64)
    dt = inputs.kinetic_dt(n)
    m = 2000
    pos = rng.uniform(-0.5, 0.5, (m, 3)).astype(np.float32)
    vel = (rng.choice([-1.0, 1.0], (m, 3)) * rng.uniform(0.4, 0.7, (m, 3)) / n / dt).astype(np.float32)
    mass = np.full(m, 0.2 / m, np.float32)
    g = spe.Grid(n, G=1.0, max_particles=m)
    g.set_ic(psi)
    g.add_particles(pos, vel, mass)
    o = oracle.Oracle(n, n, n, 1.0, G=1.0)
    o.set_ic(as_oracle(psi))
    o.set_particles(as_oracle(pos), as_oracle(vel), as_oracle(mass))
    for call in range(3):
        g.step(5, dt)
        o.step(5, dt)
        eg, eo = g.energy(), o.energy()
        assert abs(eg["potential"] - eo["potential"]) <= 1e-5 * abs(eo["potential"]), call
    assert rel_l2(g.get_psi(), o.get_psi()) <= PSI_TOL
    gp, _ = g.get_particles()
    op, _ = o.get_particles()
    assert periodic_err(gp, op, 1.0) <= POS_TOL


def test_heavy_star_cluster_uses_the_64bit_deposit_box_parity(spe):
    """64 equal stars in a compact cluster: each holds 1/64 of the star mass, so its CIC shares
    (up to 2^44 quanta) exceed what the star block's 32-bit deposit halves hold, and the block
    deposits through 64-bit shared counters instead; the cluster is small enough for the block's
    shared-memory boxes.  Density, psi and the stars must match the oracle."""
    n = 32
    rng = np.random.default_rng(93)
    psi = inputs.gaussian_packets(n, seed=94).astype(np.complex64)
    dt = inputs.kinetic_dt(n)
    m = 64
    pos = rng.uniform(-0.05, 0.05, (m, 3)).astype(np.float32)
    vel = rng.normal(0.0, 0.05 / n / dt, (m, 3)).astype(np.float32)
    mass = np.full(m, 0.3 / m, np.float32)
    g = spe.Grid(n, G=1.0, max_particles=m)
    g.set_ic(psi)
    g.add_particles(pos, vel, mass)
    o = oracle.Oracle(n, n, n, 1.0, G=1.0)
    o.set_ic(as_oracle(psi))
    o.set_particles(as_oracle(pos), as_oracle(vel), as_oracle(mass))
    rho_g, rho_o = g.density().astype(np.float64), o.density()
    assert np.abs(rho_g - rho_o).max() <= 1e-5 * np.abs(rho_o).max()
    g.step(8, dt)
    o.step(8, dt)
    rho_g, rho_o = g.density().astype(np.float64), o.density()
    assert np.abs(rho_g - rho_o).max() <= 1e-5 * np.abs(rho_o).max()
    assert rel_l2(g.get_psi(), o.get_psi()) <= PSI_TOL
    gp, _ = g.get_particles()
    op, _ = o.get_particles()
    assert periodic_err(gp, op, 1.0) <= POS_TOL


# --------------------------------------------------------------------------- properties at any size


def test_reversibility_and_mass_512(spe):
    """512^3 soliton halo: n steps with +dt and n with -dt return psi(0) (KDK is time
    reversible), and the mass is conserved (unitary steps) -- properties that hold at any size."""
    psi = inputs.soliton_halo(512, psi_mass=1.0, seed=1240)
    dt = inputs.kinetic_dt(512)
    g = spe.Grid(512, G=1.0)
    g.set_ic(psi)
    m0 = g.energy()["mass"]
    g.step(5, dt)
    assert abs(g.last_mass() - m0) <= 1e-6 * m0
    g.step(5, -dt)
    err = rel_l2(g.get_psi(), psi.astype(np.complex128))
    assert err <= 2e-6, err


def test_determinism_with_stars(spe):
    psi, pos, vel, mass, dt, _ = inputs.make_workload("halo256_stars1e6", n=32, n_star=5000)
    outs = []
    for _ in range(2):
        g = spe.Grid(32, G=1.0, max_particles=len(mass))
        g.set_ic(psi)
        g.add_particles(pos, vel, mass)
        g.step(7, dt)
        outs.append((g.get_psi(), g.get_particles()[0]))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_restart_from_checkpoint(spe):
    psi, pos, vel, mass, dt, _ = inputs.make_workload("halo256_stars1e6", n=32, n_star=3000)
    g = spe.Grid(32, G=1.0, max_particles=len(mass))
    g.set_ic(psi)
    g.add_particles(pos, vel, mass)
    g.step(5, dt)
    cpsi = g.get_psi()
    cpos, cvel = g.get_particles()
    g.step(5, dt)
    h = spe.Grid(32, G=1.0, max_particles=len(mass))
    h.set_ic(cpsi)
    h.add_particles(cpos, cvel, mass)
    h.step(5, dt)
    assert rel_l2(h.get_psi(), g.get_psi()) <= 1e-6
    assert periodic_err(h.get_particles()[0], g.get_particles()[0], 1.0) <= 1e-6


# --------------------------------------------------------------------------- errors


def test_error_statuses(spe):
    with pytest.raises(spe.SpeError) as e:
        spe.Grid(100)
    assert e.value.status == spe.SPE_EINVAL
    g = spe.Grid(16, max_particles=4)
    g.set_ic(np.ones((16, 16, 16), np.complex64))
    with pytest.raises(spe.SpeError) as e:
        g.step(1, 1.0)  # far above the kinetic CFL bound
    assert e.value.status == spe.SPE_ECFL
    with pytest.raises(spe.SpeError) as e:
        g.add_particles(np.zeros((5, 3)), np.zeros((5, 3)), np.ones(5))
    assert e.value.status == spe.SPE_ENOMEM
    bad = np.ones((16, 16, 16), np.complex64)
    bad[3, 4, 5] = np.nan
    g.set_ic(bad)
    with pytest.raises(spe.SpeError) as e:
        g.step(1, 1e-4)
    assert e.value.status == spe.SPE_ENONFINITE


def test_device_buffers_and_launch_count(spe):
    import torch
    psi = inputs.gaussian_packets(32, seed=3).astype(np.complex64)
    g = spe.Grid(32, G=1.0)
    g.set_ic(torch.from_numpy(psi).cuda())
    g.launch_count(reset=True)
    g.step(4, 1e-4)
    assert g.launch_count() == 4 * 8 + 4      # 8 kernels per step, Phi(0) solve; the closing kick deferred
    g.settle()
    assert g.launch_count() == 4 * 8 + 4 + 1  # ... and applied
    out = torch.empty(psi.shape, dtype=torch.complex64, device="cuda")
    g.get_psi(out)
    assert rel_l2(out.cpu().numpy(), g.get_psi()) == 0.0
    d = torch.empty(psi.shape, dtype=torch.float32, device="cuda")
    g.density(d)
    assert np.allclose(d.cpu().numpy(), np.abs(g.get_psi()) ** 2, rtol=1e-6, atol=0)
