"""The closing half kick of spe_step is deferred into the next call's leading kick (KDK with the
half kicks of neighbouring steps merged, Sec. 3.1 / Algorithm 1): a run of single-step calls
must do exactly what one multi-step call does, every observation must see the synchronised
state, and a change of dt must first apply the owed kick with the old step's size."""
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


def halo(n, n_star, seed=0):
    psi, pos, vel, mass, dt, _ = inputs.make_workload("halo256_stars1e6", n=n, n_star=n_star)
    return psi.astype(np.complex64), pos.astype(np.float32), vel.astype(np.float32), mass.astype(np.float32), dt


def grid(spe, n, psi, pos, vel, mass, **kw):
    g = spe.Grid(n, G=1.0, max_particles=len(mass), **kw)
    g.set_ic(psi)
    g.add_particles(pos, vel, mass)
    return g


def test_single_step_calls_equal_one_call_bitwise(spe):
    n, steps = 64, 6
    psi, pos, vel, mass, dt = halo(n, 4000)
    a = grid(spe, n, psi, pos, vel, mass)
    b = grid(spe, n, psi, pos, vel, mass)
    for _ in range(steps):
        a.step(1, dt)
    b.step(steps, dt)
    pa, va = a.get_particles()
    pb, vb = b.get_particles()
    assert np.array_equal(a.get_psi(), b.get_psi())
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)


def test_last_mass_needs_no_closing_kick(spe):
    """The mass is measured inside the step; reading it leaves the kick deferred, and it equals the
    mass of the settled state (the kick is a phase)."""
    n = 64
    psi, pos, vel, mass, dt = halo(n, 2000)
    a = grid(spe, n, psi, pos, vel, mass)
    b = grid(spe, n, psi, pos, vel, mass)
    for _ in range(4):
        a.step(1, dt)
        a.last_mass()
    b.step(4, dt)
    assert np.array_equal(a.get_psi(), b.get_psi())
    m = a.last_mass()
    e = a.energy()["mass"]
    assert abs(m - e) <= 1e-6 * e


def test_observations_between_calls_see_the_synchronised_state(spe):
    """get_psi / energy between single-step calls apply the owed kick; the run then differs from
    the merged one only by rounding, and each observation matches the oracle's synchronised
    state."""
    n, steps = 64, 5
    psi, pos, vel, mass, dt = halo(n, 3000)
    a = grid(spe, n, psi, pos, vel, mass)
    b = grid(spe, n, psi, pos, vel, mass)
    o = oracle.Oracle(n, n, n, 1.0, G=1.0)
    o.set_ic(psi.astype(np.complex128))
    o.set_particles(pos.astype(np.float64), vel.astype(np.float64), mass.astype(np.float64))
    for _ in range(steps):
        a.step(1, dt)
        o.step(1, dt)
        got = a.get_psi()
        assert rel_l2(got, o.get_psi()) <= 1e-5
        ea, eo = a.energy(), o.energy()
        assert abs(ea["mass"] - eo["mass"]) <= 1e-6 * eo["mass"]
    b.step(steps, dt)
    assert rel_l2(a.get_psi(), b.get_psi()) <= 1e-6
    pa, _ = a.get_particles()
    pb, _ = b.get_particles()
    d = (pa - pb + 0.5) % 1.0 - 0.5
    assert np.abs(d).max() <= 1e-6


def test_dt_change_applies_the_owed_kick_first(spe):
    n = 64
    psi, pos, vel, mass, dt = halo(n, 3000)
    g = grid(spe, n, psi, pos, vel, mass)
    o = oracle.Oracle(n, n, n, 1.0, G=1.0)
    o.set_ic(psi.astype(np.complex128))
    o.set_particles(pos.astype(np.float64), vel.astype(np.float64), mass.astype(np.float64))
    for h in (dt, 0.5 * dt, 0.5 * dt, dt, -dt):
        g.step(2, h)
        o.step(2, h)
    assert rel_l2(g.get_psi(), o.get_psi()) <= 1e-5
    gp, gv = g.get_particles()
    op, ov = o.get_particles()
    d = (gp - op + 0.5) % 1.0 - 0.5
    assert np.abs(d).max() <= 1e-5


def test_set_ic_and_add_particles_settle_first(spe):
    """Replacing psi or adding stars after a step: the stars present before get the owed kick, the
    new ones do not (the oracle applies its closing kick inside each call)."""
    n = 64
    psi, pos, vel, mass, dt = halo(n, 2000)
    k = 1000
    g = spe.Grid(n, G=1.0, max_particles=len(mass))
    g.set_ic(psi)
    g.add_particles(pos[:k], vel[:k], mass[:k])
    o = oracle.Oracle(n, n, n, 1.0, G=1.0)
    o.set_ic(psi.astype(np.complex128))
    o.set_particles(pos[:k].astype(np.float64), vel[:k].astype(np.float64), mass[:k].astype(np.float64))
    g.step(3, dt)
    o.step(3, dt)
    g.add_particles(pos[k:], vel[k:], mass[k:])
    op, ov = o.get_particles()
    allp = np.concatenate([op, pos[k:].astype(np.float64)])
    allv = np.concatenate([ov, vel[k:].astype(np.float64)])
    o.set_particles(allp, allv, mass.astype(np.float64))
    psi2 = g.get_psi()
    g.set_ic(psi2)
    o.set_ic(psi2.astype(np.complex128))
    g.step(3, dt)
    o.step(3, dt)
    assert rel_l2(g.get_psi(), o.get_psi()) <= 1e-5
    gp, _ = g.get_particles()
    op, _ = o.get_particles()
    d = (gp - op + 0.5) % 1.0 - 0.5
    assert np.abs(d).max() <= 1e-5


def test_settle_is_idempotent(spe):
    n = 32
    psi, pos, vel, mass, dt = halo(n, 500)
    a = grid(spe, n, psi, pos, vel, mass)
    b = grid(spe, n, psi, pos, vel, mass)
    a.step(3, dt)
    a.settle()
    a.settle()
    a.sync()
    b.step(3, dt)
    assert np.array_equal(a.get_psi(), b.get_psi())


def test_mass_async_matches_last_mass(spe):
    """spe_mass_async queues the step's mass (cell volume applied on the device) without waiting;
    pinned-host and device destinations get exactly what spe_last_mass reports."""
    import torch
    n = 32
    psi, pos, vel, mass, dt = halo(n, 500)
    g = grid(spe, n, psi, pos, vel, mass, flags=spe.SPE_ASYNC)
    host = torch.zeros(4, dtype=torch.float64).pin_memory()
    dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    for k in range(4):
        g.step(1, dt)
        g.mass_async(host[k:k + 1])
    g.mass_async(dev)
    g.sync()
    last = g.last_mass()
    assert host[3].item() == last and dev.item() == last
    assert np.all(np.abs(host.numpy() / last - 1.0) < 1e-6)
    with pytest.raises(ValueError):
        g.mass_async(torch.zeros(1, dtype=torch.float64))          # pageable host memory


@pytest.mark.parametrize("flags_name", ["graph", "direct"])
def test_side_stream_stars_equal_serial_steps(spe, flags_name):
    """Outside profile mode the stars' kick-drift-deposit runs on a side stream beside the y and z
    transforms of psi (joined before the density pass, which reads their deposit).  The result must
    be bitwise that of the serial order profile mode keeps, with graphs and with direct launches."""
    n = 64
    psi, pos, vel, mass, dt = halo(n, 20000)
    flags = 0 if flags_name == "graph" else spe.SPE_NO_GRAPH
    a = grid(spe, n, psi, pos, vel, mass, flags=flags)
    b = grid(spe, n, psi, pos, vel, mass, flags=spe.SPE_PROFILE)
    for g in (a, b):
        g.step(70, dt)   # crosses a reordering of the stars
        g.step(3, dt)
    assert np.array_equal(a.get_psi(), b.get_psi())
    pa, va = a.get_particles()
    pb, vb = b.get_particles()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)
    assert np.array_equal(a.density(), b.density())
    a.destroy()
    b.destroy()
