"""The batch's persistent launch: one cooperative kernel per step walks the step's passes as eight
phases, each a work list of every member's tiles, with a grid-wide barrier between phases.

The members run the same pass bodies as lone grids with the same radix plans (tile widths only
regroup independent lines), so every member must be bitwise equal to the same grid stepped alone;
one member is also checked against the FP64 oracle.  The barrier's bounded wait is exercised by a
wait limit of zero injected from the host: the step must return SPE_ETIMEOUT instead of hanging,
and the context must stay usable."""
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


@pytest.fixture(scope="module")
def members():
    # sizes 128, 128, 96, 96, 192, 64; the second member without stars (the passes without the real
    # Phi store and without the deposit)
    ms = inputs.ensemble(count=6, sizes=(64, 96, 128, 192), max_stars=3000, seed=84)
    assert {m["n"] for m in ms} == {64, 96, 128, 192}
    z = np.zeros((0, 3))
    ms[1].update(pos=z, vel=z, mass=np.zeros(0))
    return ms


def make_batch(spe, members, persistent=True):
    b = spe.Batch([dict(nx=m["n"], G=1.0, max_particles=len(m["mass"])) for m in members])
    b.set_persistent(persistent)
    for g, m in zip(b.members, members):
        g.set_ic(m["psi"])
        if len(m["mass"]):
            g.add_particles(m["pos"], m["vel"], m["mass"])
    return b


def run_alone(spe, m, calls, steps):
    g = spe.Grid(m["n"], G=1.0, max_particles=len(m["mass"]))
    g.set_ic(m["psi"])
    if len(m["mass"]):
        g.add_particles(m["pos"], m["vel"], m["mass"])
    for _ in range(calls):
        g.step(steps, m["dt"])
    out = g.get_psi(), g.get_particles()[0], g.energy()["mass"]
    g.destroy()
    return out


def test_persistent_batch_equals_lone_grids_bitwise(spe, members):
    b = make_batch(spe, members)
    assert b.persistent()
    dts = [m["dt"] for m in members]
    l0 = b.launch_count()
    for _ in range(2):
        b.step(40, dts)                 # 80 steps: crosses a star reordering
    launches = b.launch_count() - l0
    for g, m in zip(b.members, members):
        psi, pos, mass = run_alone(spe, m, 2, 40)
        assert np.array_equal(g.get_psi(), psi), m["n"]
        assert np.array_equal(g.get_particles()[0], pos), m["n"]
        assert g.energy()["mass"] == mass
    # one launch per step (plus the stars' reordering every 64 steps), not 8-9 per member and step
    assert launches < 2 * 80 + 8 * len(members), launches
    b.destroy()


def test_persistent_batch_member_matches_oracle(spe, members):
    b = make_batch(spe, members)
    assert b.persistent()
    b.step(10, [m["dt"] for m in members])
    i = max(range(len(members)), key=lambda k: (len(members[k]["mass"]) > 0, members[k]["n"]))
    m = members[i]
    n = m["n"]
    o = oracle.Oracle(n, n, n, 1.0, G=1.0)
    o.set_ic(m["psi"].astype(np.complex128))
    if len(m["mass"]):
        o.set_particles(m["pos"].astype(np.float32).astype(np.float64),
                        m["vel"].astype(np.float32).astype(np.float64),
                        m["mass"].astype(np.float32).astype(np.float64))
    o.step(10, m["dt"])
    ref = o.get_psi()
    got = b.members[i].get_psi()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    if len(m["mass"]):
        d = (b.members[i].get_particles()[0] - o.get_particles()[0] + 0.5) % 1.0 - 0.5
        assert np.abs(d).max() <= 1e-5
    b.destroy()


def test_persistent_barrier_timeout_returns_status(spe, members):
    """A wait limit of zero: every grid-wide barrier that is not already complete gives up at once,
    the kernel leaves, and the step returns SPE_ETIMEOUT.  Afterwards the default limit and a fresh
    initial state give the lone-grid result again."""
    b = make_batch(spe, members)
    dts = [m["dt"] for m in members]
    b.set_persistent(True, wait_limit=0)
    assert b.step_status(1, dts) == spe.SPE_ETIMEOUT
    b.set_persistent(True, wait_limit=-1)
    for g, m in zip(b.members, members):
        g.clear_particles()
        g.set_ic(m["psi"])
        if len(m["mass"]):
            g.add_particles(m["pos"], m["vel"], m["mass"])
    b.step(5, dts)
    for g, m in zip(b.members, members):
        psi, pos, _ = run_alone(spe, m, 1, 5)
        assert np.array_equal(g.get_psi(), psi)
    b.destroy()


def test_graph_branches_when_persistent_is_off(spe, members):
    """The same batch through the graph of per-member branches gives the same bits."""
    a = make_batch(spe, members, persistent=True)
    c = make_batch(spe, members, persistent=False)
    assert a.persistent() and not c.persistent()
    dts = [m["dt"] for m in members]
    a.step(6, dts)
    c.step(6, dts)
    for ga, gc in zip(a.members, c.members):
        assert np.array_equal(ga.get_psi(), gc.get_psi())
    a.destroy()
    c.destroy()
