"""Benchmark: split-step Schroedinger-Poisson grid-cell-steps/s on GB300.

Workload (default, ``halo512``): one 512^3 complex64 grid, central soliton + granular halo (the
256^3 family at twice the resolution), no stars, FP32, dt from the Sec. 3.5 kinetic CFL term.  One
"step" is one full kick-drift-kick step (every kernel of the hot path).  The same line carries the
256^3 grid with 1e6 Plummer stars (CIC coupling) as the nested key ``halo256_stars1e6``.

Prints one JSON line (rank 0).  ``value`` is device-resident throughput (inputs already in HBM,
CUDA events on the grid's stream, K steps in one spe_step call: every step after the first is a
CUDA graph replay).  ``e2e`` is the same metric through the C ABI with host buffers: pinned-host
upload of the initial field (and stars), K single-step calls each followed by a device->host read
of the step's mass, and the final download, all inside the timed region.  ``roofline`` is the
dominant kernel's algorithmic bytes (the per-pass byte model of the fused axis-pass schedule: 20 B
per cell for each x pass, 24 with stars) over its CUDA-event duration, taken in a second run of the
same K steps with events around every (direct) launch, against the measured HBM copy bandwidth.
``cpu_baseline`` is the FP64 oracle on the host cores on a time-bounded number of steps of the same
workload from the same initial state, and ``psi_error`` compares the GPU after that many steps with
it.

Multi-GPU: the grid does not shard here; N ranks run N independent replicas (weak scaling).
``--impl reference`` times the FP64 CPU oracle as the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2606_25026_gb300 import replicas  # noqa: E402

# Algorithmic HBM bytes per grid cell for one launch of each kernel kind: the per-pass byte model of
# the fused axis-pass schedule (reads + writes the step cannot avoid at that pass; psi complex64
# 8 B/cell, a half spectrum 4 B/cell, a real field 4 B/cell):
#   x_kick_fwd        : R psi 8 + R Phi_hat 4 + W psi 8                 = 20  (+ W Phi 4 with stars)
#   y_fft_psi         : R 8 + W 8                                       = 16
#   z_fft_drift       : R 8 + W 8                                       = 16
#   x_inv_density_r2c : R psi_hat 8 + W psi 8 + W rho_hat 4             = 20  (+ R rho_* 4 with stars)
#   y_fft_rho, z_fft_poisson : R 4 + W 4 (half spectrum)                = 8
#   x_kick_final      : as x_kick_fwd without the transform
# Step: 112 B/cell without stars, 120 with, plus about 100 B per star for the star kernel.
MODEL_BYTES = {
    "x_kick_fwd": 20.0, "y_fft_psi": 16.0, "z_fft_drift": 16.0, "x_inv_density_r2c": 20.0,
    "y_fft_rho": 8.0, "z_fft_poisson": 8.0, "x_kick_final": 20.0,
}
MODEL_BYTES_STARS = dict(MODEL_BYTES, x_kick_fwd=24.0, x_inv_density_r2c=24.0, x_kick_final=24.0)
MODEL_BYTES_PER_STAR = 100.0
# The implementation's own accounting with stars: its deposit is int64 fixed point, read (8) and
# cleared (8) by the density pass on the fraction f of rows (y, z) the stars' stencils touch, instead
# of a 4-byte real rho_* read: 20 + 16 f for that pass (36 at f = 1).
IMPL_BYTES_STARS = dict(MODEL_BYTES_STARS, x_inv_density_r2c=36.0)
FALLBACK_HBM_GBS = 6800.0


def deposit_row_fraction(pos, shape, L=1.0):
    """Fraction of the (y, z) rows that the stars' CIC stencils (nodes i0, i0 + 1 per axis) touch:
    the density pass reads and clears the deposit of those rows only."""
    nz, ny, nx = shape
    if len(pos) == 0:
        return 0.0
    u = (np.asarray(pos, dtype=np.float64) + 0.5 * L) / L
    j0 = np.floor(u[:, 1] * ny).astype(np.int64) % ny
    k0 = np.floor(u[:, 2] * nz).astype(np.int64) % nz
    rows = np.concatenate([((k0 + dz) % nz) * ny + (j0 + dy) % ny for dy in (0, 1) for dz in (0, 1)])
    return float(np.unique(rows).size) / (ny * nz)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="halo512",
                    choices=["halo256_stars1e6", "halo512", "packets32", "ensemble64", "fno64", "precision512"])
    ap.add_argument("--members", type=int, default=64, help="ensemble64: number of halos")
    ap.add_argument("--fno-epochs", type=int, default=8, help="fno64: training epochs over the pairs")
    ap.add_argument("--fno-train", type=int, default=2000, help="fno64: training trajectories")
    ap.add_argument("--fno-test", type=int, default=200, help="fno64: held-out trajectories")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tiles", default=None,
                    help="Y,Z: pin the strided passes' tile widths instead of autotuning (with --plans)")
    ap.add_argument("--plans", default=None, help="Y,Z: pin the strided passes' radix schedules (0, 1, 2)")
    ap.add_argument("--grid", default=None,
                    help="NXxNYxNZ: run the workload's initial-condition family on this grid instead "
                         "(profiling cases; the stars keep their count)")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "split16"],
                    help="split16: radix-16 DFT stages of 256/512-point axes on the tensor cores")
    ap.add_argument("--no-tma", action="store_true",
                    help="strided passes stage their tiles with per-thread copies instead of TMA")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-nested", action="store_true",
                    help="halo512: skip the nested 256^3 + 1e6-star measurement")
    return ap.parse_args()


def source_hash() -> str:
    """Hash of the solver's CUDA sources (the surrogate's fno* and surrogate.cu files excluded),
    comments and whitespace left out, so that only a change of the code itself invalidates the
    recorded DRAM traffic."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2606_25026_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")) and not f.startswith(("fno", "surrogate")):
            text = open(os.path.join(csrc, f), encoding="utf-8").read()
            text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
            text = re.sub(r"//[^\n]*", " ", text)
            h.update(f.encode())
            h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def recorded_traffic(kernel: str, workload: str):
    """dram bytes per launch from the committed ncu summary, if taken on the current sources."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    want = source_hash()
    for line in open(path):
        if line.startswith("#") or "=" not in line:
            continue
        kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
        if kv.get("kernel") == kernel and kv.get("workload") == workload and kv.get("source_hash") == want:
            return float(kv["bytes_per_launch"])
    return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"spe_clocks_{os.getpid()}.csv")

    def start(self, ready_s=10.0):
        """Start sampling every 100 ms and return once the first sample is written, so that the
        sampler is live when the timed region begins."""
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t_end = time.time() + ready_s
        while time.time() < t_end and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)
        self.t0 = time.time()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.remove(self.path)
        if not rows:
            return None
        window_ms = (time.time() - self.t0) * 1e3
        sm = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows), "interval_ms": 100, "window_ms": round(window_ms, 1)}


def make_inputs(workload, grid=None):
    from paper_2606_25026_gb300 import inputs
    n = tuple(int(v) for v in grid.lower().split("x")) if grid else None
    psi, pos, vel, mass, dt, _ = inputs.make_workload(workload, n=n)
    return (psi.astype(np.complex64), pos.astype(np.float32), vel.astype(np.float32), mass.astype(np.float32),
            float(dt))


def cpu_baseline(psi, pos, vel, mass, dt, budget_s=10.0, max_steps=20, min_steps=1):
    """The FP64 oracle on the host cores: KDK steps of the same workload, one at a time until
    about budget_s seconds of CPU work (at least min_steps; the Phi(0) solve before them is not
    timed).  Returns (cell-steps/s, threads, seconds, steps, (psi, star positions) after the last
    step, energy at the start, energy at the end)."""
    import oracle
    oracle.build()
    nz, ny, nx = psi.shape
    o = oracle.Oracle(nx, ny, nz, 1.0, G=1.0)
    o.set_ic(psi.astype(np.complex128))
    if len(mass):
        o.set_particles(pos.astype(np.float64), vel.astype(np.float64), mass.astype(np.float64))
    o.potential()
    e0 = o.energy()
    sec, steps = 0.0, 0
    while steps < max_steps and (steps < min_steps or sec < budget_s):
        t0 = time.perf_counter()
        o.step(1, dt)
        sec += time.perf_counter() - t0
        steps += 1
    last = (o.get_psi(), o.get_particles()[0] if len(mass) else None)
    e1 = o.energy()
    del o
    return psi.size * steps / sec, oracle.threads(), sec, steps, last, e0, e1


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    if world > 1:
        # the launcher sets one OpenMP thread per rank; rank 0 runs alone here and takes the cores
        os.environ["OMP_NUM_THREADS"] = str(os.cpu_count() or 1)
    psi, pos, vel, mass, dt = make_inputs(args.workload)
    import oracle
    oracle.build()
    nz, ny, nx = psi.shape
    o = oracle.Oracle(nx, ny, nz, 1.0, G=1.0)
    o.set_ic(psi.astype(np.complex128))
    if len(mass):
        o.set_particles(pos.astype(np.float64), vel.astype(np.float64), mass.astype(np.float64))
    budget = 150.0
    t_start = time.perf_counter()
    for _ in range(min(args.warmup, 1)):
        o.step(1, dt)
    done, t_tot = 0, 0.0
    while done < args.steps and (time.perf_counter() - t_start) < budget:
        t0 = time.perf_counter()
        o.step(1, dt)
        t_tot += time.perf_counter() - t0
        done += 1
    value = psi.size * done / t_tot
    line = {
        "impl": "reference", "metric": "grid_cell_steps_per_s", "value": value, "unit": "cell-steps/s",
        "n_gpus": world, "steps": done, "steps_requested": args.steps, "warmup": min(args.warmup, 1),
        "ms_per_step": 1e3 * t_tot / done, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128", "data": "synthetic",
        "config": {"workload": args.workload, "grid": list(psi.shape[::-1]), "n_star": int(len(mass)), "dt": dt},
        "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": oracle.threads(), "kind": "oracle",
                         "sample": f"{done} oracle KDK steps of the workload (time-bounded at {budget:.0f} s)"},
        "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def ensemble_arm(args, r):
    """64 independent halos of uneven sizes stepped as one batch: the graph of per-member branches
    (the batch default, value = sum over members of cells x steps / time), and for comparison the
    persistent form (one cooperative launch per step: eight phases, each a work list of every
    member's tiles, with grid-wide barriers)."""
    import torch
    from paper_2606_25026_gb300 import inputs, spe
    rank, world, local = r.rank, r.world, r.local
    members = inputs.ensemble(count=args.members)
    stream = torch.cuda.Stream()
    b = spe.Batch([dict(nx=m["n"], G=1.0, max_particles=len(m["mass"])) for m in members], stream=stream)
    for g, m in zip(b.members, members):
        g.set_ic(m["psi"])
        if len(m["mass"]):
            g.add_particles(m["pos"], m["vel"], m["mass"])
    if not args.no_autotune:
        b.autotune()          # the graph form's strided tiles; the persistent form has its own
    dts = [m["dt"] for m in members]
    cells = sum(m["n"] ** 3 for m in members)
    stars = sum(len(m["mass"]) for m in members)
    # 112 B/cell without stars; with stars + 8 (Phi for the stars, rho_* for the density) and about
    # 100 B per star
    bytes_step = sum((120.0 if len(m["mass"]) else 112.0) * m["n"] ** 3 + 100.0 * len(m["mass"]) for m in members)
    peak, kind = measured_peak()

    def timed(persistent):
        b.set_persistent(persistent)
        b.step(max(args.warmup, 3), dts)
        l0 = b.launch_count()
        replicas.barrier(r)
        clocks = ClockSampler(local)
        clocks.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        b.step(args.steps, dts)
        b.settle()          # the members' closing half kicks, inside the timed region
        ev1.record(stream)
        ev1.synchronize()
        replicas.barrier(r)
        clk = clocks.stop()
        ms = replicas.max_over_ranks(r, ev0.elapsed_time(ev1), device="cuda")
        return ms, int(b.launch_count() - l0), clk, b.persistent()

    ms, launches, clk, _ = timed(False)
    ms_p, launches_p, clk_p, used_p = timed(True)
    ach = bytes_step * args.steps / (ms * 1e-3) / 1e9
    ach_p = bytes_step * args.steps / (ms_p * 1e-3) / 1e9
    line = {"metric": "grid_cell_steps_per_s", "value": replicas.job_rate(r, cells * args.steps, ms * 1e-3),
            "unit": "cell-steps/s", "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64", "data": "synthetic",
            "config": {"workload": "ensemble64", "members": len(members),
                       "sizes": {str(n): sum(1 for m in members if m["n"] == n) for n in (64, 96, 128, 192)},
                       "cells": cells, "stars": stars, "autotune": not args.no_autotune,
                       "launch": "graph of per-member branches (the batch default)"},
            "step_roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                              "model": "per member 112 B/cell/step without stars, 120 with, + 100 B per star"},
            "persistent": {"used": used_p, "value": replicas.job_rate(r, cells * args.steps, ms_p * 1e-3),
                           "ms_per_step": ms_p / args.steps, "frac": ach_p / peak, "gpu_launches": launches_p,
                           "clocks": clk_p, "speed_vs_graph_branches": ms / ms_p},
            "gpu_launches": launches, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    b.destroy()
    return 0


def fno_flops(n=64, C=32, M=16, H=64, L=4, fin=4):
    """Algorithmic FLOPs of one forward pass of the FNO on one n^3 sample (2 per multiply-add; a
    complex multiply-add counts 4): the lift with the first x DFT, per layer the y and z DFTs, the
    mode mixing, the z and y inverses and the row kernel (W v, the real x inverse, the next x
    DFT), and the projection."""
    cells = n ** 3
    spectral = 4 * (2 * n * n * M * M * C + 2 * n * M ** 3 * C + M ** 3 * C * C)
    row = cells * (C * C + 2 * M * C + 2 * M * C)
    last_row = cells * (C * C + 2 * M * C + C * H + H * 2)
    lift = cells * (C * fin + 2 * M * C)
    return 2.0 * (lift + (L - 1) * (spectral + row) + spectral + last_row)


def fno_bytes(kind, n=64, C=32, M=16, batch=1):
    """Algorithmic HBM bytes of one inference launch of an FNO kernel kind (BF16 activations,
    complex64 spectral buffers, BF16 weights)."""
    act = batch * n ** 3 * C * 2            # one BF16 activation tensor
    xrow = batch * n * n * M * C * 8        # x-stage buffer
    ystage = batch * n * M * M * C * 8      # y-stage buffer
    field = batch * n ** 3 * 8              # one complex64 field
    r = M ** 3 * C * C * 4                  # one layer's BF16 complex R
    return {"fno_lift": 2 * field + act + xrow, "fno_layer": 2 * act + 2 * xrow, "fno_last_layer": 2 * act + xrow,
            "fno_projection": act + 2 * field, "fno_y_dft": xrow + ystage, "fno_z_mix": 2 * ystage + r,
            "fno_y_idft": ystage + xrow}[kind]


def surrogate_arm(args, r):
    """The FNO surrogate against the plain solver on 64^3 halos: train on solver trajectories,
    then advance held-out grids by K = 16 steps through the judge (proposal accepted when its mass
    and energy drifts pass, spot-checked against the solver every 8th advance) and by the solver
    alone.  value = cell-steps/s of the surrogate path; plain.value the solver's."""
    import torch
    from paper_2606_25026_gb300 import inputs, spe, surrogate as sg
    rank, world, local = r.rank, r.world, r.local
    n, K = 64, 16
    specs = sg.ic_specs(args.fno_train + args.fno_test, seed=2026)
    ics = sg.make_ics(n, specs)
    dt = inputs.kinetic_dt(n)
    t0 = time.perf_counter()
    train = sg.generate_pairs(ics[:args.fno_train], n, K, dt, pairs_per_ic=2, warmup_steps=16)
    test = sg.generate_pairs(ics[args.fno_train:], n, K, dt, pairs_per_ic=1, warmup_steps=48)
    t_gen = time.perf_counter() - t0
    sigma = sg.correction_scale(train)
    inv_A = 1.0 / math.sqrt(0.95)
    net = spe.Fno(n=n, layers=4, modes=16, max_batch=8, train=True, inv_A=inv_A, sigma=sigma)
    net.set_params(inputs.fno_init_params(seed=0, out_gain=0.1))
    t0 = time.perf_counter()
    l_train0 = net.launch_count()
    hist = sg.train(net, train, epochs=args.fno_epochs, batch=8, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    e_coarse, e_prop = sg.evaluate(net, test)
    params = net.get_params()
    # per-kernel breakdown of one training step (forward, backward, Adam) at batch 8: a profiled
    # copy of the trained network on the first 8 pairs, 3 untimed and 20 timed steps
    pnet = spe.Fno(n=n, layers=4, modes=16, max_batch=8, train=True, profile=True, inv_A=inv_A, sigma=sigma)
    pnet.set_params(params)
    xb, bb, tb = (train.psi[:8].contiguous(), train.psi_b[:8].contiguous(), train.target[:8].contiguous())
    pout = torch.empty_like(xb)
    for _ in range(3):
        pnet.forward(xb, bb, out=pout)
        pnet.backward(tb)
        pnet.adam(lr=0.0)
    torch.cuda.synchronize()
    pnet.profile_read()
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record()
    for _ in range(20):
        pnet.forward(xb, bb, out=pout)
        pnet.backward(tb)
        pnet.adam(lr=0.0)
    pe1.record()
    pe1.synchronize()
    tprof = pnet.profile_read()
    ttot = sum(v[1] for v in tprof.values())
    train_step = {"ms": pe0.elapsed_time(pe1) / 20, "batch": 8,
                  "what": "forward, backward (tensor-core row kernels for BF16 activations) and Adam; "
                          "per-kind device time from events around each kind's launches",
                  "kernels": {k: {"launches_per_step": v[0] // 20, "ms_per_step": round(v[1] / 20, 4),
                                  "share": round(v[1] / ttot, 4)}
                              for k, v in sorted(tprof.items(), key=lambda kv: -kv[1][1])}}
    del train, net, pnet
    torch.cuda.empty_cache()

    inf = spe.Fno(n=n, layers=4, modes=16, max_batch=1, inv_A=inv_A, sigma=sigma)
    inf.set_params(params)
    g = spe.Grid(n, G=1.0)
    jc = dict(max_mass_drift=1e-5, max_energy_drift=1e-4, max_rel_l2=2e-5)
    sur = spe.Surrogate(g, inf, **jc)
    S = len(test)
    steps = max(1, min(args.steps, S))
    spot_every = 8
    # untimed pass: the error of what the surrogate path leaves on the grid, per held-out sample
    errs, verdicts = [], []
    for i in range(S):
        g.set_ic(test.psi[i])
        verdicts.append(sur.advance(g, K, dt, spot_check=(i % spot_every == 0)))
        got = torch.empty_like(test.psi[i])
        g.get_psi(out=got)
        torch.cuda.synchronize()
        errs.append(float(sg.rel_errors(got[None], test.target[i][None])[0]))
    accepted = [v for v in verdicts if v["accepted"]]
    spot = [v for v in verdicts if v["spot_checked"]]

    def run_plain(count):
        for i in range(count):
            g.set_ic(test.psi[i % S])
            g.step(K, dt)

    def run_surrogate(count):
        for i in range(count):
            g.set_ic(test.psi[i % S])
            sur.advance(g, K, dt, spot_check=(i % spot_every == 0))

    warm = max(args.warmup, 3)
    run_plain(warm)
    run_surrogate(warm)
    replicas.barrier(r)
    clocks = ClockSampler(local)
    clocks.start()
    t_plain = sg.timed(lambda: run_plain(steps), reps=1)
    replicas.barrier(r)
    sur.launch_count(reset=True)
    t_sur = sg.timed(lambda: run_surrogate(steps), reps=1)
    sur_launches = sur.launch_count()
    replicas.barrier(r)
    clk = clocks.stop()
    t_plain = replicas.max_over_ranks(r, t_plain, device="cuda")
    t_sur = replicas.max_over_ranks(r, t_sur, device="cuda")
    cells = n ** 3
    value = replicas.job_rate(r, cells * K * steps, t_sur)
    plain = replicas.job_rate(r, cells * K * steps, t_plain)

    # the forward pass alone (batch 1, graph replay), CUDA events on the network's stream
    x1, b1 = test.psi[:1].contiguous(), test.psi_b[:1].contiguous()
    o1 = torch.empty_like(x1)
    for _ in range(3):
        inf.forward(x1, b1, out=o1)
    st = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 50
    ev0.record(st)
    for _ in range(reps):
        inf.forward(x1, b1, out=o1)
    ev1.record(st)
    ev1.synchronize()
    fwd_s = ev0.elapsed_time(ev1) * 1e-3 / reps
    flops = fno_flops()
    # per-kernel CUDA events (profile mode launches directly, without the graph)
    pnet = spe.Fno(n=n, layers=4, modes=16, max_batch=1, inv_A=inv_A, sigma=sigma, profile=True)
    pnet.set_params(params)
    for _ in range(3):
        pnet.forward(x1, b1, out=o1)
    pnet.profile_read()
    for _ in range(reps):
        pnet.forward(x1, b1, out=o1)
    prof = pnet.profile_read()
    pnet.destroy()
    dom = max(prof, key=lambda k: prof[k][1])
    dom_launch_s = prof[dom][1] * 1e-3 / prof[dom][0]
    peak, peak_kind = measured_peak()
    dom_bytes = fno_bytes(dom)

    # e2e: the initial field from pinned host memory and the result back to it, every advance
    h_in = test.psi[:min(S, 16)].cpu().pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    ke = min(steps, 16)
    replicas.barrier(r)
    t0 = time.perf_counter()
    for i in range(ke):
        g.set_ic(h_in[i % len(h_in)])
        sur.advance(g, K, dt, spot_check=(i % spot_every == 0))
        g.get_psi(out=h_out[i % len(h_out)])
    replicas.barrier(r)
    t_e2e = replicas.max_over_ranks(r, time.perf_counter() - t0, device="cuda")

    line = {
        "metric": "grid_cell_steps_per_s", "value": value, "unit": "cell-steps/s", "n_gpus": world,
        "steps": steps, "warmup": warm, "ms_per_step": 1e3 * t_sur / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64 solver + bf16/fp32 network", "data": "synthetic",
        "config": {"workload": "fno64", "grid": [n, n, n], "K": K, "dt": dt,
                   "step": "one advance of one held-out grid by K solver steps (surrogate path)",
                   "train_trajectories": args.fno_train, "train_pairs": 2 * args.fno_train,
                   "held_out": S, "epochs": args.fno_epochs, "batch": 8, "judge": jc,
                   "spot_check_every": spot_every, "l2": "2 MB fields, launch-bound; no flush"},
        "plain": {"value": plain, "unit": "cell-steps/s", "ms_per_advance": 1e3 * t_plain / steps},
        "speedup_vs_plain": value / plain,
        "psi_error": {"vs": "solver K fine steps (FP32)", "surrogate_path_mean": float(np.mean(errs)),
                      "proposal_mean": float(e_prop.mean()), "coarse_step_mean": float(e_coarse.mean()),
                      "proposal_better_than_coarse": float(np.mean(e_prop < e_coarse))},
        "judge": {"accept_rate": len(accepted) / S, "spot_checked": len(spot),
                  "spot_rel_l2_mean": float(np.mean([v["rel_l2"] for v in spot])) if spot else None,
                  "mass_drift_max": float(max(v["mass_drift"] for v in verdicts)),
                  "energy_drift_max": float(max(v["energy_drift"] for v in verdicts))},
        "training": {"loss_first_epoch": hist[0], "loss_last_epoch": hist[-1], "seconds": t_train,
                     "pair_generation_s": t_gen, "sigma": sigma, "step": train_step},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": dom_bytes / dom_launch_s / 1e9, "peak": peak,
                     "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
                     else "fallback 6800 GB/s", "unit": "GB/s",
                     "frac": dom_bytes / dom_launch_s / 1e9 / peak, "traffic": None,
                     "bytes_per_launch": dom_bytes, "avg_launch_ms": dom_launch_s * 1e3,
                     "launches": prof[dom][0]},
        "fno_forward": {"ms": fwd_s * 1e3, "flops": flops, "tflops_fp32_equivalent": flops / fwd_s / 1e12,
                        "kernels": {k: {"launches": v[0], "ms_per_launch": round(v[1] / max(1, v[0]), 4),
                                        "GBs": round(fno_bytes(k) / (v[1] * 1e-3 / max(1, v[0])) / 1e9, 1)}
                                    for k, v in prof.items()}},
        "gpu_launches": int(sur_launches),
        "clocks": clk,
        "e2e": {"value": replicas.job_rate(r, cells * K * ke, t_e2e), "unit": "cell-steps/s", "steps": ke,
                "h2d_bytes_per_step": cells * 8, "d2h_bytes_per_step": cells * 8,
                "what": "pinned-host upload of each held-out field, the judged advance, download of the result"},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        psi0 = test.psi[0].cpu().numpy()
        z = np.zeros((0, 3), np.float32)
        v, cores, sec, nsteps = cpu_baseline(psi0, z, z, np.zeros(0, np.float32), dt)[:4]
        line["cpu_baseline"] = {"value": v, "unit": "cell-steps/s", "cores": cores, "kind": "oracle",
                                "sample": f"{nsteps} plain KDK steps of one held-out 64^3 field ({sec:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    sur.destroy()
    return 0


def power_spectrum(rho, shells=16):
    """P(k) of the density contrast rho / <rho> - 1 in integer shells |m| = 1 .. shells - 1
    (k = 2 pi m / L)."""
    d = np.fft.fftn(rho / rho.mean() - 1.0)
    nz, ny, nx = rho.shape
    mz, my, mx = np.meshgrid(np.fft.fftfreq(nz) * nz, np.fft.fftfreq(ny) * ny, np.fft.fftfreq(nx) * nx,
                             indexing="ij", sparse=True)
    shell = np.rint(np.sqrt(mx ** 2 + my ** 2 + mz ** 2)).astype(np.int64)
    p = np.bincount(shell.ravel(), weights=(np.abs(d) ** 2).ravel(), minlength=shells)
    c = np.bincount(shell.ravel(), minlength=shells)
    return p[1:shells] / c[1:shells]


def precision_arm(args, r):
    """The precision study on one 512^3 grid of the halo family (no stars): the FP32 Stockham path
    and the split-FP16 tensor-core path against the FP64 oracle, the same initial state and dt,
    200 steps (--steps), errors at every quarter of the run: relative L2 of psi, mass and energy
    drift, and the largest relative error of the density power spectrum in shells 1..15.  The
    oracle takes about 8 s per step on 16 host cores."""
    import torch
    from paper_2606_25026_gb300 import spe
    import oracle
    if r.rank != 0:
        return 0
    psi, _, _, _, dt = make_inputs("halo512", args.grid)
    nz, ny, nx = psi.shape
    total = args.steps
    marks = sorted({max(1, total * q // 4) for q in (1, 2, 3, 4)})
    stream = torch.cuda.Stream()
    arms = {}
    snaps = {}
    for name, flag in (("fp32", 0), ("split16", spe.SPE_PREC_SPLIT16)):
        g = spe.Grid(nx, ny, nz, L=1.0, G=1.0, flags=flag, stream=stream)
        if not args.no_autotune and flag == 0:
            g.autotune()
        g.set_ic(torch.from_numpy(psi).cuda())
        e0 = g.energy()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        done, ms = 0, 0.0
        snaps[name] = {}
        en = {}
        for mk in marks:
            ev0.record(stream)
            g.step(mk - done, dt)
            g.settle()
            ev1.record(stream)
            ev1.synchronize()
            ms += ev0.elapsed_time(ev1)
            done = mk
            snaps[name][mk] = g.get_psi()
            en[mk] = g.energy()
        arms[name] = {"cell_steps_per_s": psi.size * total / (ms * 1e-3), "ms_per_step": ms / total,
                      "e0": e0, "energies": en}
        g.destroy()
        del g
        torch.cuda.empty_cache()
        print(f"precision512: {name} done, {ms / total:.3f} ms/step", file=sys.stderr, flush=True)
    oracle.build()
    o = oracle.Oracle(nx, ny, nz, 1.0, G=1.0)
    o.set_ic(psi.astype(np.complex128))
    o.potential()
    eo0 = o.energy()
    t0 = time.perf_counter()
    done = 0
    out = {name: {} for name in arms}
    out["fp64"] = {}
    for mk in marks:
        o.step(mk - done, dt)
        done = mk
        ref = o.get_psi()
        eo = o.energy()
        pk_ref = power_spectrum(np.abs(ref) ** 2)
        nref = np.linalg.norm(ref)
        out["fp64"][str(mk)] = {"mass_drift": abs(eo["mass"] - eo0["mass"]) / eo0["mass"],
                                "energy_drift": abs(eo["total"] - eo0["total"]) / abs(eo0["total"])}
        for name, a in arms.items():
            got = snaps[name].pop(mk).astype(np.complex128)
            eg = a["energies"][mk]
            pk = power_spectrum(np.abs(got) ** 2)
            out[name][str(mk)] = {
                "psi_rel_l2": float(np.linalg.norm(got - ref) / nref),
                "mass_drift": abs(eg["mass"] - a["e0"]["mass"]) / a["e0"]["mass"],
                "energy_drift": abs(eg["total"] - a["e0"]["total"]) / abs(a["e0"]["total"]),
                "pk_max_rel_err": float(np.max(np.abs(pk - pk_ref) / pk_ref))}
            del got
        del ref
        print(f"precision512: oracle at step {mk} ({time.perf_counter() - t0:.0f} s)", file=sys.stderr, flush=True)
    sec = time.perf_counter() - t0
    line = {"metric": "grid_cell_steps_per_s", "value": arms["fp32"]["cell_steps_per_s"], "unit": "cell-steps/s",
            "n_gpus": 1, "steps": total, "warmup": 0, "ms_per_step": arms["fp32"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "precision512", "grid": [nx, ny, nz], "dt": dt, "checkpoints": marks},
            "split16": {"value": arms["split16"]["cell_steps_per_s"],
                        "speedup_vs_fp32": arms["split16"]["cell_steps_per_s"] / arms["fp32"]["cell_steps_per_s"]},
            "errors_vs_fp64": out,
            "cpu_baseline": {"value": psi.size * total / sec, "unit": "cell-steps/s", "cores": oracle.threads(),
                             "kind": "oracle", "sample": f"{total} KDK steps of the 512^3 grid ({sec:.0f} s)"}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    r = replicas.from_env()
    if args.impl == "reference":
        return reference_arm(args, r.rank, r.world)

    import torch
    from paper_2606_25026_gb300 import build as spe_build
    # the leader compiles; the other ranks find the library up to date after the first barrier
    if r.leader:
        spe_build.build()
    replicas.init(r, "nccl", torch.device("cuda", r.local))
    spe_build.build()
    torch.cuda.set_device(r.local)
    try:
        if args.workload == "ensemble64":
            return ensemble_arm(args, r)
        if args.workload == "fno64":
            return surrogate_arm(args, r)
        if args.workload == "precision512":
            return precision_arm(args, r)
        return grid_arm(args, r)
    finally:
        replicas.finish(r)


def grid_line(args, r, workload, grid_spec=None, steps=None, warmup=None, e2e=True, cpu=True,
              oracle_budget_s=45.0):
    """Measure one grid workload; returns the JSON line's fields (device-resident value, roofline,
    kernel split, e2e, CPU oracle baseline and psi error vs FP64)."""
    import torch
    from paper_2606_25026_gb300 import spe
    rank, world, local = r.rank, r.world, r.local
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup

    psi, pos, vel, mass, dt = make_inputs(workload, grid_spec)
    nz, ny, nx = psi.shape
    ncells = psi.size
    nstar = len(mass)
    stream = torch.cuda.Stream()

    def barrier():
        replicas.barrier(r)

    # ---------------- device-resident timed region (the production path: every step after a call's
    # first one is a CUDA graph replay; no per-kernel events)
    prec_flag = (spe.SPE_PREC_SPLIT16 if args.prec == "split16" else 0) | (spe.SPE_NO_TMA if args.no_tma else 0)

    def make_grid(flags):
        grid = spe.Grid(nx, ny, nz, L=1.0, G=1.0, max_particles=nstar, flags=flags | prec_flag, stream=stream)
        grid.set_ic(torch.from_numpy(psi).cuda())
        if nstar:
            grid.add_particles(torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda(),
                               torch.from_numpy(mass).cuda())
        return grid

    def timed_steps(grid, k):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        grid.step(k, dt)
        grid.settle()          # the closing half kick of the last step, inside the timed region
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1)

    g = make_grid(spe.SPE_ASYNC)
    if args.tiles or args.plans:
        pin_t = tuple(int(v) for v in (args.tiles or "0,0").split(","))
        pin_p = tuple(int(v) for v in (args.plans or "0,0").split(","))
        g.set_schedule(pin_t, pin_p)
        tiles = pin_t
    else:
        tiles = g.autotune() if not args.no_autotune else None
    schedule = g.schedule()
    schedule_half = g.schedule_half()

    def same_schedule(other):
        # the timed grid's schedule on another grid of the same shape: pinned as given, or the
        # autotuner's cached choices (psi's and the half spectrum's), which re-applies them untimed
        if args.tiles or args.plans:
            other.set_schedule(pin_t, pin_p)
        else:
            other.autotune()
    g.step(warmup, dt)
    g.sync()
    g.launch_count(reset=True)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ms = timed_steps(g, steps)
    barrier()
    clk = clocks.stop()
    launches = g.launch_count()
    ms = replicas.max_over_ranks(r, ms, device="cuda")
    value = replicas.job_rate(r, ncells * steps, ms * 1e-3)
    g.destroy()
    del g
    torch.cuda.empty_cache()

    # ---------------- the same steps with CUDA events around every kernel launch (direct launches,
    # no graphs): per-kernel durations for the roofline and the kernel split
    gp = make_grid(spe.SPE_ASYNC | spe.SPE_PROFILE)
    if tiles is not None:
        same_schedule(gp)
    gp.step(warmup, dt)
    gp.sync()
    gp.profile_read()
    # an NVTX range around these steps lets a profiler pick out their launches
    torch.cuda.nvtx.range_push("spe_timed_steps")
    ms_prof = timed_steps(gp, steps)
    torch.cuda.nvtx.range_pop()
    prof = gp.profile_read()
    workspace_mib = gp.workspace.numel() / 2 ** 20
    gp.destroy()
    del gp
    torch.cuda.empty_cache()

    # roofline of the dominant kernel on the per-pass byte model
    bpc = MODEL_BYTES_STARS if nstar else MODEL_BYTES
    dom = max((k for k in prof if k in bpc), key=lambda k: prof[k][1])
    n_launch, dom_ms = prof[dom]
    per_launch_s = dom_ms * 1e-3 / max(n_launch, 1)
    peak, peak_kind = measured_peak()
    achieved = bpc[dom] * ncells / per_launch_s / 1e9
    traffic = recorded_traffic(dom, workload if grid_spec is None else f"{workload}@{grid_spec}")
    # x kick pass, y fwd, z drift, y inv, x density pass, and the three half-spectrum passes
    step_bytes = (bpc["x_kick_fwd"] + 2 * bpc["y_fft_psi"] + bpc["z_fft_drift"] + bpc["x_inv_density_r2c"] +
                  2 * bpc["y_fft_rho"] + bpc["z_fft_poisson"])
    step_total = step_bytes * ncells + MODEL_BYTES_PER_STAR * nstar
    step_gbs = step_total * steps / (ms * 1e-3) / 1e9
    kernel_split = {k: {"launches": v[0], "ms": round(v[1], 4),
                        "us_per_launch": round(1e3 * v[1] / max(1, v[0]), 2),
                        "share": round(v[1] / max(1e-9, sum(x[1] for x in prof.values())), 4)}
                    for k, v in prof.items() if v[0]}
    for k, v in kernel_split.items():
        if k in bpc:
            v["frac_hbm"] = round(bpc[k] * ncells / (v["us_per_launch"] * 1e-6) / 1e9 / peak, 4)

    line = {
        "metric": "grid_cell_steps_per_s", "value": value, "unit": "cell-steps/s", "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": {"workload": workload, "grid": [nx, ny, nz], "n_star": nstar, "dt": dt,
                   "precision": args.prec, "tile_staging": "cp.async" if args.no_tma else "tma",
                   "strided_schedule_yz": {"tiles": list(schedule[0]),
                                                                   "alt_radix_plan": list(schedule[1]),
                                                                   "half_spectrum_tiles": list(schedule_half[0]),
                                                                   "half_spectrum_radix_plan": list(schedule_half[1]),
                                                                   "autotuned": tiles is not None and
                                                                   not (args.tiles or args.plans)},
                   "l2": f"working set {workspace_mib:.0f} MiB > 129 MB L2 (no flush needed)",
                   "parallelism": f"{world} independent replica(s)"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
                     else "fallback 6800 GB/s", "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "bytes_per_cell": bpc[dom], "launches": n_launch,
                     "avg_launch_ms": per_launch_s * 1e3,
                     "model": "per-pass algorithmic bytes of the fused axis-pass schedule"},
        "step_roofline": {"bytes_per_cell_step": step_bytes, "bytes_per_star_step": MODEL_BYTES_PER_STAR,
                          "achieved_GBs": step_gbs, "frac": step_gbs / peak,
                          # against the 64 B/cell/step floor of two-pass 3D transforms with every
                          # pointwise operation fused
                          "frac_vs_64B_floor": 64.0 * ncells * steps / (ms * 1e-3) / 1e9 / peak},
        "kernel_timing": {"what": "per-kernel CUDA events in a second run of the same steps with direct "
                                  "launches (no graphs); value above is the graph-replayed run",
                          "ms_per_step": ms_prof / steps},
        "kernels": kernel_split,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if nstar:
        # the implementation's own accounting of the density pass (int64 deposit read and cleared
        # on the marked rows), beside the model's
        frows = deposit_row_fraction(pos, psi.shape)
        impl_b = 20.0 + 16.0 * frows
        d_ms = prof.get("x_inv_density_r2c", (0, 0.0))
        if d_ms[0]:
            s_ = d_ms[1] * 1e-3 / d_ms[0]
            line["roofline_impl_accounting"] = {
                "kernel": "x_inv_density_r2c", "bytes_per_cell": impl_b, "deposit_row_fraction": frows,
                "achieved": impl_b * ncells / s_ / 1e9, "frac": impl_b * ncells / s_ / 1e9 / peak}

    # ---------------- end to end through the C ABI with host buffers
    if e2e:
        h_psi = torch.from_numpy(psi).pin_memory()
        h_pos = torch.from_numpy(pos).pin_memory()
        h_vel = torch.from_numpy(vel).pin_memory()
        h_mass = torch.from_numpy(mass).pin_memory()
        o_psi = torch.empty(psi.shape, dtype=torch.complex64).pin_memory()
        ge = spe.Grid(nx, ny, nz, L=1.0, G=1.0, max_particles=nstar, flags=prec_flag | spe.SPE_ASYNC, stream=stream)
        if tiles is not None:
            same_schedule(ge)
        ke = max(1, min(steps, 200))
        h_mass_out = torch.zeros(ke, dtype=torch.float64).pin_memory()
        # warm the path once
        ge.set_ic(h_psi)
        if nstar:
            ge.add_particles(h_pos, h_vel, h_mass)
        ge.step(2, dt)
        ge.mass_async(h_mass_out[:1])
        ge.sync()
        barrier()
        t0 = time.perf_counter()
        ge.set_ic(h_psi)
        ge.clear_particles()
        if nstar:
            ge.add_particles(h_pos, h_vel, h_mass)
        for k in range(ke):
            ge.step(1, dt)
            ge.mass_async(h_mass_out[k:k + 1])
        ge.get_psi(o_psi)
        if nstar:
            ge.get_particles()
        barrier()
        sec = time.perf_counter() - t0
        masses = h_mass_out.numpy()
        if not (np.isfinite(masses).all() and np.abs(masses / masses[0] - 1.0).max() < 1e-5):
            raise RuntimeError(f"per-step masses read back in the e2e loop are off: {masses[:4]} ...")
        sec = replicas.max_over_ranks(r, sec, device="cuda")
        h2d = psi.nbytes + pos.nbytes + vel.nbytes + mass.nbytes
        d2h = ke * 8 + psi.nbytes + pos.nbytes + vel.nbytes
        line["e2e"] = {"value": replicas.job_rate(r, ncells * ke, sec), "unit": "cell-steps/s", "steps": ke,
                       "h2d_bytes_per_step": h2d / ke, "d2h_bytes_per_step": d2h / ke,
                       "what": "pinned-host upload of psi (and stars); single-step SPE_ASYNC spe_step calls, "
                               "each followed by a device->host copy of that step's mass into pinned memory "
                               "(spe_mass_async, checked after the loop); final download of psi (and stars)"}
        ge.destroy()
        del ge
        torch.cuda.empty_cache()

    # ---------------- CPU oracle baseline and the psi error vs FP64 over the oracle's steps
    # (rank 0, N = 1): the oracle runs a time-bounded number of steps (at least two) from the
    # initial state, the GPU the same number from the same state
    if cpu and rank == 0 and world == 1:
        v, cores, sec, nsteps, last, e0, e1 = cpu_baseline(psi, pos, vel, mass, dt, budget_s=oracle_budget_s,
                                                           max_steps=max(2, min(steps, 50)), min_steps=2)
        line["cpu_baseline"] = {"value": v, "unit": "cell-steps/s", "cores": cores, "kind": "oracle",
                                "sample": f"{nsteps} KDK steps of the {workload} workload ({sec:.1f} s), "
                                          "Phi(0) solve untimed"}
        gc = spe.Grid(nx, ny, nz, L=1.0, G=1.0, max_particles=nstar, flags=prec_flag, stream=stream)
        if tiles is not None:
            same_schedule(gc)
        gc.set_ic(psi)
        if nstar:
            gc.add_particles(pos, vel, mass)
        eg0 = gc.energy()
        gc.step(nsteps, dt)
        eg1 = gc.energy()
        ref, op = last
        got = gc.get_psi()
        err = {"steps": nsteps, "rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
               "bar": 1e-5,
               "mass_drift_gpu": abs(eg1["mass"] - eg0["mass"]) / eg0["mass"],
               "energy_drift_gpu": abs(eg1["total"] - eg0["total"]) / abs(eg0["total"]),
               "mass_drift_fp64": abs(e1["mass"] - e0["mass"]) / e0["mass"],
               "energy_drift_fp64": abs(e1["total"] - e0["total"]) / abs(e0["total"])}
        if nstar:
            gpos, _ = gc.get_particles()
            d = (gpos - op + 0.5) % 1.0 - 0.5
            err["star_pos_max_box"] = float(np.abs(d).max())
        line["psi_error"] = err
        gc.destroy()
        del gc
        torch.cuda.empty_cache()
    return line


def grid_arm(args, r):
    line = grid_line(args, r, args.workload, args.grid, e2e=not args.no_e2e, cpu=not args.no_cpu_baseline,
                     oracle_budget_s=45.0 if args.workload == "halo512" else 12.0)
    if args.workload == "halo512" and args.grid is None and not args.no_nested:
        # the 256^3 grid with 1e6 stars: the field and the star coupling together
        sub = grid_line(args, r, "halo256_stars1e6", None, steps=min(max(args.steps, 100), 1000),
                        e2e=False, cpu=not args.no_cpu_baseline, oracle_budget_s=12.0)
        keep = ("value", "unit", "steps", "ms_per_step", "config", "roofline", "roofline_impl_accounting",
                "step_roofline", "kernel_timing", "kernels", "gpu_launches", "clocks", "cpu_baseline",
                "psi_error")
        line["halo256_stars1e6"] = {k: sub[k] for k in keep if k in sub}
    if r.rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
