"""Benchmark: split-step Schroedinger-Poisson grid-cell-steps/s on GB300.

Workload (default): 256^3 complex64 grid, central soliton + granular halo, 1e6 Plummer stars
(5% of the mass), CIC coupling, dt from the Sec. 3.5 kinetic CFL term.  One "step" is one full
kick-drift-kick step of the field and the stars (every kernel of the hot path).

Prints one JSON line (rank 0).  ``value`` is device-resident throughput (inputs already in HBM,
CUDA events on the grid's stream, K steps in one spe_step call: every step after the first is a
CUDA graph replay).  ``e2e`` is the same metric through
the C ABI with host buffers: pinned-host upload of the initial field and stars, K single-step calls
each followed by a device->host read of the step's mass, and the final download of psi and the
stars, all inside the timed region.  ``roofline`` is the dominant kernel's algorithmic bytes over
its CUDA-event duration, taken in a second run of the same K steps with events around every
(direct) launch, against the measured HBM copy bandwidth.  ``cpu_baseline`` is the FP64
oracle on the host cores on about ten seconds of steps of the same workload.

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

# Algorithmic HBM bytes per grid cell for one launch of each kernel kind, with stars (the
# fused axis-pass schedule): reads + writes that the step cannot avoid at that pass.
#   x_kick_fwd        : R psi 8 + R Phi_hat 4 + W psi 8 + W Phi 4           = 24
#   y_fft_psi         : R 8 + W 8                                           = 16
#   z_fft_drift       : R 8 + W 8                                           = 16
#   x_inv_density_r2c : R psi_hat 8 + R deposit 8 + W deposit 8 (clear) + W psi 8 + W rho_hat 4 = 36,
#                       the deposit's 16 only on rows (y, z) that hold stars' mass: 20 + 16 f, f the
#                       fraction of such rows (deposit_row_fraction), 36 at f = 1
#   y_fft_rho, z_fft_poisson : R 4 + W 4 (half spectrum)                    = 8
#   x_kick_final      : R psi 8 + R Phi_hat 4 + W psi 8 + W Phi 4           = 24
BYTES_PER_CELL = {
    "x_kick_fwd": 24.0, "y_fft_psi": 16.0, "z_fft_drift": 16.0, "x_inv_density_r2c": 36.0,
    "y_fft_rho": 8.0, "z_fft_poisson": 8.0, "x_kick_final": 24.0,
}
BYTES_PER_CELL_NO_STARS = dict(BYTES_PER_CELL, x_kick_fwd=20.0, x_inv_density_r2c=20.0, x_kick_final=20.0)
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
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="halo256_stars1e6",
                    choices=["halo256_stars1e6", "halo512", "packets32", "ensemble64", "fno64"])
    ap.add_argument("--fno-epochs", type=int, default=8, help="fno64: training epochs over the pairs")
    ap.add_argument("--fno-train", type=int, default=2000, help="fno64: training trajectories")
    ap.add_argument("--fno-test", type=int, default=200, help="fno64: held-out trajectories")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--grid", default=None,
                    help="NXxNYxNZ: run the workload's initial-condition family on this grid instead "
                         "(profiling cases; the stars keep their count)")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "split16"],
                    help="split16: radix-16 DFT stages of 256/512-point axes on the tensor cores")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
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

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

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
        sm = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def make_inputs(workload, grid=None):
    from paper_2606_25026_gb300 import inputs
    n = tuple(int(v) for v in grid.lower().split("x")) if grid else None
    psi, pos, vel, mass, dt, _ = inputs.make_workload(workload, n=n)
    return (psi.astype(np.complex64), pos.astype(np.float32), vel.astype(np.float32), mass.astype(np.float32),
            float(dt))


def cpu_baseline(psi, pos, vel, mass, dt, budget_s=10.0, max_steps=20):
    """The FP64 oracle on the host cores: KDK steps of the same workload, one at a time until
    about budget_s seconds of CPU work (the Phi(0) solve before them is not timed).  Returns
    (cell-steps/s, threads, seconds, steps, the oracle state after its first step)."""
    import oracle
    oracle.build()
    nz, ny, nx = psi.shape
    o = oracle.Oracle(nx, ny, nz, 1.0, G=1.0)
    o.set_ic(psi.astype(np.complex128))
    if len(mass):
        o.set_particles(pos.astype(np.float64), vel.astype(np.float64), mass.astype(np.float64))
    o.potential()
    sec, steps, first = 0.0, 0, None
    while steps < max_steps and (steps == 0 or sec < budget_s):
        t0 = time.perf_counter()
        o.step(1, dt)
        sec += time.perf_counter() - t0
        steps += 1
        if first is None:
            first = (o.get_psi(), o.get_particles()[0] if len(mass) else None)
    return psi.size * steps / sec, oracle.threads(), sec, steps, first


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
    """64 independent halos of uneven sizes stepped as one batch (a CUDA graph with a branch per
    member); value = sum over members of cells x steps / time."""
    import torch
    from paper_2606_25026_gb300 import inputs, spe
    rank, world, local = r.rank, r.world, r.local
    members = inputs.ensemble()
    stream = torch.cuda.Stream()
    b = spe.Batch([dict(nx=m["n"], G=1.0, max_particles=len(m["mass"])) for m in members], stream=stream)
    for g, m in zip(b.members, members):
        g.set_ic(m["psi"])
        if len(m["mass"]):
            g.add_particles(m["pos"], m["vel"], m["mass"])
    if not args.no_autotune:
        b.autotune()
    dts = [m["dt"] for m in members]
    b.step(max(args.warmup, 3), dts)
    cells = sum(m["n"] ** 3 for m in members)
    stars = sum(len(m["mass"]) for m in members)
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
    # 112 B/cell without stars; with stars + 4 (Phi for the stars) + 16 f (the deposit's rows)
    bytes_step = sum(((116.0 + 16.0 * deposit_row_fraction(m["pos"], (m["n"],) * 3)) if len(m["mass"]) else 112.0)
                     * m["n"] ** 3 for m in members)
    peak, kind = measured_peak()
    ach = bytes_step * args.steps / (ms * 1e-3) / 1e9
    line = {"metric": "grid_cell_steps_per_s", "value": replicas.job_rate(r, cells * args.steps, ms * 1e-3),
            "unit": "cell-steps/s", "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64", "data": "synthetic",
            "config": {"workload": "ensemble64", "members": len(members),
                       "sizes": {str(n): sum(1 for m in members if m["n"] == n) for n in (64, 96, 128, 192)},
                       "cells": cells, "stars": stars, "autotune": not args.no_autotune},
            "step_roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                              "model": "per member 112 B/cell/step without stars, 116 + 16 f with (f the "
                                       "fraction of rows holding deposits)"},
            "gpu_launches": int(b.launch_count() - l0), "clocks": clk}
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
    del train, net
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
                     "pair_generation_s": t_gen, "sigma": sigma},
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
        v, cores, sec, nsteps, _ = cpu_baseline(psi0, z, z, np.zeros(0, np.float32), dt)
        line["cpu_baseline"] = {"value": v, "unit": "cell-steps/s", "cores": cores, "kind": "oracle",
                                "sample": f"{nsteps} plain KDK steps of one held-out 64^3 field ({sec:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    sur.destroy()
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
        return grid_arm(args, r)
    finally:
        replicas.finish(r)


def grid_arm(args, r):
    import torch
    from paper_2606_25026_gb300 import spe
    rank, world, local = r.rank, r.world, r.local

    psi, pos, vel, mass, dt = make_inputs(args.workload, args.grid)
    nz, ny, nx = psi.shape
    ncells = psi.size
    nstar = len(mass)
    stream = torch.cuda.Stream()

    def barrier():
        replicas.barrier(r)

    # ---------------- device-resident timed region (the production path: every step after a call's
    # first one is a CUDA graph replay; no per-kernel events)
    prec_flag = spe.SPE_PREC_SPLIT16 if args.prec == "split16" else 0

    def make_grid(flags):
        grid = spe.Grid(nx, ny, nz, L=1.0, G=1.0, max_particles=nstar, flags=flags | prec_flag, stream=stream)
        grid.set_ic(torch.from_numpy(psi).cuda())
        if nstar:
            grid.add_particles(torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda(),
                               torch.from_numpy(mass).cuda())
        return grid

    def timed_steps(grid, steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        grid.step(steps, dt)
        grid.settle()          # the closing half kick of the last step, inside the timed region
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1)

    g = make_grid(spe.SPE_ASYNC)
    tiles = g.autotune() if not args.no_autotune else None
    schedule = g.schedule()
    g.step(args.warmup, dt)
    g.sync()
    g.launch_count(reset=True)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ms = timed_steps(g, args.steps)
    barrier()
    clk = clocks.stop()
    launches = g.launch_count()
    ms = replicas.max_over_ranks(r, ms, device="cuda")
    value = replicas.job_rate(r, ncells * args.steps, ms * 1e-3)
    g.destroy()
    del g
    torch.cuda.empty_cache()

    # ---------------- the same steps with CUDA events around every kernel launch (direct launches,
    # no graphs): per-kernel durations for the roofline and the kernel split
    gp = make_grid(spe.SPE_ASYNC | spe.SPE_PROFILE)
    if tiles is not None:
        gp.set_schedule(*schedule)
    gp.step(args.warmup, dt)
    gp.sync()
    gp.profile_read()
    ms_prof = timed_steps(gp, args.steps)
    prof = gp.profile_read()

    # roofline of the dominant kernel
    frows = deposit_row_fraction(pos, psi.shape) if nstar else 0.0
    bpc = dict(BYTES_PER_CELL, x_inv_density_r2c=20.0 + 16.0 * frows) if nstar else BYTES_PER_CELL_NO_STARS
    dom = max((k for k in prof if k in bpc), key=lambda k: prof[k][1])
    n_launch, dom_ms = prof[dom]
    per_launch_s = dom_ms * 1e-3 / max(n_launch, 1)
    alg_bytes = bpc[dom] * ncells
    peak, peak_kind = measured_peak()
    achieved = alg_bytes / per_launch_s / 1e9
    traffic = recorded_traffic(dom, args.workload)
    # x kick pass, y fwd, z drift, y inv, x density pass, and the three half-spectrum passes
    step_bytes = (bpc["x_kick_fwd"] + 2 * bpc["y_fft_psi"] + bpc["z_fft_drift"] + bpc["x_inv_density_r2c"] +
                  2 * bpc["y_fft_rho"] + bpc["z_fft_poisson"])
    # DRAM bytes of one step from the committed ncu capture (null unless taken on these sources)
    per_step = {"x_kick_fwd": 1, "x_inv_density_r2c": 1, "y_fft_psi": 2, "z_fft_drift": 1, "y_fft_rho": 2,
                "z_fft_poisson": 1}
    if nstar:
        per_step["particles_kdk_deposit"] = 1
    rec = {k: recorded_traffic(k, args.workload) for k in per_step}
    step_dram = sum(rec[k] * c for k, c in per_step.items()) if all(v is not None for v in rec.values()) else None
    kernel_split = {k: {"launches": v[0], "ms": round(v[1], 4), "share": round(v[1] / max(1e-9, sum(
        x[1] for x in prof.values())), 4)} for k, v in prof.items() if v[0]}

    line = {
        "metric": "grid_cell_steps_per_s", "value": value, "unit": "cell-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": {"workload": args.workload, "grid": [nx, ny, nz], "n_star": nstar, "dt": dt,
                   "precision": args.prec, "strided_schedule_yz": {"tiles": list(schedule[0]),
                                                                   "alt_radix_plan": list(schedule[1]),
                                                                   "autotuned": tiles is not None},
                   "l2": f"working set {gp.workspace.numel() / 2**20:.0f} MiB > 129 MB L2 (no flush needed)",
                   "parallelism": f"{world} independent replica(s)"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
                     else "fallback 6800 GB/s", "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "bytes_per_cell": bpc[dom], "deposit_row_fraction": frows,
                     "launches": n_launch,
                     "avg_launch_ms": per_launch_s * 1e3},
        "step_roofline": {"bytes_per_cell_step": step_bytes,
                          "achieved_GBs": step_bytes * ncells * args.steps / (ms * 1e-3) / 1e9,
                          "frac": step_bytes * ncells * args.steps / (ms * 1e-3) / 1e9 / peak,
                          # against the 64 B/cell/step floor of two-pass 3D transforms with every
                          # pointwise operation fused
                          "frac_vs_64B_floor": 64.0 * ncells * args.steps / (ms * 1e-3) / 1e9 / peak,
                          "dram_bytes_per_step_measured": step_dram,
                          "frac_measured_dram": (step_dram * args.steps / (ms * 1e-3) / 1e9 / peak
                                                 if step_dram else None)},
        "kernel_timing": {"what": "per-kernel CUDA events in a second run of the same steps with direct "
                                  "launches (no graphs); value above is the graph-replayed run",
                          "ms_per_step": ms_prof / args.steps},
        "kernels": kernel_split,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    gp.destroy()
    del gp
    torch.cuda.empty_cache()

    # ---------------- end to end through the C ABI with host buffers
    if not args.no_e2e:
        h_psi = torch.from_numpy(psi).pin_memory()
        h_pos = torch.from_numpy(pos).pin_memory()
        h_vel = torch.from_numpy(vel).pin_memory()
        h_mass = torch.from_numpy(mass).pin_memory()
        o_psi = torch.empty(psi.shape, dtype=torch.complex64).pin_memory()
        ge = spe.Grid(nx, ny, nz, L=1.0, G=1.0, max_particles=nstar, flags=prec_flag | spe.SPE_ASYNC, stream=stream)
        if not args.no_autotune:
            ge.autotune()
        ke = max(1, min(args.steps, 200))
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
                       "what": "pinned-host upload of psi and stars; single-step SPE_ASYNC spe_step calls, each "
                               "followed by a device->host copy of that step's mass into pinned memory "
                               "(spe_mass_async, checked after the loop); final download of psi and stars"}
        ge.destroy()
        del ge

    # ---------------- CPU oracle baseline and the stated psi error vs FP64 (rank 0, N = 1)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sec, nsteps, first = cpu_baseline(psi, pos, vel, mass, dt)
        line["cpu_baseline"] = {"value": v, "unit": "cell-steps/s", "cores": cores, "kind": "oracle",
                                "sample": f"{nsteps} KDK steps of the {args.workload} workload ({sec:.1f} s), "
                                          "Phi(0) solve untimed"}
        gc = spe.Grid(nx, ny, nz, L=1.0, G=1.0, max_particles=nstar, flags=prec_flag, stream=stream)
        gc.set_ic(psi)
        if nstar:
            gc.add_particles(pos, vel, mass)
        gc.step(1, dt)
        ref, op = first
        got = gc.get_psi()
        line["psi_rel_l2_vs_fp64_1step"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        if nstar:
            gp, _ = gc.get_particles()
            d = (gp - op + 0.5) % 1.0 - 0.5
            line["pos_err_vs_fp64_1step_box"] = float(np.abs(d).max())
        gc.destroy()

    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
