"""Training and evaluation of the FNO surrogate on trajectories the solver generates.

Orchestration only: every field operation runs in libspe (the solver's kernels make the
trajectories and the coarse steps, the network's kernels do forward, backward and Adam);
PyTorch holds the device tensors.  The pairs are (psi_t, psi_b, psi_{t+K dt}) with psi_b one
solver step of length K dt from psi_t, kept resident in device memory.
"""
from __future__ import annotations

import math
import multiprocessing as mp
import time
from dataclasses import dataclass

import numpy as np

from . import inputs
from . import spe


@dataclass
class PairSet:
    psi: "torch.Tensor"       # (S, n, n, n) complex64 on the device
    psi_b: "torch.Tensor"
    target: "torch.Tensor"
    dt: float
    K: int

    def __len__(self):
        return int(self.psi.shape[0])


def ic_specs(count, seed=0, rc_range=(0.03, 0.08)):
    """(seed, r_c) of each soliton + granule initial condition of a seeded family."""
    rng = np.random.default_rng(seed)
    return [(int(seed * 100_003 + i), float(rng.uniform(*rc_range))) for i in range(count)]


def _make_ic(args):
    n, s, rc = args
    return inputs.soliton_halo(n, r_c=rc, seed=s)


def make_ics(n, specs, workers=None):
    """Initial conditions on the host, built in a spawned process pool (safe after CUDA use)."""
    jobs = [(n, s, rc) for s, rc in specs]
    workers = workers or min(16, mp.cpu_count())
    if workers <= 1 or len(jobs) < 4:
        return [_make_ic(j) for j in jobs]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_make_ic, jobs, chunksize=max(1, len(jobs) // (4 * workers)))


def generate_pairs(ics, n, K, dt, pairs_per_ic=1, warmup_steps=0, G=1.0):
    """Run each initial condition through the solver and keep pairs_per_ic consecutive
    (psi_t, psi_b, psi_{t+K dt}) triples, starting after warmup_steps steps."""
    import torch
    S = len(ics) * pairs_per_ic
    dev = torch.device("cuda")
    psi = torch.empty((S, n, n, n), dtype=torch.complex64, device=dev)
    psib = torch.empty_like(psi)
    tgt = torch.empty_like(psi)
    fine = spe.Grid(n, G=G)
    coarse = spe.Grid(n, G=G, flags=spe.SPE_NO_CFL_CHECK)
    s = 0
    for ic in ics:
        fine.set_ic(ic)
        if warmup_steps:
            fine.step(warmup_steps, dt)
        for _ in range(pairs_per_ic):
            fine.get_psi(out=psi[s])
            coarse.set_ic(psi[s])
            coarse.step(1, K * dt)
            coarse.get_psi(out=psib[s])
            fine.step(K, dt)
            fine.get_psi(out=tgt[s])
            s += 1
    torch.cuda.synchronize()
    fine.destroy()
    coarse.destroy()
    return PairSet(psi, psib, tgt, dt, K)


def correction_scale(pairs: PairSet) -> float:
    """rms |psi_{t+K dt} - psi_b| over the set: the output scale sigma (sums by the library's
    FP64 reduction kernel)."""
    num, _ = spe.pair_norms(pairs.target, pairs.psi_b)
    return float(np.sqrt(num.sum() / (len(num) * pairs.psi[0].numel())))


def rel_errors(a, b):
    """Per-sample ||a - b|| / ||b|| of (S, n, n, n) tensors (sums by the library's FP64 reduction
    kernel)."""
    num, den = spe.pair_norms(a.contiguous(), b.contiguous())
    return np.sqrt(num / den)


def train(net: spe.Fno, pairs: PairSet, epochs=10, batch=8, lr=1e-3, lr_min=1e-5, seed=0, log=None):
    """Adam on shuffled mini-batches with a cosine learning-rate schedule; returns the mean loss
    of each epoch."""
    import torch
    S = len(pairs)
    rng = np.random.default_rng(seed)
    steps_per_epoch = max(1, S // batch)
    total = epochs * steps_per_epoch
    shape = (batch,) + tuple(pairs.psi.shape[1:])
    xb = torch.empty(shape, dtype=torch.complex64, device=pairs.psi.device)
    bb = torch.empty_like(xb)
    tb = torch.empty_like(xb)
    out = torch.empty_like(xb)
    hist = []
    it = 0
    for ep in range(epochs):
        perm = torch.as_tensor(rng.permutation(S)[:steps_per_epoch * batch], device=pairs.psi.device)
        acc = 0.0
        for k in range(steps_per_epoch):
            idx = perm[k * batch:(k + 1) * batch]
            torch.index_select(pairs.psi, 0, idx, out=xb)
            torch.index_select(pairs.psi_b, 0, idx, out=bb)
            torch.index_select(pairs.target, 0, idx, out=tb)
            net.forward(xb, bb, out=out)
            acc += net.backward(tb)
            cur = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * it / max(1, total - 1)))
            net.adam(lr=cur)
            it += 1
        hist.append(acc / steps_per_epoch)
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    return hist


def evaluate(net: spe.Fno, pairs: PairSet, batch=8):
    """Per-sample relative L2 errors against psi_{t+K dt}: of the coarse step alone and of the
    network's proposal."""
    import torch
    S = len(pairs)
    e_prop = []
    out = torch.empty((batch,) + tuple(pairs.psi.shape[1:]), dtype=torch.complex64, device=pairs.psi.device)
    for s in range(0, S, batch):
        m = min(batch, S - s)
        net.forward(pairs.psi[s:s + m].contiguous(), pairs.psi_b[s:s + m].contiguous(), out=out[:m])
        e_prop.append(rel_errors(out[:m], pairs.target[s:s + m]))
    e_coarse = rel_errors(pairs.psi_b, pairs.target)
    return e_coarse, np.concatenate(e_prop)


def timed(fn, reps=5):
    """Median wall time of fn() in seconds, synchronised on the device."""
    import torch
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    return float(np.median(ts))
