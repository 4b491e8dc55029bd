"""Pins of the FP64 FNO oracle (oracle/fno_oracle.py) against things other than itself:
standard-normal CDF values for GELU, closed forms of the spectral layer on single Fourier modes,
the identity on band-limited fields, a brute-force DFT of the layer's definition, translation
equivariance, central finite differences of the loss, and Adam's first-step closed form plus
torch.optim.Adam over several steps."""
import math

import numpy as np
import pytest
import torch

from oracle import fno_oracle as fo
from paper_2606_25026_gb300 import inputs

# Phi(1) and Phi(-1) of the standard normal distribution (tabulated values).
PHI_1 = 0.8413447460685429


def test_gelu_values():
    u = torch.tensor([0.0, 1.0, -1.0, 2.5, -2.5], dtype=torch.float64)
    g = fo.gelu(u)
    assert g[0] == 0.0
    assert float(g[1]) == pytest.approx(PHI_1, abs=1e-15)
    assert float(g[2]) == pytest.approx(-(1.0 - PHI_1), abs=1e-15)
    # GELU(u) - GELU(-u) = u
    assert torch.allclose(g[3] - g[4], torch.tensor(2.5, dtype=torch.float64), atol=1e-15)


def grid(n):
    i = torch.arange(n, dtype=torch.float64)
    return torch.meshgrid(i, i, i, indexing="ij")          # z, y, x


def identity_R(M, C, r=1.0 + 0.0j):
    R = torch.zeros((M, M, M, C, C), dtype=torch.complex128)
    for c in range(C):
        R[..., c, c] = r
    return R


def theta(n, kx, ky, kz):
    z, y, x = grid(n)
    return 2 * math.pi * (kx * x + ky * y + kz * z) / n


@pytest.mark.parametrize("kx,ky,kz", [(1, 2, -3), (5, -4, 0), (7, 3, -4)])
def test_single_mode_complex_multiplier(kx, ky, kz):
    """cos(theta) with kx >= 1 through R = r I gives Re(r e^{i theta})."""
    n, M = 16, 8
    th = theta(n, kx, ky, kz)
    r = 0.7 - 0.45j
    v = torch.cos(th)[None]
    s = fo.spectral_conv(v, identity_R(M, 1, r), M)[0]
    want = r.real * torch.cos(th) - r.imag * torch.sin(th)
    assert torch.max(torch.abs(s - want)) < 1e-12


def test_kx0_mode_takes_real_part():
    """kx = 0: both +-(ky, kz) lie in the box; the x real inverse keeps Re(r) cos(theta)."""
    n, M = 16, 8
    th = theta(n, 0, 3, -2)
    r = 0.7 - 0.45j
    s = fo.spectral_conv(torch.cos(th)[None], identity_R(M, 1, r), M)[0]
    assert torch.max(torch.abs(s - r.real * torch.cos(th))) < 1e-12


def test_box_edge_and_outside():
    """ky = -M/2 is in the box but +M/2 is not, so cos(2 pi (M/2) y / n) comes out halved; a
    mode with kx = M is outside and vanishes."""
    n, M = 16, 8
    v = torch.cos(theta(n, 0, M // 2, 0))[None]
    s = fo.spectral_conv(v, identity_R(M, 1), M)[0]
    assert torch.max(torch.abs(s - 0.5 * v[0])) < 1e-12
    v = torch.cos(theta(n, M, 1, 1))[None]
    s = fo.spectral_conv(v, identity_R(M, 1), M)[0]
    assert torch.max(torch.abs(s)) < 1e-12


def test_band_limited_identity():
    """R = I reproduces any real field whose modes lie strictly inside the box."""
    n, M, C = 16, 8, 3
    rng = np.random.default_rng(4)
    v = torch.zeros((C, n, n, n), dtype=torch.float64)
    for c in range(C):
        for _ in range(6):
            kx = int(rng.integers(0, M))
            ky, kz = (int(t) for t in rng.integers(-(M // 2) + 1, M // 2, 2))
            v[c] += float(rng.standard_normal()) * torch.cos(theta(n, kx, ky, kz) + float(rng.random() * 6))
    s = fo.spectral_conv(v, identity_R(M, C), M)
    assert torch.max(torch.abs(s - v)) < 1e-12


def test_spectral_conv_brute_force_definition():
    """The layer equals its written-out definition on an 8^3 grid:
    X(k) = sum_x v(x) e^{-i k.x 2pi/n}, Y = R X, s(x) = Re sum_k w(kx) Y(k) e^{+i k.x 2pi/n} / n^3
    with w(0) = 1, w(kx > 0) = 2, k over the mode box."""
    n, M, C = 8, 4, 2
    rng = np.random.default_rng(9)
    v = rng.standard_normal((C, n, n, n))
    R = rng.standard_normal((M, M, M, C, C)) + 1j * rng.standard_normal((M, M, M, C, C))
    got = fo.spectral_conv(torch.tensor(v), torch.tensor(R), M).numpy()
    f = [m if m < M // 2 else m - M for m in range(M)]
    idx = np.arange(n)
    s = np.zeros((C, n, n, n))
    for a in range(M):          # kz
        for bb in range(M):     # ky
            for kx in range(M):
                ph = np.exp(-2j * np.pi * (f[a] * idx[:, None, None] + f[bb] * idx[None, :, None]
                                           + kx * idx[None, None, :]) / n)
                X = np.array([np.sum(v[c] * ph) for c in range(C)])
                Y = R[a, bb, kx].T @ X            # R[k][i][o]: Y_o = sum_i R_io X_i
                w = 1.0 if kx == 0 else 2.0
                for o in range(C):
                    s[o] += np.real(w * Y[o] * np.conj(ph)) / n ** 3
    assert np.max(np.abs(got - s)) < 1e-10


def tiny_shape():
    return fo.FnoShape(n=8, width=4, modes=4, layers=2, hidden=8)


def tiny_problem(seed=0):
    s = tiny_shape()
    rng = np.random.default_rng(seed)
    flat = inputs.fno_init_params(s.layers, s.modes, seed=seed, out_gain=1.0, width=s.width,
                                  hidden=s.hidden).astype(np.float64)
    # make the spectral weights as large as the pointwise ones so their gradients matter
    p = fo.unpack(s, flat)
    for l in range(s.layers):
        p[f"R{l}"][:] = torch.tensor(rng.standard_normal(tuple(p[f"R{l}"].shape)) * 0.3)
    shp = (s.n,) * 3
    mk = lambda: rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    psis = [mk(), mk()]
    pbs = [q + 0.1 * mk() for q in psis]
    tgs = [q + 0.1 * mk() for q in pbs]
    return s, flat, psis, pbs, tgs


def test_loss_gradient_matches_central_differences():
    s, flat, psis, pbs, tgs = tiny_problem()
    sig = 0.3
    _, g = fo.loss_and_grad(s, flat, psis, pbs, tgs, inv_A=0.8, sigma=sig)
    rng = np.random.default_rng(1)
    offs, off = {}, 0
    for name, shape in fo.param_layout(s):
        offs[name] = (off, int(np.prod(shape)))
        off += int(np.prod(shape))
    picks = []
    for name, (o, cnt) in offs.items():
        picks += [o + int(i) for i in rng.choice(cnt, size=min(cnt, 4), replace=False)]
    h = 1e-5
    for i in picks:
        a = flat.copy(); a[i] += h
        b = flat.copy(); b[i] -= h
        lp = float(fo.loss(s, a, psis, pbs, tgs, 0.8, sig))
        lm = float(fo.loss(s, b, psis, pbs, tgs, 0.8, sig))
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_zero_head_returns_coarse_step():
    s, flat, psis, pbs, tgs = tiny_problem(3)
    p = fo.unpack(s, flat.copy())
    p["Q2"][:] = 0.0
    p["q2"][:] = 0.0
    out = fo.forward(s, p, psis[0], pbs[0], sigma=2.0)
    assert np.max(np.abs(out.numpy() - pbs[0])) == 0.0
    want = sum(np.sum(np.abs(b - t) ** 2) for b, t in zip(pbs, tgs)) / (4.0 * 2 * s.n ** 3)
    assert float(fo.loss(s, p, psis, pbs, tgs, sigma=2.0)) == pytest.approx(want, rel=1e-13)


def test_translation_equivariance():
    s, flat, psis, pbs, _ = tiny_problem(5)
    a = fo.forward(s, flat, psis[0], pbs[0]).numpy()
    sh = (3, -2, 5)
    b = fo.forward(s, flat, np.roll(psis[0], sh, (0, 1, 2)), np.roll(pbs[0], sh, (0, 1, 2))).numpy()
    assert np.max(np.abs(np.roll(a, sh, (0, 1, 2)) - b)) < 1e-11


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    opt = fo.Adam(50, lr=1e-2, eps=1e-8)
    t1 = opt.step(th, g)
    assert np.max(np.abs(t1 - (th - 1e-2 * g / (np.abs(g) + 1e-8)))) < 1e-15


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(7)
    th = rng.standard_normal(40)
    opt = fo.Adam(40, lr=3e-3, beta1=0.85, beta2=0.99, eps=1e-6)
    p = torch.tensor(th.copy(), requires_grad=True)
    topt = torch.optim.Adam([p], lr=3e-3, betas=(0.85, 0.99), eps=1e-6)
    for k in range(6):
        g = rng.standard_normal(40) * (k + 1)
        th = opt.step(th, g)
        p.grad = torch.tensor(g)
        topt.step()
    assert np.max(np.abs(th - p.detach().numpy())) < 1e-12


def test_param_count_of_config():
    s = fo.FnoShape()
    # P, p, 4 x (W, b, R), Q1, q1, Q2, q2
    want = 32 * 4 + 32 + 4 * (32 * 32 + 32 + 16 ** 3 * 32 * 32 * 2) + 64 * 32 + 64 + 2 * 64 + 2
    assert fo.param_count(s) == want


def test_seeded_initialiser_uses_the_oracle_layout():
    """The shared seeded initialiser and the oracle agree on the flat parameter format."""
    s = fo.FnoShape(n=32, modes=8, layers=3)
    shapes = inputs.fno_param_shapes(s.layers, s.modes)
    assert [(a, tuple(b)) for a, b in shapes] == [(a, tuple(b)) for a, b in fo.param_layout(s)]
    assert inputs.fno_init_params(s.layers, s.modes).size == fo.param_count(s)
