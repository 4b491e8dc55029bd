"""FP64 CPU oracle of the Fourier-neural-operator surrogate (test infrastructure only: the tests,
the smoke check and the CPU baseline of the benchmark may import it; the CUDA path never does).

The surrogate proposes psi K steps ahead from the state psi and the plain solver's single coarse
step psi_b = S(K dt) psi (one kick-drift-kick step of length K dt, Algorithm 1 of Sec. 3 with a
larger dt).  The network maps the four real feature channels

    f = (Re psi, Im psi, Re psi_b, Im psi_b) / A

through a pointwise lift P (4 -> C channels), L Fourier layers and a pointwise two-layer
projection Q (C -> H -> 2), and the proposal is psi_b + sigma (o_0 + i o_1).  A Fourier layer is

    u = W v + b + Re IDFT[ R . DFT_M(v) ],     v' = GELU(u)  (identity for the last layer)

where DFT_M is the 3D DFT of the real channels truncated to the mode box
kx in [0, M), ky, kz in [-M/2, M/2) (x is the half-spectrum axis), R a complex C x C matrix per
mode, and the inverse is the real inverse of the half spectrum (numpy/torch irfftn semantics:
the imaginary part of a kx = 0 term after the z, y inverses is dropped).  GELU is the exact
erf form.  None of this is in the paper: it is the learned part built on top of the method.

Parameters travel as one flat float vector in this order:
    P [C][4], p [C],
    per layer l: W_l [C][C] (out, in), b_l [C], R_l [M^3][C_in][C_out][2]  (mode index
        k = (kz * M + ky) * M + kx with signed frequency f(m) = m for m < M/2, m - M otherwise),
    Q1 [H][C], q1 [H], Q2 [2][H], q2 [2].

The loss of a batch is  sum_b sum_cells |psi_pred - psi_target|^2 / (sigma^2 B n^3).
Gradients come from torch autograd in float64; Adam is written out from Kingma & Ba (2015),
Algorithm 1.  The oracle is pinned by finite differences, closed forms of the spectral layer on
single modes, the band-limited identity and the Adam first-step closed form
(tests/test_oracle_fno_pins.py)."""
from dataclasses import dataclass
import math

import numpy as np
import torch


@dataclass(frozen=True)
class FnoShape:
    n: int = 64          # grid points per axis
    width: int = 32      # C
    modes: int = 16      # M per axis
    layers: int = 4      # L
    hidden: int = 64     # H
    in_ch: int = 4
    out_ch: int = 2


def param_layout(s: FnoShape):
    """[(name, shape)] in flat-vector order."""
    C, M, H = s.width, s.modes, s.hidden
    out = [("P", (C, s.in_ch)), ("p", (C,))]
    for l in range(s.layers):
        out += [(f"W{l}", (C, C)), (f"b{l}", (C,)), (f"R{l}", (M ** 3, C, C, 2))]
    out += [("Q1", (H, C)), ("q1", (H,)), ("Q2", (s.out_ch, H)), ("q2", (s.out_ch,))]
    return out


def param_count(s: FnoShape) -> int:
    return sum(int(np.prod(shape)) for _, shape in param_layout(s))


def unpack(s: FnoShape, flat):
    """Split a flat vector (numpy or torch) into named float64 tensors (views of one leaf if a
    torch tensor is given, so autograd flows back to it)."""
    t = flat if isinstance(flat, torch.Tensor) else torch.as_tensor(np.asarray(flat, np.float64))
    out, off = {}, 0
    for name, shape in param_layout(s):
        cnt = int(np.prod(shape))
        out[name] = t[off:off + cnt].reshape(shape)
        off += cnt
    assert off == t.numel()
    return out


def gelu(u):
    """Exact GELU: u Phi(u) with Phi the standard normal CDF."""
    return 0.5 * u * (1.0 + torch.erf(u / math.sqrt(2.0)))


def mode_index(n: int, M: int):
    """Grid indices of the signed frequencies f(m), m = 0..M-1, of a full (complex) axis."""
    return [m if m < M // 2 else n + m - M for m in range(M)]


def spectral_conv(v, R, M):
    """Re IDFT[R . DFT_M(v)] for real channels v [C, n, n, n] (z, y, x) and R [M, M, M, C_in,
    C_out] complex.  Unnormalised forward DFT, 1/n^3 on the inverse."""
    C, n = v.shape[0], v.shape[1]
    V = torch.fft.rfftn(v, dim=(1, 2, 3))                      # [C, n, n, n/2+1]
    sel = torch.tensor(mode_index(n, M))
    X = V[:, sel][:, :, sel][:, :, :, :M]                      # [C, M(kz), M(ky), M(kx)]
    Y = torch.einsum("zyxio,izyx->ozyx", R, X)
    full = torch.zeros((R.shape[-1], n, n, n // 2 + 1), dtype=V.dtype)
    idx_z = sel.view(-1, 1, 1)
    idx_y = sel.view(1, -1, 1)
    idx_x = torch.arange(M).view(1, 1, -1)
    full[:, idx_z, idx_y, idx_x] = Y
    return torch.fft.irfftn(full, s=(n, n, n), dim=(1, 2, 3))


def features(psi, psi_b, inv_A):
    psi = torch.as_tensor(psi)
    psi_b = torch.as_tensor(psi_b)
    return torch.stack([psi.real, psi.imag, psi_b.real, psi_b.imag]) * inv_A


def forward(s: FnoShape, params, psi, psi_b, inv_A=1.0, sigma=1.0):
    """psi_pred for one sample (psi, psi_b complex [n, n, n] as z, y, x)."""
    p = params if isinstance(params, dict) else unpack(s, params)
    M = s.modes
    f = features(psi, psi_b, inv_A)
    v = torch.einsum("cf,fzyx->czyx", p["P"], f) + p["p"].view(-1, 1, 1, 1)
    for l in range(s.layers):
        Rr = p[f"R{l}"].reshape(M, M, M, s.width, s.width, 2)
        R = torch.complex(Rr[..., 0], Rr[..., 1])
        u = (torch.einsum("oi,izyx->ozyx", p[f"W{l}"], v) + p[f"b{l}"].view(-1, 1, 1, 1)
             + spectral_conv(v, R, M))
        v = gelu(u) if l < s.layers - 1 else u
    h = gelu(torch.einsum("hc,czyx->hzyx", p["Q1"], v) + p["q1"].view(-1, 1, 1, 1))
    o = torch.einsum("oh,hzyx->ozyx", p["Q2"], h) + p["q2"].view(-1, 1, 1, 1)
    return torch.as_tensor(psi_b) + sigma * torch.complex(o[0], o[1])


def loss(s: FnoShape, params, psis, psi_bs, targets, inv_A=1.0, sigma=1.0):
    """Batch loss sum_b sum_cells |psi_pred - target|^2 / (sigma^2 B n^3)."""
    B = len(psis)
    tot = 0.0
    for psi, pb, tg in zip(psis, psi_bs, targets):
        d = forward(s, params, psi, pb, inv_A, sigma) - torch.as_tensor(tg)
        tot = tot + (d.real ** 2 + d.imag ** 2).sum()
    return tot / (sigma ** 2 * B * s.n ** 3)


def loss_and_grad(s: FnoShape, flat, psis, psi_bs, targets, inv_A=1.0, sigma=1.0):
    """(loss, d loss / d flat) in float64 through autograd."""
    t = torch.tensor(np.asarray(flat, np.float64), requires_grad=True)
    L = loss(s, unpack(s, t), psis, psi_bs, targets, inv_A, sigma)
    L.backward()
    return float(L.detach()), t.grad.numpy().copy()


class Adam:
    """Adam (Kingma & Ba 2015, Algorithm 1) on a flat float64 vector."""

    def __init__(self, n, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0

    def step(self, theta, g, lr=None):
        lr = self.lr if lr is None else lr
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * g
        self.v = self.b2 * self.v + (1.0 - self.b2) * g * g
        m_hat = self.m / (1.0 - self.b1 ** self.t)
        v_hat = self.v / (1.0 - self.b2 ** self.t)
        return theta - lr * m_hat / (np.sqrt(v_hat) + self.eps)


def round_bf16(x) -> np.ndarray:
    """Round float64 values to bfloat16 (round to nearest even) and back."""
    return torch.as_tensor(np.asarray(x, np.float64)).to(torch.float32).to(torch.bfloat16) \
        .to(torch.float64).numpy()
