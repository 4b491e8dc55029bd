"""GPU parity of the FNO surrogate kernels against the FP64 oracle (oracle/fno_oracle.py).

The oracle runs with the BF16-rounded weights the kernels read.  Tolerances:
  * FP32 activations: the kernels differ from the oracle only by FP32 rounding of the tables and
    of sums of up to a few thousand terms, so the proposal's correction, the loss and every
    parameter group's gradient agree to 1e-4 relative (measured ~1e-6).
  * BF16 activations (the forward's row stages then run on the tensor cores with BF16 operands,
    the DFT tables and the spectral inputs included): each stored activation and each operand
    carries a relative rounding error of up to 2^-9 (about 2e-3); five stored activations lie on
    the path (v_0 .. v_4), so the correction agrees to 2e-2 and the gradients, which multiply two
    rounded activations, to 5e-2."""
import numpy as np
import torch
import pytest

from oracle import fno_oracle as fo
from paper_2606_25026_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_25026_gb300 import build
    build.build()
    from paper_2606_25026_gb300 import spe as mod
    mod.load_library()
    return mod


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def problem(n, batch, seed):
    """Halo fields psi, a perturbed coarse step psi_b and a target near psi_b."""
    rng = np.random.default_rng(seed)
    psis, pbs, tgs = [], [], []
    for b in range(batch):
        psi = inputs.soliton_halo(n, seed=seed + b).astype(np.complex128)
        noise = lambda s: s * (rng.standard_normal(psi.shape) + 1j * rng.standard_normal(psi.shape))
        pb = psi * np.exp(0.05j) + noise(0.02)
        psis.append(psi.astype(np.complex64).astype(np.complex128))
        pbs.append(pb.astype(np.complex64).astype(np.complex128))
        tgs.append((pb + noise(0.03)).astype(np.complex64).astype(np.complex128))
    return psis, pbs, tgs


def params_for(shape, seed):
    flat = inputs.fno_init_params(shape.layers, shape.modes, seed=seed, out_gain=1.0).astype(np.float64)
    rng = np.random.default_rng(seed + 100)
    p = fo.unpack(shape, flat)
    for l in range(shape.layers):   # signed spectral weights, large enough to matter
        p[f"R{l}"][:] = torch.tensor(rng.uniform(-1, 1, tuple(p[f"R{l}"].shape)) / shape.width)
    return flat.astype(np.float32)


def to_dev(arrs):
    import torch
    return torch.tensor(np.stack(arrs).astype(np.complex64), device="cuda")


def oracle_outputs(shape, flat32, psis, pbs, tgs, inv_A, sigma):
    w = fo.round_bf16(flat32.astype(np.float64))
    outs = [fo.forward(shape, w, p, b, inv_A, sigma).detach().numpy() for p, b in zip(psis, pbs)]
    loss, grad = fo.loss_and_grad(shape, w, psis, pbs, tgs, inv_A, sigma)
    return outs, loss, grad


CASES = [
    # (n, M, layers, batch, act_fp32)
    (32, 16, 4, 2, True),
    (32, 8, 2, 1, True),
    (64, 16, 2, 1, True),
    (32, 16, 4, 2, False),
    (64, 16, 2, 1, False),
    (32, 8, 3, 2, False),
]


@pytest.mark.parametrize("n,M,L,B,fp32", CASES)
def test_forward_loss_and_gradients_match_oracle(spe, n, M, L, B, fp32):
    shape = fo.FnoShape(n=n, modes=M, layers=L)
    inv_A, sigma = 0.9, 0.05
    flat = params_for(shape, seed=n + M + L)
    psis, pbs, tgs = problem(n, B, seed=7 * n + L)
    net = spe.Fno(n=n, layers=L, modes=M, max_batch=B, train=True, act_fp32=fp32, inv_A=inv_A, sigma=sigma)
    assert net.param_count == fo.param_count(shape)
    net.set_params(flat)
    assert np.array_equal(net.get_params(), flat)
    out = net.forward(to_dev(psis), to_dev(pbs)).cpu().numpy()
    loss = net.backward(to_dev(tgs))
    g = net.grads()
    o_out, o_loss, o_grad = oracle_outputs(shape, flat, psis, pbs, tgs, inv_A, sigma)
    tol_f, tol_g = (1e-4, 1e-4) if fp32 else (2e-2, 5e-2)
    for b in range(B):
        corr = (out[b] - pbs[b]) / sigma
        want = (o_out[b] - pbs[b]) / sigma
        assert rel_l2(corr, want) <= tol_f, (b, rel_l2(corr, want))
    assert loss == pytest.approx(o_loss, rel=tol_f)
    off = 0
    worst = {}
    for name, shp in fo.param_layout(shape):
        cnt = int(np.prod(shp))
        e = rel_l2(g[off:off + cnt].astype(np.float64), o_grad[off:off + cnt])
        worst[name] = e
        off += cnt
    print({k: f"{v:.1e}" for k, v in worst.items()})
    for name, e in worst.items():
        assert e <= tol_g, (name, e)


def test_adam_step_matches_oracle(spe):
    shape = fo.FnoShape(n=32, modes=8, layers=2)
    flat = params_for(shape, seed=3)
    psis, pbs, tgs = problem(32, 1, seed=11)
    net = spe.Fno(n=32, layers=2, modes=8, train=True, act_fp32=True, sigma=0.05)
    net.set_params(flat)
    opt = fo.Adam(len(flat), lr=2e-3, beta1=0.9, beta2=0.99, eps=1e-7)
    theta = flat.astype(np.float64)
    for _ in range(3):
        net.forward(to_dev(psis), to_dev(pbs))
        net.backward(to_dev(tgs), want_loss=False)
        g = net.grads().astype(np.float64)
        net.adam(lr=2e-3, beta1=0.9, beta2=0.99, eps=1e-7)
        theta = opt.step(theta, g)
        got = net.get_params().astype(np.float64)
        # FP32 Adam against FP64 Adam on the same gradients
        assert np.max(np.abs(got - theta)) <= 1e-6 * max(1.0, np.max(np.abs(theta)))
        theta = got   # continue from the device's parameters (the next gradient is taken there)


def test_training_reduces_loss(spe):
    """A few Adam steps on one fixed batch lower the loss (the kernels' gradient is a descent
    direction of their own forward).  The target's correction, 0.03 i psi, is a pointwise linear
    map of the features, so the network can represent it."""
    shape = fo.FnoShape(n=32, modes=8, layers=2)
    flat = inputs.fno_init_params(shape.layers, shape.modes, seed=5)
    psis, pbs, _ = problem(32, 2, seed=21)
    tgs = [b + 0.03j * p for p, b in zip(psis, pbs)]
    net = spe.Fno(n=32, layers=2, modes=8, max_batch=2, train=True, sigma=0.03)
    net.set_params(flat)
    P, B, T = to_dev(psis), to_dev(pbs), to_dev(tgs)
    losses = []
    for _ in range(30):
        net.forward(P, B)
        losses.append(net.backward(T))
        net.adam(lr=3e-3)
    print("losses", losses[0], losses[-1])
    assert losses[-1] < 0.5 * losses[0]


def test_inference_mode_matches_training_forward(spe):
    shape = fo.FnoShape(n=32, modes=16, layers=3)
    flat = params_for(shape, seed=9)
    psis, pbs, _ = problem(32, 2, seed=31)
    outs = []
    for train in (True, False):
        net = spe.Fno(n=32, layers=3, modes=16, max_batch=2, train=train, sigma=0.05)
        net.set_params(flat)
        outs.append(net.forward(to_dev(psis), to_dev(pbs)).cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_forward_in_place_and_deterministic(spe):
    import torch
    shape = fo.FnoShape(n=32, modes=16, layers=2)
    flat = params_for(shape, seed=13)
    psis, pbs, tgs = problem(32, 1, seed=41)
    net = spe.Fno(n=32, layers=2, modes=16, train=True, sigma=0.05)
    net.set_params(flat)
    a = net.forward(to_dev(psis), to_dev(pbs)).cpu().numpy()
    l1 = net.backward(to_dev(tgs))
    g1 = net.grads()
    net.forward(to_dev(psis), to_dev(pbs))
    l2 = net.backward(to_dev(tgs))
    assert l1 == l2 and np.array_equal(g1, net.grads())          # fixed-order reductions
    inf = spe.Fno(n=32, layers=2, modes=16, sigma=0.05)
    inf.set_params(flat)
    buf = to_dev(pbs)
    inf.forward(to_dev(psis), buf, out=buf)
    assert np.array_equal(buf.cpu().numpy(), a)


def test_bad_arguments(spe):
    with pytest.raises(spe.SpeError):
        spe.Fno(n=48)
    with pytest.raises(spe.SpeError):
        spe.Fno(n=32, modes=32)
    net = spe.Fno(n=32, layers=1, modes=8, sigma=0.1)
    import torch
    z = torch.zeros((1, 32, 32, 32), dtype=torch.complex64, device="cuda")
    with pytest.raises(spe.SpeError) as e:
        net.backward(z)
    assert e.value.status == spe.SPE_ESTATE
    with pytest.raises(spe.SpeError):
        net.forward(torch.zeros((2, 32, 32, 32), dtype=torch.complex64, device="cuda"),
                    torch.zeros((2, 32, 32, 32), dtype=torch.complex64, device="cuda"))


@pytest.mark.parametrize("n,M", [(64, 16), (32, 8)])
def test_tensor_core_forward_matches_fp32_path(spe, n, M):
    """The BF16 tensor-core forward against the FP32 CUDA-core forward of the same weights."""
    shape = fo.FnoShape(n=n, modes=M, layers=3)
    flat = params_for(shape, seed=40 + n)
    psis, pbs, _ = problem(n, 2, seed=50 + n)
    outs = []
    for fp32 in (True, False):
        net = spe.Fno(n=n, layers=3, modes=M, max_batch=2, act_fp32=fp32, sigma=0.05)
        net.set_params(flat)
        outs.append(net.forward(to_dev(psis), to_dev(pbs)).cpu().numpy())
        net.sync()
    for b in range(2):
        c32 = (outs[0][b] - pbs[b]) / 0.05
        c16 = (outs[1][b] - pbs[b]) / 0.05
        assert rel_l2(c16, c32) <= 2e-2, rel_l2(c16, c32)


def test_graph_replay_matches_direct_forward(spe):
    """The inference forward replayed as a CUDA graph (third and later identical calls) equals
    the directly launched one bitwise, and follows parameter updates without re-capture."""
    import torch
    shape = fo.FnoShape(n=32, modes=16, layers=2)
    flat = params_for(shape, seed=77)
    psis, pbs, _ = problem(32, 1, seed=78)
    P, B = to_dev(psis), to_dev(pbs)
    direct = spe.Fno(n=32, layers=2, modes=16, sigma=0.05, graph=False)
    graphed = spe.Fno(n=32, layers=2, modes=16, sigma=0.05)
    outs = {}
    for name, net in (("direct", direct), ("graphed", graphed)):
        net.set_params(flat)
        o = torch.empty_like(B)
        for _ in range(4):
            net.forward(P, B, out=o)
        outs[name] = o.cpu().numpy()
        net.set_params(flat * 1.5)
        net.forward(P, B, out=o)
        outs[name + "2"] = o.cpu().numpy()
    assert np.array_equal(outs["direct"], outs["graphed"])
    assert np.array_equal(outs["direct2"], outs["graphed2"])
    assert not np.array_equal(outs["direct"], outs["direct2"])


def test_profile_mode_counts_kernels(spe):
    import torch
    shape = fo.FnoShape(n=32, modes=16, layers=2)
    net = spe.Fno(n=32, layers=2, modes=16, sigma=0.05, profile=True)
    net.set_params(params_for(shape, seed=3))
    psis, pbs, _ = problem(32, 1, seed=4)
    P, B = to_dev(psis), to_dev(pbs)
    o = torch.empty_like(B)
    for _ in range(3):
        net.forward(P, B, out=o)
    prof = net.profile_read()
    assert prof["fno_layer"][0] == 3 and prof["fno_last_layer"][0] == 3 and prof["fno_z_mix"][0] == 6
    assert all(ms > 0 for _, ms in prof.values())
    assert net.profile_read() == {}
    with pytest.raises(spe.SpeError):
        spe.Fno(n=32, layers=1, modes=8, sigma=0.1).profile_read()
