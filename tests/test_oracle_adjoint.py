"""Pins of the adjoint oracle (oracle/adjoint.py) on the CPU.

- its vectorised Philox4x32-10 against the published known answers and the
  C oracle's scalar implementation;
- the noise: exact Irwin-Hall(12) moments;
- the smooth variant's adjoint against central finite differences of the
  same forward (float64);
- the surrogate adjoint against PyTorch autograd of an independently
  written, unrolled forward with a custom spike function.
"""
import os

import numpy as np
import pytest

import oracle
import oracle.adjoint as adj
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    return rows


def test_vector_philox_known_answers_and_scalar_oracle():
    for r in _kat():
        out = adj.philox_blocks(np.array([r[0]], np.uint64), r[1], r[2], r[3], r[4], r[5])[0]
        assert list(out) == r[6:10]
    rng = np.random.default_rng(3)
    c = rng.integers(0, 2 ** 32, 64, dtype=np.uint64)
    out = adj.philox_blocks(c, 12345, adj.NOISE_TAG, 0, 0xDEADBEEF, 77)
    for i in range(64):
        ref = oracle.philox4x32_10([int(c[i]), 12345, adj.NOISE_TAG, 0], [0xDEADBEEF, 77])
        assert np.array_equal(out[i], ref)


def test_noise_moments():
    x = np.concatenate([adj.noise(11, 4096, t) for t in range(16)]).astype(np.float64)
    # 12 bytes of mean 127.5 sum to mean 1530: the draws are centred at 0, with the
    # variance of 12 uniform bytes / 256^2
    assert abs(x.mean()) < 0.02
    assert abs(x.var() - 12 * (256 ** 2 - 1) / 12 / 256 ** 2) < 0.03
    assert np.all(x * 256 == np.round(x * 256))  # exact multiples of 2^-8


def _tiny(M=192, K=14, P=4, n_vn=2, dmax=4, seed=21):
    cfg = synth.NetConfig(name="adj", M=M, P=P, n_vn=n_vn, K=K, uniform_all=False, n_part=K - 6, n_vn_t=4,
                          n_remote=2, dmax=dmax, seed=seed, dyn=synth.Dynamics(w_ext=89, drive_seed=5))
    g = synth.make_network(cfg)
    part = oracle.partition_planted(M, P)
    vn = oracle.group_contiguous(P, n_vn)
    alpha = oracle.alpha32(cfg.dyn.dt_ms, cfg.dyn.tau_ms)
    return adj.from_synth(g, cfg.dyn, part, vn, alpha)


def _loss(rates, target):
    return float(((rates - target) ** 2).sum() / len(rates))


def test_smooth_adjoint_equals_finite_differences():
    net = _tiny()
    rng = np.random.default_rng(5)
    G = 1.0 + 0.3 * rng.standard_normal((net.n_pop, net.n_pop))
    lam = 0.8 + 0.2 * rng.random(net.n_pop)
    T = 40
    target = 0.02 * rng.random(net.n_pop)
    v0 = net.v0.copy()
    net.v0 = (v0.astype(np.float64) + 8.0).astype(np.float32)  # start nearer threshold: active logistic
    tr = adj.forward_smooth(net, G, lam, T)
    grates = 2 * (tr.rates - target) / net.n_pop
    dG, dlam = adj.backward(net, G, lam, tr, grates, smooth=True)
    eps = 1e-6
    for (i, j) in [(0, 0), (0, 1), (1, 0), (2, 3), (3, 3), (3, 1)]:
        Gp, Gm = G.copy(), G.copy()
        Gp[i, j] += eps
        Gm[i, j] -= eps
        fd = (_loss(adj.forward_smooth(net, Gp, lam, T).rates, target)
              - _loss(adj.forward_smooth(net, Gm, lam, T).rates, target)) / (2 * eps)
        assert abs(fd - dG[i, j]) <= 1e-6 * max(1e-9, abs(fd)) + 1e-13, (i, j, fd, dG[i, j])
    for a in range(net.n_pop):
        lp, lm = lam.copy(), lam.copy()
        lp[a] += eps
        lm[a] -= eps
        fd = (_loss(adj.forward_smooth(net, G, lp, T).rates, target)
              - _loss(adj.forward_smooth(net, G, lm, T).rates, target)) / (2 * eps)
        assert abs(fd - dlam[a]) <= 1e-6 * max(1e-9, abs(fd)) + 1e-13, (a, fd, dlam[a])
    assert np.abs(dG).max() > 1e-9 and np.abs(dlam).max() > 1e-9


def _torch_surrogate(net, G, lam, T, target):
    """An unrolled hard-threshold forward in torch (float64) with a surrogate
    spike function and a detached reset; returns the loss, the trajectory
    and the leaf parameters."""
    torch = pytest.importorskip("torch")

    class Spike(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x):
            ctx.save_for_backward(x)
            return (x >= 0).to(x.dtype)

        @staticmethod
        def backward(ctx, g):
            (x,) = ctx.saved_tensors
            return g / (1.0 + adj.BETA * x.abs()) ** 2

    Gt = torch.tensor(G, dtype=torch.float64, requires_grad=True)
    lt = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
    M, npop = net.M, net.n_pop
    D = net.dmax + 1
    src = torch.tensor(net.src)
    tgt = torch.tensor(net.tgt)
    w = torch.tensor(net.w, dtype=torch.float64)
    dly = torch.tensor(net.d)
    pop = torch.tensor(net.pop)
    spop = pop[src]
    ring = [torch.zeros(M, npop, dtype=torch.float64) for _ in range(D)]
    V = torch.tensor(net.v0.astype(np.float64))
    ref = torch.zeros(M, dtype=torch.int64)
    alpha = float(net.alpha)
    vps, spks, refrs, As = [], [], [], []
    total = torch.zeros(npop, dtype=torch.float64)
    for t in range(T):
        A = ring[t % D]
        ring[t % D] = torch.zeros(M, npop, dtype=torch.float64)
        xi = torch.tensor(adj.noise(net.seed, M, t).astype(np.float64))
        I = (Gt[pop] * A).sum(dim=1) + net.w_ext * (lt[pop] + float(adj.SIGMA) * xi)
        vp = net.e_l + alpha * (V - net.e_l) + I * 2.0 ** -10
        refr = ref > 0
        S = Spike.apply(vp - net.v_th) * (~refr).to(torch.float64)
        vps.append(vp.detach().numpy().copy())
        spks.append(S.detach().numpy() > 0.5)
        refrs.append(refr.numpy().copy())
        As.append(A.detach().numpy().copy())
        Sd = S.detach()
        V = torch.where(refr, torch.full_like(vp, net.v_reset), vp * (1 - Sd) + net.v_reset * Sd)
        ref = torch.where(refr, ref - 1, torch.where(Sd > 0, torch.full_like(ref, net.t_ref), torch.zeros_like(ref)))
        total = total + torch.zeros(npop, dtype=torch.float64).index_add(0, pop, S)
        contrib = w * S[src]
        for dd in range(1, D):
            m = dly == dd
            if m.any():
                slot = (t + dd) % D
                ring[slot] = ring[slot].index_put((tgt[m], spop[m]), contrib[m], accumulate=True)
    rates = total / (T * torch.tensor(net.pop_sizes()))
    loss = ((rates - torch.tensor(target)) ** 2).sum() / npop
    loss.backward()
    tr = adj.Trajectory(np.array(vps), np.array(spks), np.array(refrs), np.array(As), rates.detach().numpy())
    return tr, Gt.grad.numpy(), lt.grad.numpy()


def test_surrogate_adjoint_equals_autograd():
    net = _tiny(M=160, K=12, seed=33)
    rng = np.random.default_rng(9)
    G = 1.0 + 0.2 * rng.standard_normal((net.n_pop, net.n_pop))
    lam = np.array([0.9, 1.1, 1.0, 1.2])
    net.v0 = (net.v0.astype(np.float64) + 6.0).astype(np.float32)
    T = 50
    target = 0.05 * rng.random(net.n_pop)
    tr, gG, glam = _torch_surrogate(net, G, lam, T, target)
    assert tr.spk.sum() > 20
    grates = 2 * (tr.rates - target) / net.n_pop
    dG, dlam = adj.backward(net, G, lam, tr, grates, smooth=False)
    assert np.allclose(dG, gG, rtol=1e-10, atol=1e-14)
    assert np.allclose(dlam, glam, rtol=1e-10, atol=1e-14)
    assert np.abs(gG).max() > 0


def test_fp32_forward_matches_surrogate_reference_spikes():
    """The float32 forward (the GPU's reference) and the float64 torch forward
    agree on the spikes of a short run (rounding does not flip a crossing here)."""
    net = _tiny(M=160, K=12, seed=33)
    rng = np.random.default_rng(9)
    G = 1.0 + 0.2 * rng.standard_normal((net.n_pop, net.n_pop))
    lam = np.array([0.9, 1.1, 1.0, 1.2])
    net.v0 = (net.v0.astype(np.float64) + 6.0).astype(np.float32)
    tr64, _, _ = _torch_surrogate(net, G, lam, 50, np.zeros(net.n_pop))
    tr32 = adj.forward_fp32(net, G.astype(np.float32), lam.astype(np.float32), 50)
    assert np.array_equal(tr32.spk, tr64.spk)
    assert np.array_equal(tr32.A, tr64.A.astype(np.int64))
    assert np.allclose(tr32.vpre, tr64.vpre, rtol=1e-5, atol=1e-4)
