"""GPU parity of the surrogate-gradient adjoint (through the C ABI) against
the CPU oracle (oracle/adjoint.py): the float32 forward bit for bit (every
spike), the gradients against the float64 backward on the same trajectory
(relative error reported, bound 1e-5), gradients independent of the
checkpoint interval, and the torch.autograd.Function wrapper."""
import numpy as np
import pytest

import oracle
import oracle.adjoint as adj
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_07125_gb300 as m
    return m


def _setup(snn, M=4096, P=4, n_vn=2, K=64, T=120, ckpt=32, seed=41):
    cfg = synth.NetConfig(name="adjgpu", M=M, P=P, n_vn=n_vn, K=K, uniform_all=False,
                          n_part=int(round(0.7 * K)), n_vn_t=int(round(0.2 * K)),
                          n_remote=K - int(round(0.7 * K)) - int(round(0.2 * K)), dmax=8, seed=seed,
                          dyn=synth.Dynamics(w_ext=89, drive_seed=4000 + seed))
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    part, _ = snn.snn_partition(net, P, "planted")
    rt = snn.Routing(net, part, P, n_vn, "contiguous")
    prm = snn.sim_params(cfg.dyn, raster_cap=M * T)
    a = snn.Adjoint(net, g.is_exc, rt, prm, snn.adjoint_params(T=T, ckpt_every=ckpt), device="cuda:0")
    onet = adj.from_synth(g, cfg.dyn, oracle.partition_planted(M, P), oracle.group_contiguous(P, n_vn),
                          oracle.alpha32(cfg.dyn.dt_ms, cfg.dyn.tau_ms))
    return a, onet, cfg, g, rt


def _params(n_pop, seed=3):
    rng = np.random.default_rng(seed)
    G = (1.0 + 0.25 * rng.standard_normal((n_pop, n_pop))).astype(np.float32)
    lam = (0.7 + 0.3 * rng.random(n_pop)).astype(np.float32)
    target = (0.0005 + 0.001 * rng.random(n_pop))
    return G, lam, target


def test_adjoint_forward_bit_exact_and_gradients(snn):
    a, onet, cfg, g, rt = _setup(snn)
    T = a.aparams.T
    G, lam, target = _params(a.n_pop)
    rates = a.forward(G, lam)
    tr = adj.forward_fp32(onet, G, lam, T)
    ts, ids = a.spikes_of_last_forward()
    ot, oi = np.nonzero(tr.spk)
    assert len(ts) == len(ot) and len(ts) > 100
    assert np.array_equal(ts * (1 << 32) + ids, np.sort(ot * (1 << 32) + oi))
    assert np.allclose(rates, tr.rates, rtol=1e-6, atol=0)
    grates = 2 * (tr.rates - target) / a.n_pop
    dG, dlam = a.backward(grates)
    oG, olam = adj.backward(onet, G, lam, tr, grates)
    scale = max(np.abs(oG).max(), np.abs(olam).max())
    err = max(np.abs(dG - oG).max(), np.abs(dlam - olam).max()) / scale
    print("adjoint relative error vs float64 oracle: %.3g" % err)
    assert err <= 1e-5
    assert np.abs(oG).max() > 0


def test_adjoint_checkpoint_interval_does_not_change_gradients(snn):
    grads = []
    for ckpt in (120, 7):
        a, onet, cfg, g, rt = _setup(snn, M=2048, K=40, T=120, ckpt=ckpt, seed=43)
        G, lam, target = _params(a.n_pop, seed=4)
        r = a.forward(G, lam)
        grads.append(a.backward(2 * (r.astype(np.float64) - target) / a.n_pop))
        a.close()
    assert np.allclose(grads[0][0], grads[1][0], rtol=1e-9, atol=1e-15)
    assert np.allclose(grads[0][1], grads[1][1], rtol=1e-9, atol=1e-15)


def test_autograd_function(snn):
    import torch
    a, onet, cfg, g, rt = _setup(snn, M=2048, K=40, T=80, ckpt=20, seed=47)
    G, lam, target = _params(a.n_pop, seed=5)
    Gt = torch.tensor(G, requires_grad=True)
    lt = torch.tensor(lam, requires_grad=True)
    f = snn.make_adjoint_function()
    rates = f.apply(Gt, lt, a)
    loss = ((rates - torch.tensor(target)) ** 2).sum() / a.n_pop
    loss.backward()
    dG, dlam = a.backward(2 * (rates.detach().numpy() - target) / a.n_pop)
    assert np.allclose(Gt.grad.numpy(), dG.astype(np.float32), rtol=1e-6)
    assert np.allclose(lt.grad.numpy(), dlam.astype(np.float32), rtol=1e-6)


def test_adjoint_config_size_against_float64_oracle(snn):
    """The adjoint workload's shape: 131,072 neurons, 8 partitions over 2 VNs,
    500 synapses per neuron (the scale locality mix), delays 1-8, membrane
    checkpoints every 50 steps; 200 steps (four checkpoint segments).  The
    forward bit-exact (every spike), the gradients within 1e-5 relative of
    the float64 oracle on the same trajectory."""
    T, CK = 200, 50
    a, onet, cfg, g, rt = _setup(snn, M=131072, P=8, n_vn=2, K=500, T=T, ckpt=CK, seed=4)
    G, lam, target = _params(a.n_pop, seed=6)
    rates = a.forward(G, lam)
    tr = adj.forward_fp32(onet, G, lam, T)
    ts, ids = a.spikes_of_last_forward()
    ot, oi = np.nonzero(tr.spk)
    assert len(ts) > 10000
    assert np.array_equal(ts * (1 << 32) + ids, np.sort(ot * (1 << 32) + oi))
    grates = 2 * (tr.rates - target) / a.n_pop
    dG, dlam = a.backward(grates)
    oG, olam = adj.backward(onet, G, lam, tr, grates)
    scale = max(np.abs(oG).max(), np.abs(olam).max())
    err = max(np.abs(dG - oG).max(), np.abs(dlam - olam).max()) / scale
    print("adjoint relative error vs float64 oracle at 131,072 neurons, %d steps: %.3g" % (T, err))
    assert err <= 1e-5
