"""snn_deliver_spikes: a caller-given spike set routed through the two-level
route and fanned out, against a numpy brute-force fan-out of the same
synapse list."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_07125_gb300 as m
    return m


def _brute(g, ids, dmax):
    out = np.zeros((dmax, g.M), np.int64)
    for i in ids:
        a, b = g.syn_ptr[i], g.syn_ptr[i + 1]
        np.add.at(out, (g.d[a:b].astype(np.int64) - 1, g.tgt[a:b].astype(np.int64)),
                  g.w[a:b].astype(np.int64))
    return out


def _setup(snn, cfg, mode, **kw):
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    part, _ = snn.snn_partition(net, cfg.P, mode, iters=2, seed=3)
    rt = snn.Routing(net, part, cfg.P, cfg.n_vn, "greedy" if mode == "greedy" else "contiguous")
    sim = snn.Sim(net, rt, snn.sim_params(cfg.dyn, **kw), device="cuda:0")
    return g, rt, sim


@pytest.mark.parametrize("mode", ["planted", "greedy"])
def test_deliver_spikes_matches_brute_force(snn, mode):
    import torch
    cfg = synth.SCALE.scaled(M=1 << 13, seed=23)
    g, rt, sim = _setup(snn, cfg, mode)
    dmax = rt.info()["max_delay"]
    rng = np.random.default_rng(1)
    out = torch.zeros((dmax, g.M), dtype=torch.int32, device="cuda:0")
    total = np.zeros((dmax, g.M), np.int64)
    for n in (300, 1, 0, 2000):
        ids = rng.integers(0, g.M, n).astype(np.int32)
        if n > 2:
            ids[1] = ids[0]  # repeated source: delivered twice
        l1, l2, ev = sim.deliver_spikes(torch.from_numpy(ids).to("cuda:0"), out)
        total += _brute(g, ids, dmax)
        assert np.array_equal(out.cpu().numpy(), total)
        assert ev == cfg.K * n
    assert l2 > l1 > 0


def test_deliver_spikes_errors(snn):
    import torch
    cfg = synth.TINY
    g, rt, sim = _setup(snn, cfg, "planted", bucket_frac=0.01)
    out = torch.zeros((1, g.M), dtype=torch.int32, device="cuda:0")
    bad = torch.tensor([5, g.M], dtype=torch.int32, device="cuda:0")
    with pytest.raises(snn.SnnError) as e:
        sim.deliver_spikes(bad, out)
    assert e.value.code == -1
    many = torch.arange(g.M, dtype=torch.int32, device="cuda:0")
    with pytest.raises(snn.SnnError) as e:
        sim.deliver_spikes(many, out)
    assert e.value.code == snn.SNN_E_CAPACITY
    # the sim still steps normally afterwards
    sim.step(10)
    assert sim.sync_status() == 0
