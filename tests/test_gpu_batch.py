"""GPU parity of batches: independent networks of uneven sizes concatenated
and stepped by one sim (one persistent launch, or one graph, per snn_step)
against one CPU oracle per network.  Each network has its own drive
(Poisson rate and Philox stream); its spikes, currents, final state and
message counts must equal those of the network simulated alone."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_07125_gb300 as m
    return m


@pytest.fixture(params=["persistent", "persistent-global", "graph", "persistent-deferred",
                        "persistent-arrival", "persistent-global-arrival", "graph-arrival", "persistent-owner"])
def path(request, monkeypatch):
    p = request.param
    monkeypatch.setenv("SNN_PERSIST", "0" if p.startswith("graph") else "1")
    monkeypatch.setenv("SNN_PERSIST_SMEM", "0" if p.startswith("persistent-global") else "1")
    monkeypatch.setenv("SNN_PERSIST_DEFER", "1" if p == "persistent-deferred" else "0")
    monkeypatch.setenv("SNN_DELIVERY", "1" if p.endswith("arrival") else "3" if p.endswith("owner") else "0")
    return p


def _batch_run(snn, b, T, rec):
    net = snn.Network.from_synth(b.net)
    rt = snn.Routing(net, b.part, b.P, b.n_vn, "contiguous")
    plist = [snn.sim_params(c.dyn, raster_cap=b.net.M * T // 5 + 4096, raster_steps=T, cur_every=rec[1],
                            cur_slots=len(rec), steps_per_graph=16) for c in b.cfgs]
    sim = snn.Sim(net, rt, plist[0], device="cuda:0", batch=(b.off, plist))
    sim.step(T)
    assert sim.sync_status() == 0
    out = {"raster": sim.read_raster(0, T), "cur": {s: sim.read_currents(s) for s in rec},
           "state": sim.read_state(), "counts": sim.read_counts(), "launches": sim.launches(T)}
    sim.close()
    return out


def _check(b, out, T, rec):
    ids, off = out["raster"]
    V, ref, t = out["state"]
    assert t == T
    tot = {}
    for k, (c, g) in enumerate(zip(b.cfgs, b.nets)):
        a, e = int(b.off[k]), int(b.off[k + 1])
        o = oracle.Oracle(g, c.P, oracle.partition_planted(g.M, c.P), c.n_vn,
                          oracle.group_contiguous(c.P, c.n_vn), c.dyn)
        r = o.run(T, rec_steps=rec, raster_cap=g.M * T // 5 + 4096)
        for s in range(T):
            step = ids[off[s]:off[s + 1]]
            mine = step[(step >= a) & (step < e)] - a
            ref_ids = r["raster_ids"][r["raster_off"][s]:r["raster_off"][s + 1]]
            assert np.array_equal(mine, ref_ids), (k, s)
        for s in rec:
            assert np.array_equal(out["cur"][s][a:e], r["currents"][s]), (k, s)
        assert np.array_equal(V[a:e].view(np.uint32), o.V.view(np.uint32)), k
        assert np.array_equal(ref[a:e], o.ref), k
        for key, v in o.count_dict().items():
            tot[key] = tot.get(key, 0) + v
    tot["steps"] = T  # one step of the batch steps every network
    for key, v in out["counts"].items():
        assert v == tot[key], (key, v, tot[key])
    return tot


def test_batch_uneven_networks(snn, path):
    """Six networks of 600-6,000 neurons, 4-8 partitions, out-degree 12-60,
    drives of 5-15 Hz scaled, 240 steps."""
    cfgs = synth.batch_configs(n=6, seed=91, m_lo=600, m_hi=6000, k_lo=12, k_hi=60, p_lo=4, p_hi=8)
    b = synth.make_batch(cfgs)
    T, rec = 240, [0, 60, 120, 180]
    out = _batch_run(snn, b, T, rec)
    assert (out["launches"] == 1) == path.startswith("persistent")
    tot = _check(b, out, T, rec)
    assert tot["spikes"] > 100


def test_batch_of_one_equals_plain_sim(snn):
    """A batch of one network is the plain sim of that network."""
    cfgs = synth.batch_configs(n=1, seed=5, m_lo=3000, m_hi=3000, k_lo=30, k_hi=30, p_lo=4, p_hi=4)
    b = synth.make_batch(cfgs)
    T = 150
    net = snn.Network.from_synth(b.net)
    rt = snn.Routing(net, b.part, b.P, b.n_vn, "contiguous")
    prm = snn.sim_params(cfgs[0].dyn, raster_cap=100000, raster_steps=T, hash_steps=T)
    s1 = snn.Sim(net, rt, prm, device="cuda:0")
    s1.step(T)
    s2 = snn.Sim(net, rt, prm, device="cuda:0", batch=(b.off, [prm]))
    s2.step(T)
    for s in (s1, s2):
        assert s.sync_status() == 0
    a, b_ = s1.read_raster(0, T), s2.read_raster(0, T)
    assert np.array_equal(a[0], b_[0]) and np.array_equal(a[1], b_[1])
    assert np.array_equal(s1.read_hashes(0, T)[1], s2.read_hashes(0, T)[1])
    assert s1.read_counts() == s2.read_counts()


def test_batch_at_workload_sizes_autotuned(snn):
    """Eight networks drawn from the batched workload's distribution at its
    sizes (12k-441k neurons, 304-825 synapses per neuron, 4-30 partitions,
    1.1M neurons and 6.2e8 synapses in all), stepped 100 steps in the launch
    shape the autotuner picks; every network against its own oracle."""
    cfgs = synth.batch_configs(n=8, seed=3000)
    b = synth.make_batch(cfgs)
    assert min(c.M for c in cfgs) < 20_000 and max(c.M for c in cfgs) > 400_000
    T, rec = 100, [0, 33, 66, 99]
    net = snn.Network.from_synth(b.net)
    rt = snn.Routing(net, b.part, b.P, b.n_vn, "contiguous")
    plist = [snn.sim_params(c.dyn, raster_cap=b.net.M * T // 5 + 4096, raster_steps=T, cur_every=33,
                            cur_slots=len(rec), steps_per_graph=32) for c in b.cfgs]
    sim = snn.Sim(net, rt, plist[0], device="cuda:0", batch=(b.off, plist))
    choice, _ = sim.autotune(40)
    sim.step(T)
    assert sim.sync_status() == 0
    out = {"raster": sim.read_raster(0, T), "cur": {s: sim.read_currents(s) for s in rec},
           "state": sim.read_state(), "counts": sim.read_counts()}
    sim.close()
    print("autotuned shape %d" % choice)
    tot = _check(b, out, T, rec)
    assert tot["spikes"] > 10_000
