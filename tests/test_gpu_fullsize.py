"""Full-size parity: the benchmark workload (1,048,576 neurons, 64 partitions
over 16 VNs, 1.05e9 synapses) in the benchmark's launch configuration (32
steps per CUDA graph), every step of a 400-step run compared with the CPU
oracle: raster, per-step current and membrane hashes, current snapshots,
final membrane bits and refractory counters, message counts.  Also checks the
message counts against their closed forms at this size.

Slow (a few minutes: generating a billion synapses and running the
sequential oracle), so it runs only with the GPU tests.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_scale_workload_bit_exact():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_07125_gb300 as snn
    cfg = synth.SCALE
    T = 400
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    part, _ = snn.snn_partition(net, cfg.P, "planted")
    rt = snn.Routing(net, part, cfg.P, cfg.n_vn, "contiguous")
    rec = [0, 137, 250, 399]
    prm = snn.sim_params(cfg.dyn, raster_cap=4_000_000, raster_steps=T, hash_steps=T, cur_every=1,
                         cur_slots=T, steps_per_graph=32)
    sim = snn.Sim(net, rt, prm, device="cuda:0")
    sim.step(T)
    assert sim.sync_status() == 0
    ids, off = sim.read_raster(0, T)
    ch, vh = sim.read_hashes(0, T)
    cur = {s: sim.read_currents(s) for s in rec}
    V, ref, t = sim.read_state()
    counts = sim.read_counts()
    sim.close()
    del sim

    o = oracle.Oracle(g, cfg.P, oracle.partition_planted(g.M, cfg.P), cfg.n_vn,
                      oracle.group_contiguous(cfg.P, cfg.n_vn), cfg.dyn)
    r = o.run(T, rec_steps=rec, raster_cap=4_000_000)
    assert t == T
    assert np.array_equal(off, r["raster_off"])
    assert np.array_equal(ids, r["raster_ids"])
    assert np.array_equal(ch, r["cur_hash"]) and np.array_equal(vh, r["v_hash"])
    for s in rec:
        assert np.array_equal(cur[s], r["currents"][s]), s
    assert np.array_equal(V.view(np.uint32), o.V.view(np.uint32))
    assert np.array_equal(ref, o.ref)
    oc = o.count_dict()
    for k, v in counts.items():
        assert v == oc[k], (k, v, oc[k])
    # closed forms of the destinations reached per spike (uniform picks)
    S = counts["spikes"]
    assert S > 50_000
    s_ = cfg.vn_size
    rem_p = cfg.P - s_
    rem = rem_p * (1 - (1 - 1 / rem_p) ** cfg.n_remote)
    vns = (cfg.n_vn - 1) * (1 - (1 - 1 / (cfg.n_vn - 1)) ** cfg.n_remote)
    assert abs(counts["direct_xvn"] / S - rem) < 0.01 * rem
    assert abs(counts["l1_xvn"] / S - vns) < 0.01 * vns
    assert counts["events"] == S * cfg.K
    st = o.fp64_stats()
    assert st["max_rel_err"] <= 1e-5


def test_paper_share_workload_bit_exact():
    """The paper-shaped per-GPU share (5,000,000 neurons, 256 partitions over
    64 VNs, 5e9 synapses) in the benchmark's launch configuration (persistent
    kernel, neuron state in global memory at this size): 40 steps compared
    with the oracle step by step, plus the closed forms of the message counts."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_07125_gb300 as snn
    cfg = synth.PAPER_SHARE
    T = 40
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    part, _ = snn.snn_partition(net, cfg.P, "planted")
    rt = snn.Routing(net, part, cfg.P, cfg.n_vn, "contiguous")
    prm = snn.sim_params(cfg.dyn, raster_cap=2_000_000, raster_steps=T, hash_steps=T, cur_every=13,
                         cur_slots=4, steps_per_graph=32)
    sim = snn.Sim(net, rt, prm, device="cuda:0")
    sim.step(T)
    assert sim.sync_status() == 0
    ids, off = sim.read_raster(0, T)
    ch, vh = sim.read_hashes(0, T)
    cur = {s: sim.read_currents(s) for s in (13, 26, 39)}
    V, ref, t = sim.read_state()
    counts = sim.read_counts()
    sim.close()
    del sim, rt, net

    o = oracle.Oracle(g, cfg.P, oracle.partition_planted(g.M, cfg.P), cfg.n_vn,
                      oracle.group_contiguous(cfg.P, cfg.n_vn), cfg.dyn)
    r = o.run(T, rec_steps=[13, 26, 39], raster_cap=2_000_000)
    assert t == T
    assert np.array_equal(off, r["raster_off"])
    assert np.array_equal(ids, r["raster_ids"])
    assert np.array_equal(ch, r["cur_hash"]) and np.array_equal(vh, r["v_hash"])
    for s in (13, 26, 39):
        assert np.array_equal(cur[s], r["currents"][s]), s
    assert np.array_equal(V.view(np.uint32), o.V.view(np.uint32))
    assert np.array_equal(ref, o.ref)
    oc = o.count_dict()
    for k, v in counts.items():
        assert v == oc[k], (k, v, oc[k])
    S = counts["spikes"]
    assert S > 1000
    assert counts["events"] == S * cfg.K
