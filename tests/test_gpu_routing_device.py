"""GPU table building (snn_routing_build_device) against the host builder:
every routing table byte for byte, the routing summary, the groups and the
connections, over planted and relabelled networks, contiguous and Algorithm 2
grouping, random mappings, neurons above the small sort's capacity, delays
up to 16, multapses, no synapses and the degenerate VN shapes; a simulation
on device-built tables equals one on host-built tables."""
import numpy as np
import pytest

import oracle
import synth
from _routing_defs import check_tables

pytestmark = pytest.mark.gpu

TABLES = ("syn_td", "syn_w", "csr", "l1_ptr", "l1_vn", "l1_l2", "l2", "l1_pair", "l2_pair", "bpair_ptr",
          "bpair_dst", "bpair_cap", "ipair_ptr", "ipair_dst", "ipair_cap", "bucket_cap", "inbox_cap", "perm_inv",
          "perm_fwd", "src_part", "pbase", "v0", "vn_of_part", "relay")


@pytest.fixture(scope="module")
def snn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_07125_gb300 as m
    return m


def _same(snn, g, part, P, n_vn, grouping="contiguous", relay="per_vn"):
    net = snn.Network.from_synth(g)
    h = snn.Routing(net, part, P, n_vn, grouping, iters=3, seed=5, relay=relay)
    d = snn.Routing(net, part, P, n_vn, grouping, iters=3, seed=5, build="device", device="cuda:0", relay=relay)
    assert np.array_equal(h.relays(), d.relays())
    for t in TABLES:
        a, b = h.export(t), d.export(t)
        assert a.shape == b.shape and np.array_equal(a.view(np.uint8), b.view(np.uint8)), t
    assert h.info() == d.info()
    for x, y in zip(h.groups(), d.groups()):
        assert np.array_equal(x, y)
    for x, y in zip(h.connections(), d.connections()):
        assert np.array_equal(x, y)
    return net, h, d


def _relabelled(g, seed):
    rng = np.random.default_rng(seed)
    perm = rng.permutation(g.M).astype(np.int64)
    src = np.repeat(np.arange(g.M), np.diff(g.syn_ptr))
    return synth.make_edges(g.M, list(zip(perm[src].tolist(), perm[g.tgt].tolist(), g.w.tolist(), g.d.tolist())),
                            v0=g.v0[np.argsort(perm)])


@pytest.mark.parametrize("grouping", ["contiguous", "greedy"])
def test_planted_network(snn, grouping):
    cfg = synth.NetConfig(name="t", M=6000, P=16, n_vn=4, K=40, uniform_all=False, n_part=28, n_vn_t=8,
                          n_remote=4, dmax=8, seed=17)
    g = synth.make_network(cfg)
    part, _ = snn.snn_partition(snn.Network.from_synth(g), 16, "planted")
    _same(snn, g, part, 16, 4, grouping)


@pytest.mark.parametrize("relay", ["per_partition", "balanced"])
def test_relay_policies(snn, relay):
    """The relay classes of the level-2 entries under each relay policy: the
    device-built tables equal the host builder's byte for byte."""
    cfg = synth.NetConfig(name="t", M=6000, P=16, n_vn=2, K=40, uniform_all=False, n_part=28, n_vn_t=8,
                          n_remote=4, dmax=8, seed=19)
    g = synth.make_network(cfg)
    part, _ = snn.snn_partition(snn.Network.from_synth(g), 16, "planted")
    _same(snn, g, part, 16, 2, "greedy", relay)


def test_relabelled_ids_random_mapping(snn):
    cfg = synth.NetConfig(name="t", M=4000, P=12, n_vn=3, K=30, uniform_all=False, n_part=20, n_vn_t=6,
                          n_remote=4, dmax=8, seed=23)
    g = _relabelled(synth.make_network(cfg), 3)
    net = snn.Network.from_synth(g)
    part, _ = snn.snn_partition(net, 12, "random", seed=9)
    _, h, _ = _same(snn, g, part, 12, 3, "greedy")
    assert not h.info()["identity_order"]


def test_large_degrees_delays_and_multapses(snn):
    """Out-degrees from 0 to 16384 (the small sort takes up to 1024), delays
    1..16, repeated synapses with equal and different weights."""
    rng = np.random.default_rng(4)
    M = 2000
    edges = []
    for i in range(M):
        k = int(rng.choice([0, 3, 40, 1023, 1024, 1025, 3000, 16384], p=[.05, .3, .4, .05, .05, .05, .05, .05]))
        if i % 97 == 0:
            k = 16384
        t = rng.integers(0, M, k)
        dl = rng.integers(1, 17, k)
        w = rng.integers(-300, 300, k)
        if k > 4:
            t[:4] = t[0]
            dl[:4] = dl[0]
            w[:2] = w[0]
        edges += list(zip([i] * k, t.tolist(), w.tolist(), dl.tolist()))
    g = synth.make_edges(M, edges)
    part = (np.arange(M) * 8 // M).astype(np.int32)
    _same(snn, g, part, 8, 4)
    _same(snn, g, np.random.default_rng(1).permutation(part).astype(np.int32), 8, 2, "greedy")


@pytest.mark.parametrize("P,n_vn", [(1, 1), (6, 6), (6, 1), (5, 5)])
def test_vn_shapes(snn, P, n_vn):
    cfg = synth.NetConfig(name="t", M=900, P=6, n_vn=2, K=16, uniform_all=True, seed=31)
    g = synth.make_network(cfg)
    part = (np.arange(g.M) * P // g.M).astype(np.int32)
    _same(snn, g, part, P, n_vn)


def test_no_synapses(snn):
    g = synth.make_edges(64, [])
    _same(snn, g, (np.arange(64) % 4).astype(np.int32), 4, 2)


def test_simulation_on_device_tables(snn):
    cfg = synth.NetConfig(name="t", M=8192, P=8, n_vn=2, K=100, uniform_all=False, n_part=70, n_vn_t=20,
                          n_remote=10, dmax=8, seed=41, dyn=synth.Dynamics(w_ext=96, drive_seed=7))
    g = _relabelled(synth.make_network(cfg), 8)
    net = snn.Network.from_synth(g)
    part, _ = snn.snn_partition(net, 8, "random", seed=2)
    _, h, d = _same(snn, g, part, 8, 2)
    out = []
    for rt in (h, d):
        sim = snn.Sim(net, rt, snn.sim_params(cfg.dyn, raster_cap=200000, raster_steps=300), device="cuda:0")
        sim.step(300)
        assert sim.sync_status() == 0
        out.append((sim.read_raster(0, 300), sim.read_counts()))
        sim.close()
    (ids_h, off_h), c_h = out[0]
    (ids_d, off_d), c_d = out[1]
    assert np.array_equal(off_h, off_d) and c_h == c_d and c_h["spikes"] > 0
    for t in range(300):
        assert np.array_equal(np.sort(ids_h[off_h[t]:off_h[t + 1]]), np.sort(ids_d[off_d[t]:off_d[t + 1]]))


def test_errors(snn):
    g = synth.make_edges(10, [(0, 1, 1, 1), (2, 12, 1, 1)])
    with pytest.raises(RuntimeError):
        snn.Routing(snn.Network.from_synth(g), np.zeros(10, np.int32), 1, 1, build="device", device="cuda:0")
    g = synth.make_edges(10, [(0, 1, 1, 1), (2, 3, 1, 17)])
    with pytest.raises(RuntimeError):
        snn.Routing(snn.Network.from_synth(g), np.zeros(10, np.int32), 1, 1, build="device", device="cuda:0")
    g = synth.make_edges(10, [(0, j % 10, 1, 1) for j in range(16385)])
    with pytest.raises(RuntimeError):
        snn.Routing(snn.Network.from_synth(g), np.zeros(10, np.int32), 1, 1, build="device", device="cuda:0")
    snn.Routing(snn.Network.from_synth(g), np.zeros(10, np.int32), 1, 1)  # the host builder takes it
    g = synth.make_edges(10, [(0, 1, 1, 1)])
    with pytest.raises(RuntimeError):  # partition 1 is empty
        snn.Routing(snn.Network.from_synth(g), np.zeros(10, np.int32), 2, 1, build="device", device="cuda:0")


def test_device_tables_follow_the_network(snn):
    """The device-built tables against their definitions rebuilt with numpy
    (not only against the host builder): internal order, sorted CSR, level-1
    and level-2 entries with relay classes and delay-1 counts, exchange pairs
    and capacities."""
    cfg = synth.NetConfig(name="t", M=1500, P=6, n_vn=3, K=18, uniform_all=False, n_part=10,
                          n_vn_t=5, n_remote=3, dmax=7, seed=12)
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    part = np.random.default_rng(3).permutation(oracle.partition_planted(g.M, 6)).astype(np.int32)
    rt = snn.Routing(net, part, 6, 3, "greedy", iters=2, seed=1, build="device", device="cuda:0")
    check_tables(rt, g, part, 6, 3)
