"""Per-partition messages of the direct and the two-level route
(snn_routing_traffic): against the definitions written out here in numpy,
and in total against the message counts the oracle's sequential run
accumulates for the same spikes.  CPU only."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def snn():
    import paper_2205_07125_gb300 as m
    return m


def _definition(g, part, vn, relay_of, ids):
    """Messages per partition label, from the definitions."""
    P = int(part.max()) + 1
    out = {k: np.zeros(P, np.int64) for k in ("direct_out", "direct_in", "two_level_out", "two_level_in")}
    for i in ids:
        p = part[i]
        h = vn[p]
        Q = set(int(part[t]) for t in g.tgt[g.syn_ptr[i]:g.syn_ptr[i + 1]])
        for q in Q - {p}:
            out["direct_out"][p] += 1
            out["direct_in"][q] += 1
            if vn[q] == h:
                out["two_level_out"][p] += 1
                out["two_level_in"][q] += 1
        for gg in sorted(set(int(vn[q]) for q in Q) - {h}):
            r = relay_of(gg, p)
            out["two_level_out"][p] += 1
            out["two_level_in"][r] += 1
            for q in Q:
                if vn[q] == gg and q != r:
                    out["two_level_out"][r] += 1
                    out["two_level_in"][q] += 1
    return out


@pytest.mark.parametrize("mode", ["planted", "greedy"])
def test_traffic_against_definition_and_oracle_totals(snn, mode):
    cfg = synth.SCALE.scaled(M=4096, P=16, n_vn=4, K=40, n_part=28, n_vn_t=8, n_remote=4, seed=61,
                             dyn=synth.Dynamics(drive_lambda=0.8, w_ext=96, drive_seed=7))
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    part, _ = snn.snn_partition(net, cfg.P, mode, iters=2, seed=3)
    grouping = "contiguous" if mode == "planted" else "greedy"
    rt = snn.Routing(net, part, cfg.P, cfg.n_vn, grouping, iters=2, seed=3)
    vn, relay = rt.groups()
    s = cfg.P // cfg.n_vn
    members = [sorted(np.nonzero(vn == gg)[0].tolist()) for gg in range(cfg.n_vn)]
    # the relay of VN g for a source in VN h: the ((h - g) mod s)-th member of g in label order
    assert all(relay[gg, h] == members[gg][(h - gg) % s] for gg in range(cfg.n_vn) for h in range(cfg.n_vn))
    o = oracle.Oracle(g, cfg.P, part, cfg.n_vn, vn, cfg.dyn)
    r = o.run(150)
    ids = r["raster_ids"]
    assert len(ids) > 200
    got = rt.traffic(ids)
    want = _definition(g, part.astype(np.int64), vn.astype(np.int64), lambda gg, p: relay[gg, vn[p]], ids)
    for k in want:
        assert np.array_equal(got[k], want[k]), k
    c = o.count_dict()
    assert got["direct_out"].sum() == got["direct_in"].sum() == c["direct"]
    two = c["l1_xvn"] + c["l2_peer"] + c["l2_relay_remote"]
    assert got["two_level_out"].sum() == got["two_level_in"].sum() == two


def test_traffic_rejects_bad_ids(snn):
    g = synth.make_network(synth.TINY.scaled(M=256, K=8, seed=2))
    net = snn.Network.from_synth(g)
    part, _ = snn.snn_partition(net, 4, "planted")
    rt = snn.Routing(net, part, 4, 2)
    with pytest.raises(snn.SnnError):
        rt.traffic(np.array([3, 256], np.uint32))
    z = rt.traffic(np.zeros(0, np.uint32))
    assert all(v.sum() == 0 for v in z.values())


POLICIES = ("per_vn", "per_partition", "balanced")


def _hand_network():
    """4 planted partitions of 8 neurons in VNs {0, 1} and {2, 3}: 5 neurons of
    partition 2 and 3 of partition 3 reach partition 0 / 1 (VN 0); 2 neurons
    of partition 0 and 7 of partition 1 reach partitions 2 / 3 (VN 1)."""
    edges = [(16 + k, 0, 10, 1) for k in range(5)] + [(24 + k, 8, 10, 1) for k in range(3)]
    edges += [(k, 16, 10, 1) for k in range(2)] + [(8 + k, 24, 10, 1) for k in range(7)]
    return synth.make_edges(32, edges)


@pytest.mark.parametrize("policy,want", [
    # relay[g, p]: -1 inside the own VN
    ("per_vn", [[-1, -1, 1, 1], [3, 3, -1, -1]]),
    ("per_partition", [[-1, -1, 0, 1], [2, 3, -1, -1]]),
    # loads into VN 0: p2 5, p3 3 -> p2 to member 0, p3 to member 1;
    # into VN 1: p1 7, p0 2 -> p1 to member 0 (partition 2), p0 to member 1
    ("balanced", [[-1, -1, 0, 1], [3, 2, -1, -1]]),
])
def test_relay_policies_hand_worked(snn, policy, want):
    g = _hand_network()
    net = snn.Network.from_synth(g)
    part = oracle.partition_planted(32, 4)
    rt = snn.Routing(net, part, 4, 2, "contiguous", relay=policy)
    assert np.array_equal(rt.relays(), np.array(want, np.int32))
    o = oracle.Oracle(g, 4, part, 2, oracle.group_contiguous(4, 2), synth.TINY.dyn, relay=policy)
    assert np.array_equal(o.relay, np.array(want, np.int32))


@pytest.mark.parametrize("policy", POLICIES)
def test_relay_maps_library_equal_oracle(snn, policy):
    """Library and oracle compute each policy's relays independently; on a
    relabelled greedy mapping (labels not in VN order) they agree, also when
    the library derives another policy's map from a routing built with the
    default one."""
    cfg = synth.SCALE.scaled(M=6000, P=24, n_vn=4, K=30, n_part=21, n_vn_t=6, n_remote=3, seed=71)
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    part, _ = snn.snn_partition(net, cfg.P, "greedy", iters=2, seed=5)
    rt = snn.Routing(net, part, cfg.P, cfg.n_vn, "greedy", iters=2, seed=5, relay=policy)
    vn, _ = rt.groups()
    o = oracle.Oracle(g, cfg.P, part, cfg.n_vn, vn, cfg.dyn, relay=policy)
    assert np.array_equal(rt.relays(), o.relay)
    rt0 = snn.Routing(net, part, cfg.P, cfg.n_vn, "greedy", iters=2, seed=5)
    assert np.array_equal(rt0.relays(policy), o.relay)


@pytest.mark.parametrize("policy", POLICIES)
def test_traffic_under_each_policy(snn, policy):
    cfg = synth.SCALE.scaled(M=4096, P=16, n_vn=2, K=40, n_part=28, n_vn_t=8, n_remote=4, seed=63,
                             dyn=synth.Dynamics(drive_lambda=0.8, w_ext=96, drive_seed=8))
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    part = oracle.partition_planted(g.M, cfg.P)
    rt = snn.Routing(net, part, cfg.P, cfg.n_vn, relay=policy)
    vn, _ = rt.groups()
    o = oracle.Oracle(g, cfg.P, part, cfg.n_vn, vn, cfg.dyn, relay=policy)
    ids = o.run(150)["raster_ids"]
    assert len(ids) > 200
    got = rt.traffic(ids)
    want = _definition(g, part.astype(np.int64), vn.astype(np.int64), lambda gg, p: o.relay[gg, p], ids)
    for k in want:
        assert np.array_equal(got[k], want[k]), k
    c = o.count_dict()
    assert got["two_level_out"].sum() == c["l1_xvn"] + c["l2_peer"] + c["l2_relay_remote"]
    # the default routing computes the same traffic for this policy's relays
    rt0 = snn.Routing(net, part, cfg.P, cfg.n_vn)
    got0 = rt0.traffic(ids, policy)
    assert all(np.array_equal(got0[k], got[k]) for k in got)
