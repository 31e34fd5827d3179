"""GPU parity: the CUDA step (through the C ABI) against the CPU oracle.

Integer work (rasters, routes, message counts, int32 currents) must match
bit for bit, and so must the FP32 membrane (both sides use the same fixed
operation order with no fused multiply-add).  Where several results are
valid (the order of spikes inside a step, of bucket and inbox entries), the
comparison is on sorted multisets.
"""
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


def _oracle_mapping(g, cfg, part_mode, group_mode, P, n_vn, iters=3, seed=5):
    if part_mode == "planted":
        po = oracle.partition_planted(g.M, P)
    elif part_mode == "greedy":
        po, _ = oracle.partition_greedy(g, P, iters=iters, seed=seed)
    else:
        raise ValueError(part_mode)
    if group_mode == "contiguous":
        vn = oracle.group_contiguous(P, n_vn)
    else:
        vn, _ = oracle.group_greedy(g, po, P, n_vn, iters=iters, seed=seed)
    return po, vn


def _run_pair(snn, g, cfg, T, P, n_vn, part_mode="planted", group_mode="contiguous", cur_every=None,
              steps_per_graph=32, iters=3, seed=5, relay="per_vn", **prm_kw):
    net = snn.Network.from_synth(g)
    if part_mode == "planted":
        part, _ = snn.snn_partition(net, P, "planted")
    else:
        part, _ = snn.snn_partition(net, P, part_mode, iters=iters, seed=seed)
    rt = snn.Routing(net, part, P, n_vn, group_mode, iters=iters, seed=seed, relay=relay)
    ce = cur_every if cur_every is not None else max(1, T // 8)
    prm = snn.sim_params(cfg.dyn, raster_cap=max(4096, g.M * T // 10), raster_steps=T, hash_steps=T,
                         cur_every=ce, cur_slots=T // ce + 1, steps_per_graph=steps_per_graph,
                         **prm_kw)
    sim = snn.Sim(net, rt, prm, device="cuda:0")
    po, vn = _oracle_mapping(g, cfg, part_mode, group_mode, P, n_vn, iters, seed)
    assert np.array_equal(part, po)
    assert np.array_equal(rt.groups()[0], vn)
    o = oracle.Oracle(g, P, po, n_vn, vn, cfg.dyn, relay=relay)
    rec = list(range(0, T, ce))
    return sim, o, rec, rt


def _compare(sim, o, T, rec, t0=0):
    r = o.run(T, rec_steps=[t0 + s for s in rec], pairs=True)
    ids, off = sim.read_raster(t0, t0 + T)
    assert np.array_equal(off, r["raster_off"]), "raster offsets"
    assert np.array_equal(ids, r["raster_ids"]), "raster ids"
    ch, vh = sim.read_hashes(t0, t0 + T)
    assert np.array_equal(ch, r["cur_hash"]), "current hashes"
    assert np.array_equal(vh, r["v_hash"]), "membrane hashes"
    for s in rec:
        assert np.array_equal(sim.read_currents(t0 + s), r["currents"][t0 + s]), "currents at %d" % s
    V, ref, t = sim.read_state()
    assert t == o.t
    assert np.array_equal(V.view(np.uint32), o.V.view(np.uint32)), "membrane bits"
    assert np.array_equal(ref, o.ref), "refractory counters"
    c = sim.read_counts()
    oc = o.count_dict()
    for k in c:
        assert c[k] == oc[k], (k, c[k], oc[k])
    pairs = np.sort(sim.read_inbox_pairs())
    assert np.array_equal(pairs, r["pairs"]), "two-level inbox multiset vs direct route"
    return c, r


@pytest.fixture(params=["persistent", "persistent-global", "graph", "persistent-deferred",
                        "persistent-arrival", "persistent-global-arrival", "graph-arrival", "persistent-owner"])
def path(request, monkeypatch):
    """Run a test on the persistent kernel (neuron state resident in shared
    memory where it fits, or read from global memory every step; with
    minimum-delay batching of the delay >= 2 synapses) and on the CUDA-graph
    path, each with delivery into the delay ring or by arrival step."""
    p = request.param
    monkeypatch.setenv("SNN_PERSIST", "0" if p.startswith("graph") else "1")
    monkeypatch.setenv("SNN_PERSIST_SMEM", "0" if p.startswith("persistent-global") else "1")
    monkeypatch.setenv("SNN_PERSIST_DEFER", "1" if p == "persistent-deferred" else "0")
    monkeypatch.setenv("SNN_DELIVERY", "1" if p.endswith("arrival") else "3" if p.endswith("owner") else "0")
    return p


def test_tiny_full_run(snn, path):
    """4,096 neurons, 4 partitions over 2 VNs, 1,000 steps: everything bit-exact."""
    cfg = synth.TINY
    g = synth.make_network(cfg)
    sim, o, rec, _ = _run_pair(snn, g, cfg, cfg.steps, cfg.P, cfg.n_vn, cur_every=50)
    assert (sim.launches(10) == 1) == path.startswith("persistent")
    sim.step(cfg.steps)
    c, _ = _compare(sim, o, cfg.steps, rec)
    assert sim.sync_status() == 0
    assert c["spikes"] > 1000 and c["events"] == c["spikes"] * cfg.K
    st = o.fp64_stats()
    assert st["max_rel_err"] <= 1e-5


def test_tiny_greedy_partition_and_grouping(snn, path):
    """Algorithm 1 + Algorithm 2 mapping: neurons reordered internally, ids stay global."""
    cfg = synth.TINY
    g = synth.make_network(cfg)
    sim, o, rec, rt = _run_pair(snn, g, cfg, 300, cfg.P, cfg.n_vn, "greedy", "greedy")
    assert rt.info()["identity_order"] == 0
    sim.step(300)
    _compare(sim, o, 300, rec)


@pytest.mark.parametrize("spg", [1, 7, 32])
def test_locality_delays_several_tiles(snn, spg, path):
    """Locality mix and delays 1..8 over 64 partitions / 16 VNs, several graph unrollings."""
    cfg = synth.SCALE.scaled(M=1 << 16, seed=41)
    g = synth.make_network(cfg)
    sim, o, rec, _ = _run_pair(snn, g, cfg, 150, cfg.P, cfg.n_vn, steps_per_graph=spg)
    sim.step(150)
    _compare(sim, o, 150, rec)


def test_ragged_sizes_and_uneven_partitions(snn, path):
    """M not a multiple of the block size, uneven greedy partitions, 3 VNs of 1
    (partition-owned delivery needs M % 4 == 0 and reports SNN_E_RANGE)."""
    if path == "persistent-owner":
        cfg = synth.NetConfig(name="ragged", M=1007, P=3, n_vn=3, K=37, uniform_all=True, dmax=4, seed=99)
        g = synth.make_network(cfg)
        net = snn.Network.from_synth(g)
        part, _ = snn.snn_partition(net, 3, "greedy", iters=3, seed=5)
        rt = snn.Routing(net, part, 3, 3)
        with pytest.raises(snn.SnnError) as e:
            snn.Sim(net, rt, snn.sim_params(cfg.dyn), device="cuda:0")
        assert e.value.code == -5
        return
    cfg = synth.NetConfig(name="ragged", M=1000 + 7, P=3, n_vn=3, K=37, uniform_all=True, dmax=4,
                          seed=99, dyn=synth.Dynamics(drive_lambda=1.1, w_ext=120, drive_seed=9))
    g = synth.make_network(cfg)
    sim, o, rec, _ = _run_pair(snn, g, cfg, 200, 3, 3, "greedy", "contiguous")
    sim.step(200)
    _compare(sim, o, 200, rec)


def test_degenerate_networks(snn):
    """No synapses at all; one partition and one VN; a silent network."""
    g = synth.make_edges(300, [], v0=np.linspace(-70, -45, 300).astype(np.float32))
    cfg = synth.NetConfig(name="iso", M=300, P=1, n_vn=1, K=0, uniform_all=True,
                          dyn=synth.Dynamics(drive_lambda=0.5, w_ext=200))
    sim, o, rec, _ = _run_pair(snn, g, cfg, 64, 1, 1)
    sim.step(64)
    c, _ = _compare(sim, o, 64, rec)
    assert c["events"] == 0 and c["spikes"] > 0
    silent = synth.TINY.scaled(dyn=synth.Dynamics(drive_lambda=0.0))
    g2 = synth.make_network(silent.scaled(M=512, seed=3))
    g2.v0[:] = -65.0
    sim2, o2, rec2, _ = _run_pair(snn, g2, silent, 40, 4, 2)
    sim2.step(40)
    c2, _ = _compare(sim2, o2, 40, rec2)
    assert c2["spikes"] == 0


@pytest.mark.parametrize("group_mode", ["contiguous", "greedy"])
def test_raster_of_wide_steps(snn, group_mode):
    """A step with more spikes than the device-side raster sort takes (all
    20,000 neurons start above threshold, so step 0 has 20,000 spikes) comes
    back sorted by global id, in the identity and in a permuted internal
    order, beside steps the device sorts."""
    M = 20000
    g = synth.make_edges(M, [], v0=np.full(M, -45.0, np.float32))
    cfg = synth.NetConfig(name="burst", M=M, P=4, n_vn=2, K=0, uniform_all=True,
                          dyn=synth.Dynamics(drive_lambda=0.5, w_ext=200))
    sim, o, rec, _ = _run_pair(snn, g, cfg, 48, 4, 2, group_mode=group_mode)
    sim.step(48)
    c, _ = _compare(sim, o, 48, rec)
    ids, off = sim.read_raster(0, 48)
    assert off[1] - off[0] == M and c["spikes"] >= M


def test_step_in_chunks_equals_one_call(snn, path):
    cfg = synth.TINY
    g = synth.make_network(cfg)
    sim, o, rec, _ = _run_pair(snn, g, cfg, 200, cfg.P, cfg.n_vn, steps_per_graph=16)
    for T in (1, 15, 16, 33, 135):
        sim.step(T)
    _compare(sim, o, 200, rec)


def test_capacity_overflow_is_reported(snn):
    """Buckets far below their worst case overflow; the status says so, nothing faults."""
    cfg = synth.TINY
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    rt = snn.Routing(net, oracle.partition_planted(g.M, 4), 4, 2)
    prm = snn.sim_params(cfg.dyn, bucket_frac=0.0005, inbox_frac=1.0)
    sim = snn.Sim(net, rt, prm, device="cuda:0")
    sim.step(100)
    assert sim.sync_status() == snn.SNN_E_CAPACITY
    prm = snn.sim_params(cfg.dyn, bucket_frac=1.0, inbox_frac=0.0005)
    sim = snn.Sim(net, rt, prm, device="cuda:0")
    sim.step(100)
    assert sim.sync_status() == snn.SNN_E_CAPACITY
    prm = snn.sim_params(cfg.dyn)
    sim = snn.Sim(net, rt, prm, device="cuda:0")
    sim.step(100)
    assert sim.sync_status() == 0


def test_checkpoint_resume_bit_exact(snn, path):
    cfg = synth.SCALE.scaled(M=1 << 15, seed=17)
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    rt = snn.Routing(net, oracle.partition_planted(g.M, cfg.P), cfg.P, cfg.n_vn)
    prm = snn.sim_params(cfg.dyn, hash_steps=400)
    sim = snn.Sim(net, rt, prm, device="cuda:0")
    sim.step(150)
    blob = sim.save_state()
    sim.step(200)
    a = sim.read_hashes(150, 350)
    ca = sim.read_counts()
    Va, _, _ = sim.read_state()
    sim.load_state(blob)
    sim.step(200)
    b = sim.read_hashes(150, 350)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    Vb, _, t = sim.read_state()
    assert t == 350 and np.array_equal(Va.view(np.uint32), Vb.view(np.uint32))
    assert sim.read_counts() == ca


def test_reset_replays_identically(snn):
    cfg = synth.TINY
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    rt = snn.Routing(net, oracle.partition_planted(g.M, 4), 4, 2)
    prm = snn.sim_params(cfg.dyn, raster_cap=100000, raster_steps=300, hash_steps=300)
    sim = snn.Sim(net, rt, prm, device="cuda:0")
    sim.step(300)
    a = sim.read_raster(0, 300), sim.read_hashes(0, 300), sim.read_counts()
    sim.reset(reupload=True)
    sim.step(300)
    b = sim.read_raster(0, 300), sim.read_hashes(0, 300), sim.read_counts()
    assert np.array_equal(a[0][0], b[0][0]) and np.array_equal(a[1][0], b[1][0]) and a[2] == b[2]


def test_barrier_wait_is_bounded(snn, monkeypatch):
    """A grid barrier whose wait cannot complete gives up and reports a timeout.

    Block 0 skips its first arrival (test switch), so the other blocks' wait
    runs out after the shortened bound; the host reads SNN_E_TIMEOUT and the
    context stays usable: a reset sim steps correctly afterwards.
    """
    monkeypatch.setenv("SNN_PERSIST", "1")
    monkeypatch.setenv("SNN_BARRIER_LIMIT_NS", "20000000")  # 20 ms
    monkeypatch.setenv("SNN_TEST_SKIP_BARRIER", "1")
    cfg = synth.TINY
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    rt = snn.Routing(net, oracle.partition_planted(g.M, 4), 4, 2)
    sim = snn.Sim(net, rt, snn.sim_params(cfg.dyn), device="cuda:0")
    if sim.launches(10) != 1:
        pytest.skip("no cooperative launch on this device")
    sim.step(50)
    assert sim.sync_status() == -8  # SNN_E_TIMEOUT
    _, _, t = sim.read_state()
    assert t < 50
    monkeypatch.delenv("SNN_TEST_SKIP_BARRIER")
    sim.reset()
    sim.step(20)
    assert sim.sync_status() == 0
    _, _, t = sim.read_state()
    assert t == 20


@pytest.mark.parametrize("groups", [4, 16])
def test_two_level_barrier_bit_exact(snn, monkeypatch, groups):
    """The two-level grid-barrier arrival (blocks arrive on group words, the
    last of a group forwards one arrival and the group's spike count) gives
    the oracle's spikes, currents and counts on every persistent shape, and a
    block that never arrives still ends in a reported timeout."""
    monkeypatch.setenv("SNN_PERSIST", "1")
    monkeypatch.setenv("SNN_BAR_GROUPS", str(groups))
    cfg = synth.SCALE.scaled(M=1 << 16, seed=43)
    g = synth.make_network(cfg)
    for smem in ("1", "0"):
        monkeypatch.setenv("SNN_PERSIST_SMEM", smem)
        sim, o, rec, _ = _run_pair(snn, g, cfg, 120, cfg.P, cfg.n_vn)
        if sim.launches(10) != 1:
            pytest.skip("no cooperative launch on this device")
        sim.step(120)
        _compare(sim, o, 120, rec)
    monkeypatch.setenv("SNN_BARRIER_LIMIT_NS", "20000000")  # 20 ms
    monkeypatch.setenv("SNN_TEST_SKIP_BARRIER", "1")
    net = snn.Network.from_synth(synth.make_network(synth.TINY))
    rt = snn.Routing(net, oracle.partition_planted(synth.TINY.M, 4), 4, 2)
    sim = snn.Sim(net, rt, snn.sim_params(synth.TINY.dyn), device="cuda:0")
    sim.step(50)
    assert sim.sync_status() == -8  # SNN_E_TIMEOUT


def test_autotune_keeps_results(snn):
    """The autotuner tries every launch shape from the initial state, keeps the
    fastest and leaves the sim in its initial state: the run after it is the
    oracle's run."""
    cfg = synth.SCALE.scaled(M=16384, P=16, n_vn=4, K=200, n_part=140, n_vn_t=40, n_remote=20, steps=200)
    g = synth.make_network(cfg)
    sim, o, rec, _ = _run_pair(snn, g, cfg, 200, cfg.P, cfg.n_vn, delivery=snn.SNN_DELIVER_AUTO)
    choice, ms = sim.autotune(40)
    assert ms > 0 and (choice % 1000 == 0 or choice % 100 in (1, 2, 3, 4))
    sim.step(200)
    _compare(sim, o, 200, rec)
    assert sim.sync_status() == 0


def test_autotune_mid_run_keeps_state_and_records(snn, monkeypatch):
    """The autotuner called after 120 steps times every shape (ring, arrival,
    owner, graph) from that state and leaves the sim there with its records:
    the 260 steps (120 before, 140 after) are the oracle's run."""
    monkeypatch.delenv("SNN_DELIVERY", raising=False)
    cfg = synth.SCALE.scaled(M=16384, P=16, n_vn=4, K=200, n_part=140, n_vn_t=40, n_remote=20, seed=29)
    g = synth.make_network(cfg)
    sim, o, rec, _ = _run_pair(snn, g, cfg, 260, cfg.P, cfg.n_vn, cur_every=20, delivery=snn.SNN_DELIVER_AUTO)
    sim.step(120)
    choice, ms = sim.autotune(30)
    assert ms > 0
    sim.step(140)
    assert sim.sync_status() == 0
    _compare(sim, o, 260, rec)


def test_checkpoint_across_delivery_modes(snn, monkeypatch):
    """A checkpoint holds the delay-ring form of the state whatever the
    delivery: saved under delivery by arrival step (queued runs and the input
    slot moved into the ring) and restored into a ring sim, and the other way
    round, the run continues as the uninterrupted one, bit for bit."""
    monkeypatch.delenv("SNN_DELIVERY", raising=False)
    cfg = synth.SCALE.scaled(M=1 << 15, seed=19)
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    rt = snn.Routing(net, oracle.partition_planted(g.M, cfg.P), cfg.P, cfg.n_vn)
    for src_mode, dst_mode in ((snn.SNN_DELIVER_ARRIVAL, snn.SNN_DELIVER_RING),
                               (snn.SNN_DELIVER_RING, snn.SNN_DELIVER_ARRIVAL),
                               (snn.SNN_DELIVER_ARRIVAL, snn.SNN_DELIVER_OWNER),
                               (snn.SNN_DELIVER_OWNER, snn.SNN_DELIVER_RING)):
        a = snn.Sim(net, rt, snn.sim_params(cfg.dyn, hash_steps=400, delivery=src_mode), device="cuda:0")
        a.step(150)
        blob = a.save_state()
        a.step(200)
        ha = a.read_hashes(150, 350)
        Va, ra, _ = a.read_state()
        ca = a.read_counts()
        b = snn.Sim(net, rt, snn.sim_params(cfg.dyn, hash_steps=400, delivery=dst_mode), device="cuda:0")
        b.load_state(blob)
        b.step(200)
        hb = b.read_hashes(150, 350)
        Vb, rb, t = b.read_state()
        assert t == 350
        assert np.array_equal(ha[0], hb[0]) and np.array_equal(ha[1], hb[1]), (src_mode, dst_mode)
        assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32)) and np.array_equal(ra, rb)
        assert b.read_counts() == ca
        for s in (a, b):
            assert s.sync_status() == 0
            s.close()


def test_arrival_list_overflow_is_reported(snn, monkeypatch):
    """Arrival lists far below their worst case overflow: the status says so,
    nothing faults; at the exact worst case the run is clean."""
    monkeypatch.delenv("SNN_DELIVERY", raising=False)
    cfg = synth.SCALE.scaled(M=1 << 14, P=16, n_vn=4, K=200, n_part=140, n_vn_t=40, n_remote=20, seed=23)
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    rt = snn.Routing(net, oracle.partition_planted(g.M, cfg.P), cfg.P, cfg.n_vn)
    for mode in (snn.SNN_DELIVER_ARRIVAL, snn.SNN_DELIVER_OWNER):
        sim = snn.Sim(net, rt, snn.sim_params(cfg.dyn, delivery=mode, arrival_frac=1e-5), device="cuda:0")
        sim.step(100)
        assert sim.sync_status() == snn.SNN_E_CAPACITY, mode
        sim.close()
    sim = snn.Sim(net, rt, snn.sim_params(cfg.dyn, delivery=snn.SNN_DELIVER_ARRIVAL), device="cuda:0")
    sim.step(100)
    assert sim.sync_status() == 0
    assert sim.read_counts()["spikes"] > 0


@pytest.mark.parametrize("delivery", [0, 1, 3])
def test_abi_built_model_against_oracle_reading_its_file(snn, tmp_path, monkeypatch, delivery):
    """The whole boundary: the network built behind the C ABI
    (snn_model_build), written as an edge-list file (snn_model_save) that the
    oracle reads with its own reader, partitioned, routed and stepped on the
    GPU; 300 steps bit-exact against the oracle of the file's network."""
    monkeypatch.delenv("SNN_DELIVERY", raising=False)
    mp = snn.model_params("scale", n_neurons=32768, n_parts=16, vn_size=4, syn_per_neuron=300,
                          n_same_part=210, n_same_vn=60, n_remote=30, seed=2024)
    m = snn.Model.build(mp)
    path = str(tmp_path / "model.snnm")
    m.save(path)
    f = oracle.load_model(path)
    net = m.network()
    P, n_vn, T = 16, 4, 300
    part, _ = snn.snn_partition(net, P, "planted")
    rt = snn.Routing(net, part, P, n_vn, "contiguous")
    dyn = synth.SCALE.dyn
    prm = snn.sim_params(dyn, raster_cap=f.M * T // 10, raster_steps=T, hash_steps=T, cur_every=50, cur_slots=6,
                         delivery=delivery)
    sim = snn.Sim(net, rt, prm, device="cuda:0")
    o = oracle.Oracle(f, P, oracle.partition_planted(f.M, P), n_vn, oracle.group_contiguous(P, n_vn), dyn)
    sim.step(T)
    assert sim.sync_status() == 0
    c, _ = _compare(sim, o, T, list(range(0, T, 50)))
    assert c["spikes"] > 1000 and c["events"] == c["spikes"] * 300


@pytest.mark.parametrize("relay", ["per_partition", "balanced"])
def test_relay_policies_counts_and_currents(snn, relay):
    """Relays chosen per source partition or by load balancing change which
    level-2 entries are forwarded (the message classes), not the delivery:
    counts under the policy and currents bit-exact against the oracle under
    the same policy, on a greedy mapping."""
    cfg = synth.SCALE.scaled(M=1 << 15, P=32, n_vn=4, K=200, n_part=140, n_vn_t=40, n_remote=20, seed=47)
    g = synth.make_network(cfg)
    sim, o, rec, rt = _run_pair(snn, g, cfg, 120, cfg.P, cfg.n_vn, "greedy", "greedy", relay=relay)
    assert np.array_equal(rt.relays(), o.relay)
    sim.step(120)
    c, _ = _compare(sim, o, 120, rec)
    assert c["l2_relay_remote"] > 0
