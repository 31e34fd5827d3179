"""CPU tests of the library: the C ABI loads and exports every declared call,
and the host-side setup (Algorithm 1 partition, Algorithm 2 grouping, relay
map, routing-table sizes, static connections, argument checks) agrees with
the oracle's independent readings and with brute force."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth
from _routing_defs import check_tables

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def snn():
    import __graft_entry__
    __graft_entry__._load_builder().build()
    import paper_2205_07125_gb300 as m
    return m


def test_library_exports_every_declared_call(snn):
    hdr = open(os.path.join(ROOT, "include", "snn.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b(snn_[a-z0-9_]+)\s*\(", hdr))
    assert len(names) >= 20
    lib = ctypes.CDLL(snn.library_path())
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(snn.EXPORTS) == names


def test_strerror_names_codes(snn):
    for code in range(0, -9, -1):
        s = snn._lib_strerror(code).decode()
        assert s and s != "unknown error"


@pytest.mark.parametrize("kind", ["cliques", "planted", "uniform"])
def test_greedy_partition_equals_oracle(snn, kind):
    if kind == "cliques":
        edges = [(b + i, b + j, 1, 1) for b in (0, 6, 12) for i in range(6) for j in range(6) if i != j]
        edges += [(2, 9, 1, 1), (10, 15, 1, 1)]
        g = synth.make_edges(18, edges)
        P = 3
    elif kind == "planted":
        g = synth.make_network(synth.NetConfig(name="t", M=1536, P=6, n_vn=3, K=20, uniform_all=False,
                                               n_part=14, n_vn_t=4, n_remote=2, seed=5))
        P = 6
    else:
        g = synth.make_network(synth.NetConfig(name="t", M=700, P=4, n_vn=2, K=9, uniform_all=True,
                                               seed=8))
        P = 5
    net = snn.Network.from_synth(g)
    for iters, seed in ((1, 3), (4, 11)):
        mine, st = snn.snn_partition(net, P, "greedy", iters=iters, seed=seed)
        ref, obj = oracle.partition_greedy(g, P, iters=iters, seed=seed)
        assert np.array_equal(mine, ref)
        assert st["objective"] == obj


def test_planted_and_random_partitions(snn):
    g = synth.make_network(synth.NetConfig(name="t", M=1003, P=7, n_vn=7, K=5, uniform_all=True))
    net = snn.Network.from_synth(g)
    pl, _ = snn.snn_partition(net, 7, "planted")
    assert np.array_equal(pl, oracle.partition_planted(1003, 7))
    rnd, st = snn.snn_partition(net, 7, "random", seed=3)
    sizes = np.bincount(rnd, minlength=7)
    assert sizes.max() - sizes.min() <= 1
    assert not np.array_equal(rnd, pl)
    assert st["objective"] == oracle.cut(g, rnd)


def _brute_tables(g, part, vn):
    """Distinct destination VNs / partitions per neuron and static connections."""
    P = int(part.max()) + 1
    n_vn = int(vn.max()) + 1
    n_l1 = n_l2 = 0
    bcap = np.zeros(n_vn, np.int64)
    icap = np.zeros(P, np.int64)
    conn = np.zeros((P, P), bool)
    for i in range(g.M):
        Q = {int(part[j]) for j in g.tgt[g.syn_ptr[i]:g.syn_ptr[i + 1]]}
        G = {int(vn[q]) for q in Q}
        n_l1 += len(G)
        n_l2 += len(Q)
        for q in Q:
            icap[q] += 1
            conn[part[i], q] = True
        for x in G:
            bcap[x] += 1
    direct = np.zeros(P, np.int64)
    two = np.zeros(P, np.int64)
    for p in range(P):
        qs = [q for q in range(P) if q != p and conn[p, q]]
        direct[p] = len(qs)
        two[p] = sum(1 for q in qs if vn[q] == vn[p]) + len({int(vn[q]) for q in qs if vn[q] != vn[p]})
    return n_l1, n_l2, direct, two


@pytest.mark.parametrize("grouping", ["contiguous", "greedy"])
def test_routing_tables_and_groups(snn, grouping):
    cfg = synth.NetConfig(name="t", M=2048, P=8, n_vn=4, K=24, uniform_all=False, n_part=12,
                          n_vn_t=8, n_remote=4, dmax=5, seed=31)
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    part = oracle.partition_planted(g.M, 8)
    perm = np.array([5, 2, 7, 0, 3, 6, 1, 4], np.int32)
    part = perm[part]  # labels not aligned with the planted groups
    rt = snn.Routing(net, part, 8, 4, grouping, iters=3, seed=9, n_threads=3)
    vn, relay = rt.groups()
    if grouping == "greedy":
        ovn, ocost = oracle.group_greedy(g, part, 8, 4, iters=3, seed=9)
        assert np.array_equal(vn, ovn)
        assert rt.info()["group_cost"] == ocost
    else:
        assert np.array_equal(vn, oracle.group_contiguous(8, 4))
    # relay: ((h - g) mod s)-th member of group g in ascending label order
    s = 2
    for gg in range(4):
        members = sorted(q for q in range(8) if vn[q] == gg)
        for h in range(4):
            assert relay[gg, h] == members[(h - gg) % s]
    info = rt.info()
    n_l1, n_l2, direct, two = _brute_tables(g, part, vn)
    assert info["n_l1"] == n_l1 and info["n_l2"] == n_l2
    assert info["max_delay"] == 5 and info["n_synapses"] == g.E
    cd, ct = rt.connections()
    assert np.array_equal(cd, direct) and np.array_equal(ct, two)
    assert info["conn_direct_sum"] == direct.sum() and info["conn_two_level_sum"] == two.sum()
    assert info["identity_order"] == 0  # relabelled partitions reorder the neurons


def test_routing_thread_count_does_not_change_tables(snn):
    cfg = synth.NetConfig(name="t", M=3000, P=6, n_vn=2, K=15, uniform_all=False, n_part=9,
                          n_vn_t=4, n_remote=2, dmax=3, seed=4)
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    part = oracle.partition_planted(g.M, 6)
    a = snn.Routing(net, part, 6, 2, "greedy", n_threads=1).info()
    b = snn.Routing(net, part, 6, 2, "greedy", n_threads=5).info()
    assert a == b


def test_argument_errors(snn):
    g = synth.make_network(synth.NetConfig(name="t", M=64, P=4, n_vn=2, K=4, uniform_all=True, dmax=2))
    net = snn.Network.from_synth(g)
    part = oracle.partition_planted(64, 4)
    with pytest.raises(snn.SnnError) as e:
        snn.Routing(net, part, 4, 3)          # 4 % 3 != 0
    assert e.value.code == -1
    bad = part.copy()
    bad[5] = 9
    with pytest.raises(snn.SnnError):
        snn.Routing(net, bad, 4, 2)
    d = g.d.copy()
    d[3] = 0
    with pytest.raises(snn.SnnError) as e:
        snn.Routing(snn.Network(g.syn_ptr, g.tgt, g.w, d, g.v0), part, 4, 2)
    assert e.value.code == -5
    d[3] = 17
    with pytest.raises(snn.SnnError) as e:
        snn.Routing(snn.Network(g.syn_ptr, g.tgt, g.w, d, g.v0), part, 4, 2)
    assert e.value.code == -5
    empty = part.copy()
    empty[empty == 2] = 1
    with pytest.raises(snn.SnnError):
        snn.Routing(net, empty, 4, 2)         # partition 2 empty
    with pytest.raises(snn.SnnError):
        snn.snn_partition(net, 0, "planted")


def test_workspace_size_and_no_device(snn):
    g = synth.make_network(synth.TINY)
    net = snn.Network.from_synth(g)
    rt = snn.Routing(net, oracle.partition_planted(g.M, 4), 4, 2)
    p = snn.sim_params(synth.TINY.dyn)
    nb = ctypes.c_size_t(0)
    assert snn._lib.snn_sim_workspace_bytes(rt.h, ctypes.byref(p), ctypes.byref(nb)) == 0
    # synapse arrays (6 B/synapse) dominate the tiny workspace
    assert nb.value >= g.E * 6 and nb.value % 256 == 0
    p.steps_per_graph = 0
    assert snn._lib.snn_sim_workspace_bytes(rt.h, ctypes.byref(p), ctypes.byref(nb)) == -1
    import torch
    if not torch.cuda.is_available():
        p = snn.sim_params(synth.TINY.dyn)
        h = ctypes.c_void_p()
        rc = snn._lib.snn_sim_create(ctypes.byref(net.s), rt.h, ctypes.byref(p),
                                     ctypes.c_void_p(1 << 20), nb.value, None, ctypes.byref(h))
        assert rc == -7 and not h.value


def _small_batch():
    cfgs = synth.batch_configs(n=5, seed=77, m_lo=600, m_hi=4000, k_lo=12, k_hi=40, p_lo=4, p_hi=8)
    return synth.make_batch(cfgs)


def test_batch_concatenation_is_independent_networks():
    b = _small_batch()
    g = b.net
    assert (b.off % 4 == 0).all() and b.off[-1] == g.M
    src = np.repeat(np.arange(g.M), np.diff(g.syn_ptr))
    k_src = np.searchsorted(b.off, src, side="right") - 1
    k_tgt = np.searchsorted(b.off, g.tgt.astype(np.int64), side="right") - 1
    assert np.array_equal(k_src, k_tgt)
    for k, (c, n) in enumerate(zip(b.cfgs, b.nets)):
        a, e = b.off[k], b.off[k + 1]
        assert np.array_equal(b.part[a:e], oracle.partition_planted(c.M, c.P) + b.poff[k])
        e0 = g.syn_ptr[a]
        assert np.array_equal(g.tgt[e0:e0 + n.E], n.tgt + a) and np.array_equal(g.w[e0:e0 + n.E], n.w)


def test_batch_create_checks(snn):
    import torch
    b = _small_batch()
    net = snn.Network.from_synth(b.net)
    rt = snn.Routing(net, b.part, b.P, b.n_vn, "contiguous")
    plist = [snn.sim_params(c.dyn) for c in b.cfgs]
    n = len(plist)
    arr = (snn.snn_sim_params * n)(*plist)
    nb = ctypes.c_size_t(0)
    assert snn._lib.snn_batch_workspace_bytes(rt.h, n, arr, ctypes.byref(nb)) == 0
    plain = ctypes.c_size_t(0)
    assert snn._lib.snn_sim_workspace_bytes(rt.h, ctypes.byref(plist[0]), ctypes.byref(plain)) == 0
    assert nb.value > plain.value

    def create(off):
        off = np.ascontiguousarray(off, np.int64)
        h = ctypes.c_void_p()
        return snn._lib.snn_batch_create(ctypes.byref(net.s), rt.h, n, off.ctypes.data, arr,
                                         ctypes.c_void_p(1 << 20), nb.value, None, ctypes.byref(h))

    bad = b.off.copy()
    bad[2] += 2                       # not a multiple of 4
    assert create(bad) == -1
    bad = b.off.copy()
    bad[2] += 4                       # synapses now leave their network
    assert create(bad) == -1
    bad = b.off.copy()
    bad[-1] -= 4                      # does not end at M
    assert create(bad) == -1
    if not torch.cuda.is_available():
        assert create(b.off) == -7     # checks pass, no device here
    # partitions of a VN in two networks: group the concatenation's VNs across the seam
    part2 = b.part.copy()
    a = int(b.off[1])
    part2[a:a + 4] = part2[a - 1]     # a few ids of network 1 join network 0's last partition
    rt2 = snn.Routing(net, part2, b.P, b.n_vn, "contiguous")
    h = ctypes.c_void_p()
    off = np.ascontiguousarray(b.off, np.int64)
    assert snn._lib.snn_batch_create(ctypes.byref(net.s), rt2.h, n, off.ctypes.data, arr,
                                     ctypes.c_void_p(1 << 20), nb.value, None, ctypes.byref(h)) == -1


def test_exported_tables_follow_the_network(snn):
    """Every routing table exported by snn_routing_export, rebuilt from the
    network and the mapping with numpy (tests/_routing_defs.py)."""
    cfg = synth.NetConfig(name="t", M=1500, P=6, n_vn=3, K=18, uniform_all=False, n_part=10,
                          n_vn_t=5, n_remote=3, dmax=7, seed=12)
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    part = np.random.default_rng(3).permutation(oracle.partition_planted(g.M, 6)).astype(np.int32)
    rt = snn.Routing(net, part, 6, 3, "greedy", iters=2, seed=1)
    check_tables(rt, g, part, 6, 3)
    with pytest.raises(RuntimeError):
        rt.export("no_such_table")


def test_device_builders_check_arguments_before_the_device(snn):
    """snn_partition_device and snn_routing_build_device reject bad arguments
    and short or misaligned workspaces before any CUDA call (no GPU here)."""
    g = synth.make_network(synth.NetConfig(name="t", M=256, P=4, n_vn=2, K=6, uniform_all=True, dmax=3))
    net = snn.Network.from_synth(g)
    lib = snn._lib
    out = np.empty(g.M, np.int32)
    nb = ctypes.c_size_t(0)
    assert lib.snn_partition_device_workspace_bytes(ctypes.byref(net.s), 4, ctypes.byref(nb)) == 0
    assert nb.value >= 8 * g.E
    prm = snn.snn_partition_device_params()
    lib.snn_partition_device_params_default(ctypes.byref(prm))
    assert (prm.iters, prm.batch, prm.grow, prm.seed) == (4, 2048, 2, 7)
    fake = 1 << 20  # never dereferenced: every check below fails first

    def part(P, **kw):
        p = snn.snn_partition_device_params()
        lib.snn_partition_device_params_default(ctypes.byref(p))
        for k, v in kw.items():
            setattr(p, k, v)
        ws = kw.pop("ws", fake)
        return lib.snn_partition_device(ctypes.byref(net.s), P, ctypes.byref(p), ws, nb.value, None,
                                        out.ctypes.data, None)
    E_ARG, E_NOMEM = -1, -2
    assert part(4, batch=0) == E_ARG
    assert part(4, batch=4096) == E_ARG
    assert part(4, grow=-1) == E_ARG
    assert part(4, iters=0) == E_ARG
    assert part(0) == E_ARG and part(g.M + 1) == E_ARG
    assert lib.snn_partition_device(ctypes.byref(net.s), 4, ctypes.byref(prm), fake, nb.value - 256, None,
                                    out.ctypes.data, None) == E_NOMEM
    assert lib.snn_partition_device(ctypes.byref(net.s), 4, ctypes.byref(prm), fake + 8, nb.value, None,
                                    out.ctypes.data, None) == E_NOMEM
    # routing
    assert lib.snn_routing_build_device_workspace_bytes(ctypes.byref(net.s), 4, 2, ctypes.byref(nb)) == 0
    rp = snn.snn_routing_params(0, 1, 1, 0, 0)
    h = ctypes.c_void_p()
    po = oracle.partition_planted(g.M, 4)

    def route(P, n_vn, p_of=po, size=nb.value, ws=fake):
        return lib.snn_routing_build_device(ctypes.byref(net.s), p_of.ctypes.data, P, n_vn, ctypes.byref(rp), ws,
                                            size, None, ctypes.byref(h))
    assert route(4, 3) == E_ARG                      # P not a multiple of n_vn
    bad = po.copy()
    bad[7] = 4
    assert route(4, 2, bad) == E_ARG                 # a label out of range
    assert route(5, 1, po) == E_ARG                  # partition 4 has no neuron
    assert route(4, 2, size=nb.value - 256) == E_NOMEM
    assert route(4, 2, ws=fake + 16) == E_NOMEM
    big = synth.make_edges(4, [(0, j % 4, 1, 1) for j in range(16385)])
    bnet = snn.Network.from_synth(big)
    assert lib.snn_routing_build_device(ctypes.byref(bnet.s), np.zeros(4, np.int32).ctypes.data, 1, 1,
                                        ctypes.byref(rp), fake, 1 << 30, None, ctypes.byref(h)) == -5


def test_defer_parameter_is_checked(snn):
    """defer_delayed is 0 or 1 (minimum-delay batching switch); anything else
    is rejected before any device work."""
    g = synth.make_network(synth.NetConfig(name="t", M=64, P=4, n_vn=2, K=4, uniform_all=True, dmax=2))
    rt = snn.Routing(snn.Network.from_synth(g), oracle.partition_planted(64, 4), 4, 2)
    nb = ctypes.c_size_t(0)
    for v, rc in ((0, 0), (1, 0), (2, -1), (-1, -1)):
        p = snn.sim_params(defer_delayed=v)
        assert snn._lib.snn_sim_workspace_bytes(rt.h, ctypes.byref(p), ctypes.byref(nb)) == rc


def test_min_delay_schedule_is_exact():
    """The minimum-delay batching schedule on a delay ring of D = max delay + 1
    slots, modelled with the kernels' slot arithmetic (slot of a synapse of
    delay d from a spike of step s: (s mod D + d) mod D): delivering a step's
    delay-1 synapses in the step and its delay >= 2 synapses one step later
    (from the same base s) leaves every slot with the same sum when its step
    reads and clears it, for random spike trains and delays 1..8."""
    rng = np.random.default_rng(0)
    dmax = 8
    D = dmax + 1
    M, T = 50, 400
    for trial in range(5):
        syn = [(rng.integers(0, M, 20), rng.integers(1, dmax + 1, 20), rng.integers(-50, 50, 20))
               for _ in range(M)]
        spikes = [np.flatnonzero(rng.random(M) < 0.05) for _ in range(T)]
        ring_a = np.zeros((D, M), np.int64)
        ring_b = np.zeros((D, M), np.int64)
        deferred = []
        for t in range(T):
            # step t reads and clears its slot
            ra, rb = ring_a[t % D].copy(), ring_b[t % D].copy()
            assert np.array_equal(ra, rb), (trial, t)
            ring_a[t % D] = 0
            ring_b[t % D] = 0
            # schedule A: everything in step t
            for i in spikes[t]:
                tg, dl, w = syn[i]
                np.add.at(ring_a, ((t % D + dl) % D, tg), w)
            # schedule B: the previous step's delay >= 2 lists, then this step's delay-1 heads
            for (s, tg, dl, w) in deferred:
                np.add.at(ring_b, ((s % D + dl) % D, tg), w)
            deferred = []
            for i in spikes[t]:
                tg, dl, w = syn[i]
                one = dl == 1
                np.add.at(ring_b, ((t % D + dl[one]) % D, tg[one]), w[one])
                deferred.append((t, tg[~one], dl[~one], w[~one]))
