"""Pins of the CPU oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: every check is a published
test vector, a library routine, a closed form, an invariant, or brute force
on a tiny input.  All run on the CPU (no GPU marker).
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    return rows


# ------------------------------------------------------------------ RNG
def test_philox_known_answers():
    for r in _kat("philox4x32_10_kat.txt"):
        out = oracle.philox4x32_10(r[0:4], r[4:6])
        assert [int(x) for x in out] == r[6:10]


def test_splitmix_known_answers():
    for st, want in _kat("splitmix64_kat.txt"):
        assert oracle.mix64(st) == want


def test_poisson_table_matches_library_cdf():
    from scipy.stats import poisson
    for lam in (0.0, 0.05, 0.8, 1.7, 5.0):
        th = oracle.poisson_table(lam)
        assert th[-1] == 1 << 32
        assert np.all(np.diff(th.astype(np.float64)) >= 0)
        for k, v in enumerate(th[:-1]):
            ref = math.floor(poisson.cdf(k, lam) * 2.0**32)
            assert abs(int(v) - ref) <= 1, (lam, k, int(v), ref)


def test_drive_draw_distribution():
    """k_j(t) ~ Poisson(lambda): chi-square against the pmf, plus mean/var."""
    from scipy.stats import chi2, poisson
    lam = 0.8
    ks = np.concatenate([oracle.drive_draws(2000, lam, 0, 50000, t) for t in range(4)])
    n = len(ks)
    assert abs(ks.mean() - lam) < 4 * math.sqrt(lam / n)
    assert abs(ks.var() - lam) < 0.02
    kmax = 5
    obs = np.array([(ks == k).sum() for k in range(kmax)] + [(ks >= kmax).sum()])
    exp = np.array([poisson.pmf(k, lam) for k in range(kmax)] + [poisson.sf(kmax - 1, lam)]) * n
    stat = ((obs - exp) ** 2 / exp).sum()
    assert stat < chi2.ppf(0.999, len(obs) - 1)
    # one Philox4x32-10 block (pinned by the known answers) serves four
    # consecutive neurons: neuron j takes word j mod 4 of block (j div 4, t)
    th = oracle.poisson_table(lam)
    words = oracle.philox4x32_10([25, 7, 0, 0], [2000, 0])
    assert list(oracle.drive_draws(2000, lam, 100, 4, 7)) == [int((th <= int(w)).sum()) for w in words]
    # counter-based: a draw depends only on (seed, neuron, step)
    a = oracle.drive_draws(2000, lam, 100, 10, 7)
    b = oracle.drive_draws(2000, lam, 95, 20, 7)[5:15]
    assert np.array_equal(a, b)
    assert not np.array_equal(oracle.drive_draws(2001, lam, 0, 64, 0),
                              oracle.drive_draws(2000, lam, 0, 64, 0))


# ------------------------------------------------------------------ LIF
def _isolated(M, v0, dyn):
    net = synth.make_edges(M, [], v0=v0)
    po = np.zeros(M, np.int32)
    return oracle.Oracle(net, 1, po, 1, np.zeros(1, np.int32), dyn)


@pytest.mark.parametrize("c_units", [0, 40, -25, 250])
def test_subthreshold_closed_form(c_units):
    """Constant input c per step, no spikes: V_n = E_L + a^n (V_0 - E_L) + c (1-a^n)/(1-a)."""
    dyn = synth.Dynamics(drive_lambda=0.0, i_bias=c_units, v_th=1e9)
    v0 = np.array([-65.0, -60.0, -55.5, -70.25], np.float32)
    o = _isolated(len(v0), v0, dyn)
    a = math.exp(-dyn.dt_ms / dyn.tau_ms)
    c = c_units / 1024.0
    worst = 0.0
    for n in range(1, 601):
        o.run(1, raster=False, hashes=False)
        for j, vj in enumerate(v0):
            ref = dyn.e_l + a**n * (float(vj) - dyn.e_l) + c * (1 - a**n) / (1 - a)
            worst = max(worst, abs(float(o.V[j]) - ref) / abs(ref))
    assert worst <= 1e-5, worst
    # the FP64 shadow follows the closed form to double rounding
    ref = dyn.e_l + a**600 * (v0.astype(np.float64) - dyn.e_l) + c * (1 - a**600) / (1 - a)
    assert np.max(np.abs(o.v64 - ref) / np.abs(ref)) < 1e-12


def test_threshold_reset_refractory_trace():
    """Regular firing under a constant suprathreshold input, times from the closed form."""
    c_units = 200
    dyn = synth.Dynamics(drive_lambda=0.0, i_bias=c_units)
    o = _isolated(2, np.array([-65.0, -65.0], np.float32), dyn)
    a = math.exp(-dyn.dt_ms / dyn.tau_ms)
    c = c_units / 1024.0
    # V after the update of the n-th integrating step from rest (n = 1, 2, ...)
    n_star = next(n for n in range(1, 10000)
                  if dyn.e_l + c * (1 - a**n) / (1 - a) >= dyn.v_th)
    margin = min(abs(dyn.e_l + c * (1 - a**n) / (1 - a) - dyn.v_th) for n in (n_star - 1, n_star))
    assert margin > 1e-3  # far from a rounding tie
    period = n_star + dyn.t_ref
    T = 5 * period + 3
    r = o.run(T)
    off = r["raster_off"]
    spk_steps = [t for t in range(T) if off[t + 1] > off[t]]
    want = [n_star - 1 + m * period for m in range(5)]
    assert spk_steps[:5] == want
    # both neurons identical, and V is clamped at reset while refractory
    assert np.array_equal(np.diff(off)[: T], 2 * np.isin(np.arange(T), want))


def test_drive_mean_and_variance_closed_form():
    """Stationary V of the Poisson-driven membrane (no threshold): mean and variance.

    V = E_L + sum_k a^k w (k_{t-k}) 2^-10  =>  E[V] = E_L + lam w 2^-10 / (1-a),
    Var[V] = lam (w 2^-10)^2 / (1 - a^2).
    """
    lam, w = 0.8, 96
    dyn = synth.Dynamics(drive_lambda=lam, w_ext=w, v_th=1e9)
    M = 4096
    o = _isolated(M, np.full(M, -65.0, np.float32), dyn)
    a = math.exp(-dyn.dt_ms / dyn.tau_ms)
    o.run(2000, raster=False, hashes=False)  # burn in (10 time constants)
    vs = []
    for _ in range(20):
        o.run(50, raster=False, hashes=False)
        vs.append(o.V.astype(np.float64).copy())
    vs = np.array(vs)
    mean = dyn.e_l + lam * w / 1024.0 / (1 - a)
    var = lam * (w / 1024.0) ** 2 / (1 - a * a)
    assert abs(vs.mean() - mean) < 0.02
    assert abs(vs.var() / var - 1) < 0.05


# ------------------------------------------------------------------ delivery
def _dense_currents(net, raster_sets, T, dmax):
    """Brute force: I_t = sum_d W_d^T s_{t-d} with dense per-delay weight matrices."""
    M = net.M
    Wd = np.zeros((dmax + 1, M, M), np.int64)
    src = np.repeat(np.arange(M), np.diff(net.syn_ptr))
    np.add.at(Wd, (net.d.astype(np.int64), src, net.tgt.astype(np.int64)), net.w.astype(np.int64))
    S = np.zeros((T, M), np.int64)
    for t, ids in enumerate(raster_sets):
        S[t, ids] = 1
    I = np.zeros((T, M), np.int64)
    for t in range(T):
        for d in range(1, dmax + 1):
            if t - d >= 0:
                I[t] += S[t - d] @ Wd[d]
    return I


def test_delivery_against_dense_brute_force():
    cfg = synth.NetConfig(name="t", M=96, P=4, n_vn=2, K=12, uniform_all=False, n_part=6, n_vn_t=4,
                          n_remote=2, dmax=3, seed=11,
                          dyn=synth.Dynamics(drive_lambda=0.9, w_ext=180, drive_seed=5))
    net = synth.make_network(cfg)
    P = 4
    o = oracle.Oracle(net, P, oracle.partition_planted(net.M, P), 2, oracle.group_contiguous(P, 2),
                      cfg.dyn)
    T = 120
    r = o.run(T, rec_steps=range(T))
    off = r["raster_off"]
    sets = [r["raster_ids"][off[t]:off[t + 1]] for t in range(T)]
    assert sum(len(s) for s in sets) > 20
    I = _dense_currents(net, sets, T, cfg.dmax)
    for t in range(T):
        assert np.array_equal(r["currents"][t], I[t]), t
    # each step's events = sum of the out-degrees of its spikes
    assert o.count_dict()["events"] == sum(len(s) for s in sets) * cfg.K


# ------------------------------------------------------------------ message counts
def _brute_counts(net, part_of, vn_of_part, spikes):
    """Direct and two-level message counts from their set definitions."""
    P = int(part_of.max()) + 1
    groups = {}
    for p in range(P):
        groups.setdefault(int(vn_of_part[p]), []).append(p)
    relay = {(g, h): sorted(groups[g])[(h - g) % len(groups[g])] for g in groups for h in groups}
    c = dict.fromkeys(oracle.COUNT_NAMES[3:], 0)
    for i in spikes:
        p = int(part_of[i])
        h = int(vn_of_part[p])
        Q = {int(part_of[j]) for j in net.tgt[net.syn_ptr[i]:net.syn_ptr[i + 1]]}
        G = {int(vn_of_part[q]) for q in Q}
        c["direct"] += len(Q - {p})
        c["direct_xvn"] += sum(1 for q in Q if vn_of_part[q] != h)
        c["l1_local"] += int(h in G)
        c["l1_xvn"] += len(G - {h})
        c["l2_local"] += int(p in Q)
        c["l2_peer"] += sum(1 for q in Q if vn_of_part[q] == h and q != p)
        for g in G - {h}:
            r = relay[(g, h)]
            c["l2_relay_local"] += int(r in Q)
            c["l2_relay_remote"] += sum(1 for q in Q if vn_of_part[q] == g and q != r)
    return c


def test_counts_star_graph_by_hand():
    """Hub 0 of partition 0 reaches every partition; 8 neurons, 4 partitions, 2 VNs.

    One spike of the hub: direct route 3 messages (to partitions 1, 2, 3), 2 of
    them across VNs; two-level route: 1 L1 message to VN 1, whose relay for
    VN 0 is partition 2, plus 1 direct intra-VN message to partition 1 and 1
    relay forward to partition 3.
    """
    edges = [(0, 1, 5, 1), (0, 2, 5, 1), (0, 4, 5, 1), (0, 6, 5, 1), (0, 7, 5, 1)]
    v0 = np.full(8, -65.0, np.float32)
    v0[0] = -40.0
    net = synth.make_edges(8, edges, v0=v0)
    dyn = synth.Dynamics(drive_lambda=0.0)
    part = np.array([0, 0, 1, 1, 2, 2, 3, 3], np.int32)
    o = oracle.Oracle(net, 4, part, 2, np.array([0, 0, 1, 1], np.int32), dyn)
    r = o.run(3, pairs=True)
    assert list(r["raster_ids"]) == [0]
    c = o.count_dict()
    want = dict(direct=3, direct_xvn=2, l1_local=1, l1_xvn=1, l2_local=1, l2_peer=1,
                l2_relay_local=1, l2_relay_remote=1, events=5, spikes=1)
    for k, v in want.items():
        assert c[k] == v, (k, c[k], v)
    # relay choice depends on the source group: put the hub in VN 1 instead
    o2 = oracle.Oracle(net, 4, part, 2, np.array([1, 1, 0, 0], np.int32), dyn)
    o2.run(3)
    c2 = o2.count_dict()
    # source VN 1 -> destination VN 0 = {2, 3}; relay index 1 % 2 -> partition 3
    assert c2["l2_relay_local"] == 1 and c2["l2_relay_remote"] == 1


@pytest.mark.parametrize("step", [1, 3])
def test_counts_ring_graph_by_hand(step):
    """Directed ring over 8 partitions in 4 VNs of 2: each spike of partition p
    reaches exactly partition p + step (mod 8)."""
    M, P = 16, 8
    edges = [(i, (i + 2 * step) % M, 3, 1) for i in range(M)]
    v0 = np.full(M, -40.0, np.float32)
    net = synth.make_edges(M, edges, v0=v0)
    part = (np.arange(M) // 2).astype(np.int32)
    vn = (np.arange(P) // 2).astype(np.int32)
    o = oracle.Oracle(net, P, part, 4, vn, synth.Dynamics(drive_lambda=0.0))
    o.run(1)
    c = o.count_dict()
    # all 16 neurons spike once, two per partition
    assert c["spikes"] == 16 and c["direct"] == 16
    same_vn = [p for p in range(P) if (p + step) % P // 2 == p // 2]
    assert c["l2_peer"] == 2 * len(same_vn) and c["l2_local"] == 0
    assert c["l1_local"] == 2 * len(same_vn) and c["l1_xvn"] == 16 - 2 * len(same_vn)
    assert c["direct_xvn"] == c["l1_xvn"]
    # the relay of VN g for source VN h is member (h - g) mod 2 of g: partition 2g + (h - g) % 2
    local = 0
    for p in range(P):
        q, h = (p + step) % P, p // 2
        g = q // 2
        if g != h and q == 2 * g + (h - g) % 2:
            local += 1
    assert c["l2_relay_local"] == 2 * local
    assert c["l2_relay_remote"] == c["l1_xvn"] - 2 * local
    # step 1: odd p -> 2g with relay 2g + 1 (all forwarded); step 3: p -> the
    # relay itself (none forwarded)
    assert local == (0 if step == 1 else 8)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_counts_random_tiny_brute_force(seed):
    cfg = synth.NetConfig(name="t", M=64, P=4, n_vn=2, K=10, uniform_all=(seed == 3), n_part=5,
                          n_vn_t=3, n_remote=2, dmax=2, seed=seed,
                          dyn=synth.Dynamics(drive_lambda=1.2, w_ext=160, drive_seed=seed))
    net = synth.make_network(cfg)
    rng = np.random.default_rng(seed)
    part = rng.permutation(np.arange(64) % 4).astype(np.int32)
    vn = np.array([1, 0, 0, 1], np.int32)
    o = oracle.Oracle(net, 4, part, 2, vn, cfg.dyn)
    r = o.run(60, pairs=True)
    spikes = r["raster_ids"]
    assert len(spikes) > 10
    c = o.count_dict()
    b = _brute_counts(net, part, vn, spikes)
    for k, v in b.items():
        assert c[k] == v, (k, c[k], v)
    # conservation: the last step's direct-route pairs are exactly {(i, q): q holds a target of i}
    last = r["raster_ids"][r["raster_off"][-2]:r["raster_off"][-1]]
    want = sorted((int(i) << 32) | int(q) for i in last
                  for q in {int(part[j]) for j in net.tgt[net.syn_ptr[i]:net.syn_ptr[i + 1]]})
    assert [int(x) for x in r["pairs"]] == want


def test_counts_closed_form_at_scale():
    """Distinct destinations per spike follow K (1 - (1 - 1/K)^n) for n uniform picks."""
    cfg = synth.SCALE.scaled(M=1 << 16, seed=77)
    net = synth.make_network(cfg)
    P, nv = cfg.P, cfg.n_vn
    o = oracle.Oracle(net, P, oracle.partition_planted(net.M, P), nv, oracle.group_contiguous(P, nv),
                      cfg.dyn)
    o.run(60, raster=False, hashes=False)
    c = o.count_dict()
    S = c["spikes"]
    assert S > 2000
    s = cfg.vn_size
    n_rem_parts = P - s
    rem = n_rem_parts * (1 - (1 - 1 / n_rem_parts) ** cfg.n_remote)    # remote partitions hit
    vns = (nv - 1) * (1 - (1 - 1 / (nv - 1)) ** cfg.n_remote)        # remote VNs hit
    assert abs(c["direct"] / S - (s - 1 + rem)) < 0.05 * (s - 1 + rem)
    assert abs(c["direct_xvn"] / S - rem) < 0.05 * rem
    assert abs(c["l1_xvn"] / S - vns) < 0.05 * vns
    assert c["l1_local"] == S and c["l2_local"] == S and c["l2_peer"] == (s - 1) * S
    assert c["events"] == S * cfg.K


def test_fp64_membrane_error_within_tolerance():
    net = synth.make_network(synth.TINY)
    P = synth.TINY.P
    o = oracle.Oracle(net, P, oracle.partition_planted(net.M, P), 2, oracle.group_contiguous(P, 2),
                      synth.TINY.dyn)
    o.run(1000, raster=False, hashes=False)
    st = o.fp64_stats()
    assert st["n_compared"] > 3_000_000
    assert st["max_rel_err"] <= 1e-5
    assert st["n_disagree"] <= 10


# ------------------------------------------------------------------ Algorithm 1
def _exhaustive_best(net, P, sizes):
    """Minimum objective over all assignments with the given part sizes."""
    M = net.M
    best = None
    for lab in itertools.product(range(P), repeat=M):
        lab = np.array(lab, np.int32)
        if sorted(np.bincount(lab, minlength=P).tolist()) != sorted(sizes):
            continue
        c = oracle.cut(net, lab)
        best = c if best is None else min(best, c)
    return best


def test_greedy_partition_balance_and_optimum_on_planted_cliques():
    """Two dense 6-cliques joined by one synapse: the greedy mapping is optimal."""
    edges = []
    for blk in (0, 6):
        for i in range(6):
            for j in range(6):
                if i != j:
                    edges.append((blk + i, blk + j, 1, 1))
    edges.append((2, 9, 1, 1))
    net = synth.make_edges(12, edges)
    part, obj = oracle.partition_greedy(net, 2, iters=3, seed=1)
    assert np.bincount(part).tolist() == [6, 6]
    assert obj == oracle.cut(net, part)
    assert obj == _exhaustive_best(net, 2, [6, 6])


@pytest.mark.parametrize("seed", [4, 5])
def test_greedy_partition_vs_exhaustive_random(seed):
    cfg = synth.NetConfig(name="t", M=10, P=2, n_vn=1, K=3, uniform_all=True, seed=seed)
    net = synth.make_network(cfg)
    part, obj = oracle.partition_greedy(net, 2, iters=4, seed=seed)
    sizes = np.bincount(part, minlength=2).tolist()
    # balance: every part but the last reaches sum(W)/P; uniform W => equal sizes
    assert sizes == [5, 5]
    opt = _exhaustive_best(net, 2, sizes)
    assert opt <= obj
    assert obj <= 2 * opt + 1  # reported ratio stays bounded on these inputs


def test_greedy_partition_recovers_planted_structure():
    cfg = synth.NetConfig(name="t", M=2048, P=8, n_vn=2, K=40, uniform_all=False, n_part=34,
                          n_vn_t=4, n_remote=2, seed=9)
    net = synth.make_network(cfg)
    part, obj = oracle.partition_greedy(net, 8, iters=2, seed=3)
    planted = oracle.partition_planted(net.M, 8)
    assert np.all(np.bincount(part, minlength=8) == 256)
    assert obj <= oracle.cut(net, planted)
    # each greedy part is (mostly) one planted partition
    for k in range(8):
        assert np.bincount(planted[part == k], minlength=8).max() >= 0.9 * 256
    rnd = np.random.default_rng(0).permutation(planted)
    assert oracle.cut(net, rnd) > 3 * obj


# ---------------------------------------------------- Algorithm 1, batched growth
# Eight neurons of out-degree 2 (W = 2 each, sum 16, a part is full at weight
# 8 = four neurons).  From seed 0, neurons 1 and 2 gain 4 each; 1 leads to 3
# by two synapses, 3 to 4 by two.  Sequential growth (ranking after every
# join): 0, 1, then 3 (gain 8 > 4), then 4 (8 > 4).  A round of 3 ranked on
# the seed's gains alone: 1, 2 (gain 4 each), then 3 (gain 0, lowest id).
_HAND_EDGES = [(0, 1), (0, 2), (1, 3), (1, 3), (2, 5), (2, 6), (3, 4), (3, 4),
               (4, 5), (4, 6), (5, 6), (5, 7), (6, 7), (6, 5), (7, 2), (7, 5)]


@pytest.mark.parametrize("batch,grow,part0", [
    (1, 0, {0, 1, 3, 4}),   # the sequential greedy
    (3, 0, {0, 1, 2, 3}),   # one round ranked on the seed's gains
    (2, 0, {0, 1, 2, 3}),   # rounds {1, 2}, then {3, 5}: 3 fills the part
    (3, 2, {0, 1, 3, 4}),   # rounds of max(1, n_k // 2) = 1 while the part is small
])
def test_batched_greedy_hand_worked(batch, grow, part0):
    net = synth.make_edges(8, [(a, b, 1, 1) for a, b in _HAND_EDGES])
    part, obj = oracle.partition_greedy_batched(net, 2, batch, grow, iters=1, seed=1)
    assert set(np.flatnonzero(part == 0).tolist()) == part0
    assert obj == oracle.cut(net, part)


@pytest.mark.parametrize("seed", [2, 11, 12])
def test_batched_greedy_with_rounds_of_one_is_the_greedy(seed):
    """Rounds of one neuron are the sequential greedy, step for step (every
    seed of the t > 1 iterations included)."""
    cfg = synth.NetConfig(name="t", M=600, P=6, n_vn=2, K=12, uniform_all=(seed == 2), n_part=8,
                          n_vn_t=2, n_remote=2, seed=seed)
    net = synth.make_network(cfg)
    ref, obj = oracle.partition_greedy(net, 5, iters=3, seed=seed)
    for grow in (0, 3):
        part, o = oracle.partition_greedy_batched(net, 5, 1, grow, iters=3, seed=seed)
        assert np.array_equal(part, ref) and o == obj


@pytest.mark.parametrize("batch,grow", [(2, 0), (5, 0), (100, 0), (100, 2)])
def test_batched_greedy_balance_and_planted_cliques(batch, grow):
    """Two 6-cliques joined by one synapse: every round size finds them."""
    edges = []
    for blk in (0, 6):
        for i in range(6):
            for j in range(6):
                if i != j:
                    edges.append((blk + i, blk + j, 1, 1))
    edges.append((2, 9, 1, 1))
    net = synth.make_edges(12, edges)
    part, obj = oracle.partition_greedy_batched(net, 2, batch, grow, iters=3, seed=1)
    assert np.bincount(part).tolist() == [6, 6]
    assert obj == _exhaustive_best(net, 2, [6, 6])


@pytest.mark.parametrize("batch,grow", [(7, 0), (64, 4), (1000, 0)])
def test_batched_greedy_balance_invariant(batch, grow):
    """Every part but the last stops at the first join that brings its weight
    to sum(W)/P: sum(W)/P <= W(part) < sum(W)/P + max W."""
    cfg = synth.NetConfig(name="t", M=1500, P=6, n_vn=2, K=10, uniform_all=False, n_part=6,
                          n_vn_t=2, n_remote=2, seed=5)
    g = synth.make_network(cfg)
    # unequal weights: drop a seeded share of each neuron's synapses
    rng = np.random.default_rng(1)
    keep = rng.random(len(g.tgt)) < 0.6
    src = np.repeat(np.arange(g.M), np.diff(g.syn_ptr))
    net = synth.make_edges(g.M, list(zip(src[keep].tolist(), g.tgt[keep].tolist(),
                                         [1] * int(keep.sum()), [1] * int(keep.sum()))))
    W = np.diff(net.syn_ptr)
    part, obj = oracle.partition_greedy_batched(net, 6, batch, grow, iters=2, seed=4)
    wsum = np.bincount(part, weights=W, minlength=6)
    tot = W.sum()
    for k in range(5):
        assert wsum[k] * 6 >= tot and (wsum[k] - W.max()) * 6 < tot
    assert obj == oracle.cut(net, part)


# ------------------------------------------------------------------ Algorithm 2
def _group_cost(PG, WG, grp):
    P = len(WG)
    return sum(int(PG[p, q]) * int(WG[p]) * int(WG[q]) for p in range(P) for q in range(P)
               if grp[p] != grp[q])


def test_greedy_grouping_recovers_planted_and_is_optimal():
    cfg = synth.NetConfig(name="t", M=1024, P=8, n_vn=2, K=30, uniform_all=False, n_part=10,
                          n_vn_t=15, n_remote=5, seed=21)
    net = synth.make_network(cfg)
    part = oracle.partition_planted(net.M, 8)
    # shuffle partition labels so that planted groups are not contiguous labels
    perm = np.array([3, 6, 0, 5, 1, 7, 2, 4], np.int32)
    part = perm[part]
    vn, cost = oracle.group_greedy(net, part, 8, 2, iters=3, seed=2)
    planted_group = {int(perm[p]): p // 4 for p in range(8)}
    for g in range(2):
        members = [q for q in range(8) if vn[q] == g]
        assert len(members) == 4
        assert len({planted_group[q] for q in members}) == 1
    # brute-force optimum over all balanced 2-groupings
    src = np.repeat(np.arange(net.M), np.diff(net.syn_ptr))
    PG = np.zeros((8, 8), np.int64)
    np.add.at(PG, (part[src], part[net.tgt]), 1)
    np.fill_diagonal(PG, 0)
    WG = np.bincount(part[src], minlength=8).astype(np.int64)
    best = min(_group_cost(PG, WG, [1 if q in c else 0 for q in range(8)])
               for c in itertools.combinations(range(8), 4))
    assert cost == _group_cost(PG, WG, vn) == best
