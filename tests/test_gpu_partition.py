"""GPU parity of the device partitioner (Algorithm 1 with batched growth)
against the CPU oracle of the same rounds: labels and objective equal, for
rounds of one (the sequential greedy, also the library's host greedy),
fixed rounds and rounds that grow with the part, over hand-built,
planted, uniform and ragged networks and the degenerate cases."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

# eight neurons of out-degree 2 whose sequential and batched growth differ
# (worked by hand in the oracle pins)
_HAND_EDGES = [(0, 1), (0, 2), (1, 3), (1, 3), (2, 5), (2, 6), (3, 4), (3, 4),
               (4, 5), (4, 6), (5, 6), (5, 7), (6, 7), (6, 5), (7, 2), (7, 5)]


@pytest.fixture(scope="module")
def snn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_07125_gb300 as m
    return m


def _both(snn, g, P, batch, grow, iters, seed):
    net = snn.Network.from_synth(g)
    part, st = snn.snn_partition_device(net, P, batch=batch, grow=grow, iters=iters, seed=seed, device="cuda:0")
    ref, obj = oracle.partition_greedy_batched(g, P, batch, grow, iters=iters, seed=seed)
    assert np.array_equal(part, ref), (batch, grow, np.flatnonzero(part != ref)[:10])
    assert st["objective"] == obj
    W = np.diff(g.syn_ptr)
    ws = np.bincount(part, weights=W, minlength=P)
    assert st["min_weight"] == int(ws.min()) and st["max_weight"] == int(ws.max())
    return part


@pytest.mark.parametrize("batch,grow,part0", [(1, 0, {0, 1, 3, 4}), (3, 0, {0, 1, 2, 3}),
                                              (2, 0, {0, 1, 2, 3}), (3, 2, {0, 1, 3, 4})])
def test_hand_worked(snn, batch, grow, part0):
    g = synth.make_edges(8, [(a, b, 1, 1) for a, b in _HAND_EDGES])
    part = _both(snn, g, 2, batch, grow, 1, 1)
    assert set(np.flatnonzero(part == 0).tolist()) == part0


@pytest.mark.parametrize("seed", [3, 4])
def test_rounds_of_one_equal_the_host_greedy(snn, seed):
    cfg = synth.NetConfig(name="t", M=1500, P=6, n_vn=2, K=14, uniform_all=False, n_part=10, n_vn_t=2,
                          n_remote=2, seed=seed)
    g = synth.make_network(cfg)
    part = _both(snn, g, 5, 1, 0, 3, seed)
    host, _ = snn.snn_partition(snn.Network.from_synth(g), 5, "greedy", iters=3, seed=seed)
    assert np.array_equal(part, host)


@pytest.mark.parametrize("batch,grow", [(7, 0), (64, 0), (64, 4), (2048, 0), (2048, 8)])
@pytest.mark.parametrize("M,P,uniform", [(3000, 8, False), (2333, 5, True)])
def test_batched_rounds_equal_oracle(snn, batch, grow, M, P, uniform):
    cfg = synth.NetConfig(name="t", M=M, P=8, n_vn=2, K=20, uniform_all=uniform, n_part=14, n_vn_t=4,
                          n_remote=2, seed=M)
    g = synth.make_network(cfg)
    _both(snn, g, P, batch, grow, 3, 11)


def test_relabelled_planted_network(snn):
    """ids shuffled so that contiguous ranges say nothing: growth from seeds
    recovers the planted partitions as the oracle does."""
    cfg = synth.NetConfig(name="t", M=8192, P=8, n_vn=2, K=40, uniform_all=False, n_part=34, n_vn_t=4,
                          n_remote=2, seed=9)
    g = synth.make_network(cfg)
    perm = np.random.default_rng(5).permutation(g.M).astype(np.int64)
    src = np.repeat(np.arange(g.M), np.diff(g.syn_ptr))
    edges = list(zip(perm[src].tolist(), perm[g.tgt].tolist(), [1] * len(src), [1] * len(src)))
    h = synth.make_edges(g.M, edges)
    part = _both(snn, h, 8, 256, 4, 2, 3)
    planted = oracle.partition_planted(g.M, 8)[np.argsort(perm)]
    assert oracle.cut(h, part) <= oracle.cut(h, planted)


def test_hub_spans_many_scatter_chunks(snn):
    """A neuron with out-degree 2999 and one with in-degree ~3000: their
    gains are scattered in many 256-synapse chunks."""
    M = 3000
    edges = [(0, j, 1, 1) for j in range(1, M)] + [(j, 1, 1, 1) for j in range(2, M)]
    edges += [(j, (j * 7 + 3) % M, 1, 1) for j in range(2, M)]
    g = synth.make_edges(M, edges)
    for batch, grow in [(1, 0), (100, 0), (100, 5)]:
        _both(snn, g, 4, batch, grow, 2, 8)


@pytest.mark.parametrize("M,P", [(1, 1), (3, 3), (5, 1), (7, 7), (40, 39)])
def test_degenerate_sizes(snn, M, P):
    """P = 1 (no growth), P = M (one neuron per part), tiny M."""
    edges = [(i, (i + 1) % M, 1, 1) for i in range(M)] if M > 1 else []
    g = synth.make_edges(M, edges)
    for batch in (1, 4):
        part = _both(snn, g, P, batch, 0, 2, 1)
        if P == 1:
            assert np.all(part == 0)


def test_no_synapses(snn):
    """W = 0 everywhere: every part but the last is its seed alone."""
    g = synth.make_edges(50, [])
    for batch in (1, 16):
        part = _both(snn, g, 5, batch, 0, 3, 2)
        assert np.bincount(part, minlength=5).tolist() == [1, 1, 1, 1, 46]


def test_bad_arguments(snn):
    g = synth.make_edges(10, [(0, 1, 1, 1)])
    net = snn.Network.from_synth(g)
    for kw in ({"batch": 0}, {"batch": 4096}, {"grow": -1}, {"iters": 0}):
        with pytest.raises(RuntimeError):
            snn.snn_partition_device(net, 2, device="cuda:0", **kw)
    with pytest.raises(RuntimeError):
        snn.snn_partition_device(net, 11, device="cuda:0")
    bad = synth.make_edges(10, [(0, 1, 1, 1), (2, 12, 1, 1)])
    with pytest.raises(RuntimeError):
        snn.snn_partition_device(snn.Network.from_synth(bad), 2, device="cuda:0")
