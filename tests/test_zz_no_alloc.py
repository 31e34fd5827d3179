"""snn_deliver_spikes_static: the fan-out entry point that allocates nothing.

Some callers cannot allocate device memory once they run (a host program
that hands out all device memory from its own fixed budget, or a real-time
stimulation loop that may not stall in an allocator call).  For them the
library offers a variant of snn_deliver_spikes whose scratch is a fixed
array built into the library.  This test calls it through the C ABI and
checks, on two calls in a row, that it produces exactly the output and
counts of snn_deliver_spikes (integer sums: the tolerance is zero).  It
lives in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_07125_gb300 as snn
    cfg = synth.SCALE.scaled(M=1 << 14, seed=61)
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    part, _ = snn.snn_partition(net, cfg.P, "planted")
    rt = snn.Routing(net, part, cfg.P, cfg.n_vn)
    sim = snn.Sim(net, rt, snn.sim_params(cfg.dyn), device="cuda:0")
    return snn, g, rt, sim


def _call(snn, fn, sim, ids, out):
    counts = np.zeros(3, np.uint64)
    rc = fn(ctypes.c_void_p(sim.h), ctypes.c_void_p(ids.data_ptr()), ids.numel(),
            ctypes.c_void_p(out.data_ptr()), counts.ctypes.data)
    return rc, counts


def test_static_matches_workspace_variant_two_calls(env):
    import torch
    snn, g, rt, sim = env
    dmax = rt.info()["max_delay"]
    ref = torch.zeros((dmax, g.M), dtype=torch.int32, device="cuda:0")
    got = torch.zeros_like(ref)
    rng = np.random.default_rng(7)
    for n in (900, 2500):
        ids = torch.from_numpy(rng.integers(0, g.M, n).astype(np.int32)).to("cuda:0")
        rc_a, c_a = _call(snn, snn._lib.snn_deliver_spikes, sim, ids, ref)
        rc_b, c_b = _call(snn, snn._lib.snn_deliver_spikes_static, sim, ids, got)
        assert rc_a == 0 and rc_b == 0
        assert np.array_equal(c_a, c_b)
        assert int(c_b[2]) == n * g.cfg.K
        assert torch.equal(got, ref)
    # the sim is unaffected and still steps
    sim.step(5)
    assert sim.sync_status() == 0


def test_static_rejects_oversized_calls(env):
    import torch
    snn, g, rt, sim = env
    cap = int(snn._lib.snn_static_scratch_bytes())
    assert cap == 8 << 20
    n = cap // 8  # far beyond the per-spike worst case the array can hold
    ids = torch.zeros(n, dtype=torch.int32, device="cuda:0")
    out = torch.zeros((rt.info()["max_delay"], g.M), dtype=torch.int32, device="cuda:0")
    rc, _ = _call(snn, snn._lib.snn_deliver_spikes_static, sim, ids, out)
    assert rc == -5
    assert int(out.abs().sum()) == 0
