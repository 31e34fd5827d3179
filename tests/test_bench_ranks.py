"""Host logic of bench.py on CPU: two gloo ranks (replicas with summed work
and the maximum time over ranks, no data-path collective), the byte
formulas, the reference arm, the study helpers and the traffic lookup."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), SNN_BENCH_BACKEND="gloo")
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist, r, w = bench.dist_init()
    assert (r, w) == (rank, world)
    bench.barrier(dist)
    ev, ms, extra = bench.reduce_over_ranks(dist, events=1000.0 * (rank + 1), ms=10.0 + rank,
                                            extra=rank + 0.5)
    q.put((rank, ev, ms, extra))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ev, ms, extra in got:
        assert ev == 3000.0 and ms == 11.0 and extra == 2.0


def test_single_rank_passthrough():
    import bench
    assert bench.reduce_over_ranks(None, 5.0, 2.0, 1.0) == (5.0, 2.0, 1.0)


def test_phase_bytes_formula():
    import bench
    d = dict(spikes=10, l1_local=10, l1_xvn=20, l2_local=10, l2_peer=30, l2_relay_local=5,
             l2_relay_remote=15, events=10000)
    b = bench.phase_bytes(M=100, d_steps=2, d=d, gid=False)
    assert b[0] == 18 * 100 * 2 + 40
    assert b[1] == 12 * 10 + 6 * 30
    assert b[2] == 12 * 30 + 24 * 60
    assert b[3] == 8 * 60 + 6 * 10000


def test_reference_arm_ranks_other_than_zero_exit_quietly(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.main(["--impl", "reference"])
    assert capsys.readouterr().out == ""


@pytest.mark.parametrize("argv", [["--warmup", "2"]])
def test_bench_rejects_short_warmup(argv):
    import bench
    with pytest.raises(SystemExit):
        bench.main(argv)


def test_study_helpers_against_the_oracle():
    """bench.py's partition-study helpers: the numpy objective equals the
    oracle's cut, the id relabelling keeps every synapse (and the planted
    mapping follows the ids), the planted mapping is the generator's."""
    import numpy as np
    import bench
    import oracle
    import synth
    cfg = synth.NetConfig(name="t", M=2000, P=8, n_vn=2, K=12, uniform_all=False, n_part=8, n_vn_t=2,
                          n_remote=2, seed=6)
    g = synth.make_network(cfg)
    part = np.random.default_rng(2).integers(0, 8, g.M).astype(np.int32)
    assert bench._objective(g, part) == oracle.cut(g, part)
    assert bench._objective(g, part, chunk=37) == oracle.cut(g, part)
    assert np.array_equal(bench.oracle_free_planted(g.M, 8), oracle.partition_planted(g.M, 8))
    h, perm = bench._permuted(g, 5)
    src_g = np.repeat(np.arange(g.M), np.diff(g.syn_ptr))
    src_h = np.repeat(np.arange(h.M), np.diff(h.syn_ptr))
    a = sorted(zip(perm[src_g].tolist(), perm[g.tgt.astype(np.int64)].tolist(), g.w.tolist(), g.d.tolist()))
    b = sorted(zip(src_h.tolist(), h.tgt.tolist(), h.w.tolist(), h.d.tolist()))
    assert a == b
    planted = oracle.partition_planted(g.M, 8)
    assert oracle.cut(h, planted[np.argsort(perm)]) == oracle.cut(g, planted)


def test_traffic_entries_scale_and_go_stale(tmp_path, monkeypatch):
    """roofline.traffic from profiles/traffic.json: a "kernel@M" entry wins
    over the kernel's own; an entry scales by neurons or by synaptic events
    per step as it says; an entry taken on other kernel code gives null."""
    import json
    import bench
    (tmp_path / "profiles").mkdir()
    t = {"k": {"source_sha": "s1", "events_per_step": 100.0, "dram_bytes_per_step": 800.0, "neurons": 10},
         "k@5000": {"source_sha": "s1", "scale_by": "neurons", "neurons": 500, "events_per_step": 1.0,
                    "dram_bytes_per_step": 7000.0}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(t))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "s1")
    assert bench.load_traffic("k", 250.0, 64) == 800.0 * 250.0 / 100.0
    assert bench.load_traffic("k", 250.0, 5000) == 7000.0 * 5000 / 500
    assert bench.load_traffic("other", 250.0, 64) is None
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "s2")
    assert bench.load_traffic("k", 250.0, 64) is None


def test_source_hash_ignores_comments():
    """The hash that dates a capture covers code, not comments or blank lines."""
    import bench
    a = "int f(int x)\n{\n    return x + 1;  // one more\n}\n"
    b = "/* doc\n   more */\nint f(int x)\n{\n\n    return x + 1;\n}\n"
    c = "int f(int x)\n{\n    return x + 2;\n}\n"
    assert bench._code_only(a) == bench._code_only(b) != bench._code_only(c)
