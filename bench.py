"""Benchmark: one simulation step of a partitioned LIF network on GB300.

A "step" is one pass of the whole hot path: ring intake + Poisson drive, LIF
update and threshold, spike compaction, level-1 bucketing by destination
virtual node, level-2 relay expansion, CSR fan-out delivery.  The workload is
the 1,048,576-neuron network (64 partitions over 16 virtual nodes of 4,
1,000 synapses per neuron, 70/20/10 locality, delays 1-8 steps, Poisson
drive), synthetic and seeded.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Multi-GPU runs (torchrun) are independent
replicas of the same network with different drive seeds (weak scaling, no
collective on the data path).  `--impl reference` times the CPU oracle, the
plain sequential simulator used by the tests, on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "synaptic events/s & sim steps/s vs HBM roofline; batched/adjoint vs plain"
DELIVERY = {"ring": 0, "arrival": 1, "auto": 2, "owner": 3}
UNIT = "synaptic events/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ multi-rank
def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1
    import torch.distributed as dist
    backend = os.environ.get("SNN_BENCH_BACKEND") or ("nccl" if _cuda_ok() else "gloo")
    dist.init_process_group(backend=backend)
    return dist, dist.get_rank(), dist.get_world_size()


def _cuda_ok():
    import torch
    return torch.cuda.is_available()


def barrier(dist):
    if dist is not None:
        if dist.get_backend() == "nccl":
            import torch
            dist.barrier(device_ids=[torch.cuda.current_device()])
        else:
            dist.barrier()


def reduce_over_ranks(dist, events: float, ms: float, extra: float = 0.0):
    """Whole-job aggregate: summed work, maximum time over ranks."""
    if dist is None:
        return events, ms, extra
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    a = torch.tensor([events, extra], dtype=torch.float64, device=dev)
    b = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(a, op=dist.ReduceOp.SUM)
    dist.all_reduce(b, op=dist.ReduceOp.MAX)
    return float(a[0]), float(b[0]), float(a[1])


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled in the background."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.p = None
        self.t = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.p.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        if self.t is not None:
            self.t.join(timeout=5)

    def summary(self, t0: float, t1: float):
        rows = [r for ts, r in self.rows if t0 - 0.06 <= ts <= t1 + 0.06] or [r for _, r in self.rows]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ workload
def workload(seed_offset: int = 0, neurons: int = 0, config: str = "scale"):
    import synth
    cfg = {"scale": synth.SCALE, "paper": synth.PAPER_SHARE, "tiny": synth.TINY}[config]
    if neurons and neurons != cfg.M:
        # same per-neuron statistics on a smaller or larger network (profiling cases)
        cfg = cfg.scaled(M=neurons, name="%s-%dn-%dp-%dvn-k%d" % (config, neurons, cfg.P, cfg.n_vn, cfg.K))
    dyn = cfg.dyn
    if seed_offset:
        import dataclasses
        dyn = dataclasses.replace(dyn, drive_seed=dyn.drive_seed + seed_offset)
        cfg = cfg.scaled(dyn=dyn)
    return cfg


# per-unit algorithmic bytes of each phase (see the design notes)
def phase_bytes(M: int, d_steps: int, d: dict, gid: bool) -> list:
    upd = (18 + (4 if gid else 0)) * M * d_steps + 4 * d["spikes"]
    l1 = 12 * d["spikes"] + 6 * (d["l1_local"] + d["l1_xvn"])
    l1_entries = d["l1_local"] + d["l1_xvn"]
    l2_entries = d["l2_local"] + d["l2_peer"] + d["l2_relay_local"] + d["l2_relay_remote"]
    l2 = 12 * l1_entries + 24 * l2_entries
    dl = 8 * l2_entries + 6 * d["events"]
    return [upd, l1, l2, dl]


def model_params_of(snn, cfg):
    """snn_model_params of a workload's network recipe (the generator seed and
    statistics of `cfg`)."""
    return snn.model_params(n_neurons=cfg.M, n_parts=cfg.P, vn_size=cfg.vn_size, syn_per_neuron=cfg.K,
                            uniform=int(cfg.uniform_all), n_same_part=cfg.n_part, n_same_vn=cfg.n_vn_t,
                            n_remote=cfg.n_remote, max_delay=cfg.dmax, seed=cfg.seed, v_reset=cfg.dyn.v_reset,
                            v_th=cfg.dyn.v_th, frac_exc=cfg.frac_exc, mu_e=cfg.mu_e, sd_e=cfg.sd_e,
                            mu_i=cfg.mu_i, sd_i=cfg.sd_i)


def run_ours(args):
    import torch
    import paper_2205_07125_gb300 as snn

    dist, rank, world = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = workload(rank, args.neurons, args.config)
    K, W, PR = args.steps, args.warmup, args.preroll
    first = PR + W  # first timed step

    t_setup = time.time()
    # the network through the C ABI (snn_model_build: the seeded generator)
    model = snn.Model.build(model_params_of(snn, cfg))
    net = model.network()
    part, _ = snn.snn_partition(net, cfg.P, "planted")
    rt = snn.Routing(net, part, cfg.P, cfg.n_vn, "contiguous")
    info = rt.info()
    rec_steps = max(first + K, args.e2e_steps)
    raster_cap = int(cfg.M * rec_steps * 0.0015) + 100000
    prm = snn.sim_params(cfg.dyn, raster_cap=raster_cap, raster_steps=rec_steps, steps_per_graph=32,
                         pin_host_tables=1, defer_delayed=1 if args.defer else 0,
                         delivery=0 if args.defer else DELIVERY[args.delivery])
    sim = snn.Sim(net, rt, prm, device=dev)
    # untimed pre-roll from rest into the steady state, the launch shape
    # tuned there (every shape from the same state), warm-up, then EXACTLY K
    # timed steps
    sim.step(PR)
    if args.no_autotune:
        choice, tuned_ms = -1, -1.0
    else:
        choice, tuned_ms = sim.autotune(200)
    setup_s = time.time() - t_setup
    print("[bench] setup %.1f s (generate + partition + routing + upload + pre-roll + autotune: shape %d, "
          "%.4f ms/step)" % (setup_s, choice, tuned_ms), file=sys.stderr, flush=True)
    stream = sim.stream
    sim.step(W)
    if sim.sync_status() != 0:
        raise RuntimeError("device status after pre-roll and warm-up: %d" % sim.sync_status())
    c0 = sim.read_counts()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(dist)
    torch.cuda.synchronize()
    wall0 = time.time()
    # the NVTX range lets a profiler select the timed launches alone
    # (ncu --nvtx --nvtx-include "timed/")
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    sim.step(K)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    wall1 = time.time()
    barrier(dist)
    time.sleep(0.1)
    clocks.stop()
    ms = e0.elapsed_time(e1)
    st = sim.sync_status()
    if st != 0:
        raise RuntimeError("device status after the timed steps: %d" % st)
    c1 = sim.read_counts()
    dc = {k: c1[k] - c0[k] for k in c1}
    assert dc["steps"] == K
    events_all, ms_max, spikes_all = reduce_over_ranks(dist, float(dc["events"]), ms, float(dc["spikes"]))
    launches = sim.launches(K)
    persistent = launches == 1
    # algorithmic bytes of the timed window, from its own counters
    pbw = phase_bytes(cfg.M, K, dc, not info["identity_order"])
    step_bytes = sum(pbw) / K
    peak, peak_kind = _peaks()
    if persistent:
        # one cooperative launch runs every timed step: its duration is the
        # timed region, its algorithmic bytes those of the K steps
        kern = "k_persist"
        per_launch = step_bytes * K
        achieved = per_launch / (ms * 1e-3) / 1e9
    else:
        # two kernels per step: the step's bytes over the step's time
        kern = "k_update+k_route"
        per_launch = step_bytes
        achieved = step_bytes / (ms / K * 1e-3) / 1e9
    traffic = load_traffic(kern, events_all / world / K, cfg.M)
    roof = {"bound": "hbm", "kernel": kern, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak,
            "peak_source": ("measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                            else "fallback 6.8 TB/s"),
            "algorithmic_bytes_per_launch": per_launch,
            "bytes_per_step": dict(zip(["update", "level1", "level2", "deliver"], [x / K for x in pbw])),
            "window": "the timed steps' own counters",
            "traffic": (traffic * (K if persistent else 1)) if traffic is not None else None}
    # the deliveries are 32-bit reductions: the step's event rate against
    # the rate of the same reductions on random targets in an L2-sized
    # buffer (the input slots of delivery by arrival step, or the delay
    # ring), measured here
    arrival = 1000 <= choice < 2000
    n_red = cfg.M * 2 if arrival else cfg.M * (info["max_delay"] + 1)
    red_peak = red_rate(n_red, 1 << 22)
    atom = {"what": "synaptic events (one 32-bit reduction each) per second over the whole step, vs torch "
                    "index_add_ of 4M random int32 reductions into a buffer of the accumulators' size"
                    + (" (partition-owned delivery reduces in shared memory: context only)" if choice >= 2000 else ""),
            "buffer_mb": n_red * 4 / 1e6,
            "achieved": events_all / world / (ms_max * 1e-3), "peak": red_peak, "unit": "reductions/s",
            "frac": events_all / world / (ms_max * 1e-3) / red_peak}
    # spikes of the timed window (for the per-partition route traffic)
    ids_w, _ = sim.read_raster(first, first + K)

    # parts of a step over more steps (block 0's timers on the persistent
    # path, events around the two kernels on the graph path)
    NP = min(K, 1000)
    phase_ms = sim.profile_phases(NP)
    persistent_names = ["update", "compaction", "prefetch_and_queued_delivery", "barrier1_wait", "route_walk",
                        "route_delivery_and_copies", "next_drive_and_barrier2_wait"]
    phases = {"what": ("block 0 of the persistent kernel" if persistent else "k_update and k_route kernels")
                      + ", %d steps after the timed ones" % NP,
              "ms_per_step": dict(zip(persistent_names, [x / NP for x in phase_ms])) if persistent else
              {"k_update": phase_ms[0] / NP, "k_route": phase_ms[4] / NP}}
    print("[bench] timed %.3f ms for %d steps (steps %d..%d); parts ms per step %s" % (
        ms, K, first, first + K - 1, [round(x / NP, 5) for x in phase_ms]), file=sys.stderr, flush=True)

    # end to end through the C ABI: upload of every table from pinned host
    # memory, the steps, read-back of the raster and the counters
    e2e = None
    if not args.no_e2e:
        KE = args.e2e_steps
        torch.cuda.synchronize()
        barrier(dist)
        h0 = time.perf_counter()
        sim.reset(reupload=True)
        sim.step(KE)
        ids, off = sim.read_raster(0, KE)
        ce = sim.read_counts()
        h1 = time.perf_counter()
        e2e_ms = (h1 - h0) * 1e3
        e2e_events, e2e_ms_max, _ = reduce_over_ranks(dist, float(ce["events"]), e2e_ms)
        # the tables snn_sim_reset(reupload) copies: synapses (6 B), level-2 entries and pair
        # ids (20 B), level-1 entries and pair ids (10 B), per-neuron rows (l1_ptr, row, csr:
        # 20 B), source partitions (2 B), initial potentials (4 B), order maps when not identity
        h2d = (info["n_synapses"] * 6 + info["n_l2"] * 20 + info["n_l1"] * 10 + (cfg.M + 1) * 20
               + cfg.M * 6 + (0 if info["identity_order"] else cfg.M * 8))
        d2h = ids.nbytes + off.nbytes + 88
        e2e = {"value": e2e_events / (e2e_ms_max * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": h2d / KE, "d2h_bytes_per_step": d2h / KE, "steps": KE,
               "what": "snn_sim_reset(reupload) from pinned host tables + snn_step(%d) from rest + "
                       "snn_read_raster + snn_read_counts, host wall clock" % KE}

    result = {
        "metric": METRIC, "value": events_all / (ms_max * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": ms_max / K, "steps_per_s": K / (ms_max * 1e-3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+i32",
        "data": "synthetic (seeded generator behind snn_model_build; stands in for the paper's scanned brain "
                "model)",
        "config": {"workload": cfg.name, "neurons": cfg.M, "partitions": cfg.P,
                   "virtual_nodes": cfg.n_vn, "synapses": info["n_synapses"],
                   "synapses_per_neuron": cfg.K,
                   "locality": ("uniform" if cfg.uniform_all else "%d/%d/%d" % (cfg.n_part, cfg.n_vn_t, cfg.n_remote)),
                   "delays": "1-%d" % cfg.dmax,
                   "drive_lambda_per_step": cfg.dyn.drive_lambda, "w_ext": cfg.dyn.w_ext,
                   "parallelism": "replicas x%d" % world,
                   "step_window": {"preroll": PR, "autotune_steps": "250 per shape from step %d, then restored" % PR,
                                   "warmup": W, "first_timed_step": first,
                                   "last_timed_step": first + K - 1,
                                   "why": "untimed pre-roll from rest into the steady firing state"},
                   "l2": "inputs larger than L2: %.1f GB synapse CSR, the step's rows streamed from HBM"
                         % (info["n_synapses"] * 6 / 1e9),
                   "steps_per_graph": 32,
                   "execution": ("persistent cooperative kernel" if persistent else "CUDA graphs")
                                + (", minimum-delay batching" if args.defer else "")
                                + (", partition-owned delivery" if choice >= 2000 else
                                   ", delivery by arrival step" if choice >= 1000 else ", delay-ring delivery"),
                   "autotune": {"choice": choice, "ms_per_step": tuned_ms, "at_step": PR,
                                "meaning": "+1000 delivery by arrival step; 2000 + blocks per SM partition-owned "
                                           "delivery; else 0 graph path, or 100*mode + blocks per SM (mode 2 "
                                           "shared-memory state, 1 global 16-byte, 0 global scalar)"}},
        "spikes_per_step": spikes_all / world / K,
        "events_per_step": events_all / world / K,
        "rate_hz": spikes_all / world / K / cfg.M / (cfg.dyn.dt_ms * 1e-3),
        "roofline": roof,
        "atomic_roofline": atom,
        "phases": phases,
        "gpu_launches": launches,
        "clocks": clocks.summary(wall0, wall1),
        "e2e": e2e,
        "routing": routing_report(dc, info, rt, ids_w, K),
        "setup_s": setup_s,
    }
    # the GPU on the oracle's sample window (the first steps from rest)
    NS = oracle_sample_steps(cfg)
    sim.reset()
    ca = sim.read_counts()
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(NS)
    e1.record(stream)
    torch.cuda.synchronize()
    same_ms = e0.elapsed_time(e1)
    same_ev = sim.read_counts()["events"] - ca["events"]
    sim.close()
    del sim
    rt.close()
    del rt, net, model
    if rank == 0 and world == 1 and not args.no_forms:
        result["forms"] = forms_report(args, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(cfg, NS)
        cb["gpu_same_window"] = {"value": same_ev / (same_ms * 1e-3), "unit": UNIT,
                                 "what": "this GPU on the same steps 0..%d from rest" % (NS - 1)}
        result["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def routing_report(dc, info, rt, ids, K):
    """Messages of the timed window: per spike on each route (device
    counters), per partition (snn_routing_traffic over the window's spikes)
    with the peak -- the busiest partition, the paper's comparison -- for the
    direct route and the two-level route under each relay policy, and the
    static connections per partition."""
    import paper_2205_07125_gb300 as snn
    S = max(1, dc["spikes"])
    two = dc["l1_xvn"] + dc["l2_peer"] + dc["l2_relay_remote"]
    cd, ct = rt.connections()
    per_part = {}
    for pol in snn.RELAY_POLICIES:
        tr = rt.traffic(ids, pol)
        if "direct" not in per_part:
            d = tr["direct_out"] / K
            per_part["direct"] = {"sent_peak_per_step": float(d.max()), "sent_mean_per_step": float(d.mean()),
                                  "received_peak_per_step": float((tr["direct_in"] / K).max())}
        t = tr["two_level_out"] / K
        per_part["two_level_" + pol] = {"sent_peak_per_step": float(t.max()), "sent_mean_per_step": float(t.mean()),
                                        "received_peak_per_step": float((tr["two_level_in"] / K).max())}
    hist = lambda a: {int(k): int(v) for k, v in zip(*np.unique(a, return_counts=True))}
    return {
        "messages_per_spike": {"direct": dc["direct"] / S, "direct_cross_vn": dc["direct_xvn"] / S,
                               "two_level": two / S, "two_level_l1_cross_vn": dc["l1_xvn"] / S,
                               "two_level_l2_relay_forward": dc["l2_relay_remote"] / S},
        "bytes_per_step": {"direct": 4 * dc["direct"] / dc["steps"],
                           "two_level": 4 * two / dc["steps"]},
        "per_partition": per_part,
        "per_partition_what": "messages per partition per step over the timed window (one message = one "
                              "(spike, destination) pair); peak = the busiest partition",
        "connections_per_partition": {"direct_mean": float(cd.mean()), "direct_max": int(cd.max()),
                                      "two_level_mean": float(ct.mean()), "two_level_max": int(ct.max()),
                                      "direct_histogram": hist(cd), "two_level_histogram": hist(ct)},
    }


def _code_only(text: str) -> str:
    """C++ source without comments and blank lines (string literals in these
    files hold no comment markers)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(l.rstrip() for l in text.splitlines() if l.strip())


def kernel_source_sha() -> str:
    """Hash of the step-kernel code, comments left out (a capture taken on
    other code is stale)."""
    import hashlib
    hs = hashlib.sha256()
    for f in ("snn_step.cuh", "snn_sim.cu"):
        with open(os.path.join(ROOT, "paper_2205_07125_gb300", "csrc", f), encoding="utf-8") as fh:
            hs.update(_code_only(fh.read()).encode())
    return hs.hexdigest()[:16]


def load_traffic(kernel: str, events_per_step: float, M: int):
    """DRAM bytes per step of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source (else null).  The capture runs a
    smaller network of the same recipe, scaled to this one by the entry's
    unit: synaptic events per step (the neuron state on chip, the traffic is
    the synapse and routing-table reads of the step's spikes), or neurons
    (where two capture sizes agree per neuron-step and not per event)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    ent = t.get("%s@%d" % (kernel, M)) or t.get(kernel)
    if not ent or ent.get("source_sha") != kernel_source_sha():
        return None
    if ent.get("scale_by") == "neurons":
        return ent["dram_bytes_per_step"] * M / ent["neurons"]
    return ent["dram_bytes_per_step"] * events_per_step / ent["events_per_step"]


def red_rate(n_ring: int, n: int, reps: int = 20) -> float:
    """32-bit atomic adds per second of torch index_add_ with n random targets
    in an int32 buffer of n_ring entries (L2-resident like the delay ring)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(7)
    buf = torch.zeros(n_ring, dtype=torch.int32, device="cuda")
    idx = torch.randint(0, n_ring, (n,), device="cuda", generator=g)
    val = torch.ones(n, dtype=torch.int32, device="cuda")
    for _ in range(3):
        buf.index_add_(0, idx, val)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        buf.index_add_(0, idx, val)
    e1.record()
    torch.cuda.synchronize()
    return n * reps / (e0.elapsed_time(e1) * 1e-3)


# ------------------------------------------------------------------ CPU oracle
def oracle_sample_steps(cfg) -> int:
    """Steps of the CPU oracle's bounded sample (from rest), sized for 10-30 s
    of sequential work: 1000 at 4,096 neurons, about 30 at 5,000,000."""
    return int(max(20, min(1000, round(1.5e8 / (cfg.M + 40.0 * cfg.M * cfg.K / 1000.0)))))


def oracle_sample(cfg, steps: int) -> dict:
    """The CPU oracle, as it stands, on one host core: the first `steps`
    steps from rest of the workload's network (its own copy from the seeded
    generator), timed; the same sample in both bench arms."""
    import synth
    import oracle
    g = synth.make_network(cfg)
    P = cfg.P
    t0 = time.time()
    o = oracle.Oracle(g, P, oracle.partition_planted(g.M, P), cfg.n_vn,
                      oracle.group_contiguous(P, cfg.n_vn), cfg.dyn)
    setup = time.time() - t0
    t0 = time.perf_counter()
    o.run(steps, raster=False, hashes=False)
    el = time.perf_counter() - t0
    c = o.count_dict()
    return {"value": c["events"] / el, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
            "steps_per_s": steps / el, "spikes_per_step": c["spikes"] / steps, "seconds": el,
            "sample": "steps 0..%d from rest of the same %d-neuron network, sequential C oracle on one of the "
                      "host's %d cores (%.1f s timed, %.1f s setup untimed)"
                      % (steps - 1, g.M, os.cpu_count(), el, setup)}


def run_reference(args):
    """Reference arm: the CPU oracle timed on the host, rank 0 only: the
    first steps from rest of the workload's network, the sample the repo
    arm's cpu_baseline times."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    cfg = workload(0, args.neurons, args.config if args.config in ("scale", "paper", "tiny") else "paper")
    steps = oracle_sample_steps(cfg)
    r = oracle_sample(cfg, steps)
    v = r["value"]
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": steps, "warmup": 0, "ms_per_step": r["seconds"] * 1e3 / steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+i32", "data": "synthetic",
           "config": {"workload": cfg.name, "neurons": cfg.M, "partitions": cfg.P,
                      "virtual_nodes": cfg.n_vn, "synapses": cfg.M * cfg.K},
           "cpu_baseline": {k: r[k] for k in ("value", "unit", "cores", "host_cores", "kind", "sample")},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def batch_form(dev, n_nets: int, K: int, W: int, separate_steps: int, seed: int = 3000) -> dict:
    """The batched form: n_nets independent networks of uneven sizes (the
    batched workload's distribution: 10k-500k neurons, 4-32 partitions,
    out-degree 100-1000, scaled drives) stepped by one sim in the autotuned
    shape, against the same networks stepped one after another by one plain
    sim each (the same work, one launch per network instead of one in all)."""
    import torch
    import synth
    import paper_2205_07125_gb300 as snn

    t_setup = time.time()
    cfgs = synth.batch_configs(n=n_nets, seed=seed)
    b = synth.make_batch(cfgs)
    net = snn.Network.from_synth(b.net)
    rt = snn.Routing(net, b.part, b.P, b.n_vn, "contiguous")
    info = rt.info()
    plist = [snn.sim_params(c.dyn, steps_per_graph=32, delivery=snn.SNN_DELIVER_AUTO) for c in cfgs]
    sim = snn.Sim(net, rt, plist[0], device=dev, batch=(b.off, plist))
    choice, tuned_ms = sim.autotune(200)
    setup_s = time.time() - t_setup
    stream = sim.stream
    sim.step(W)
    if sim.sync_status() != 0:
        raise RuntimeError("device status after warm-up: %d" % sim.sync_status())
    c0 = sim.read_counts()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if sim.sync_status() != 0:
        raise RuntimeError("device status after the timed steps: %d" % sim.sync_status())
    c1 = sim.read_counts()
    dc = {k: c1[k] - c0[k] for k in c1}
    launches = sim.launches(K)
    pb = phase_bytes(b.net.M, K, dc, not info["identity_order"])
    sim.close()
    del sim
    rt.close()
    # the same networks, one plain sim each, stepped one after another
    KS = min(K, separate_steps)
    sep_ms, sep_ev = 0.0, 0.0
    for c, g, p in zip(cfgs, b.nets, plist):
        n1 = snn.Network.from_synth(g)
        part, _ = snn.snn_partition(n1, c.P, "planted")
        r1 = snn.Routing(n1, part, c.P, c.n_vn, "contiguous")
        s1 = snn.Sim(n1, r1, p, device=dev)
        s1.step(W)
        a0 = s1.read_counts()
        torch.cuda.synchronize()
        e0.record(s1.stream)
        s1.step(KS)
        e1.record(s1.stream)
        torch.cuda.synchronize()
        sep_ms += e0.elapsed_time(e1)
        sep_ev += s1.read_counts()["events"] - a0["events"]
        s1.close()
        r1.close()
        del s1, r1, n1
    value = dc["events"] / (ms * 1e-3)
    sep_rate = sep_ev / (sep_ms * 1e-3)
    return {"networks": len(cfgs), "neurons": b.net.M, "synapses": b.net.E, "partitions": b.P,
            "virtual_nodes": b.n_vn, "steps": K, "warmup": W, "ms_per_step": ms / K, "value": value,
            "unit": UNIT, "spikes_per_step": dc["spikes"] / K, "events_per_step": dc["events"] / K,
            "rate_hz": dc["spikes"] / K / b.net.M / 1e-4, "step_bytes": sum(pb) / K, "gpu_launches": launches,
            "autotune": {"choice": choice, "ms_per_step": tuned_ms}, "setup_s": setup_s,
            "vs_plain": {"what": "the same %d networks, one plain sim each (default launch shape), stepped one "
                                 "after another (%d steps each)" % (len(cfgs), KS),
                         "value": sep_rate, "unit": UNIT, "batched_over_plain": value / sep_rate}}


def adjoint_form(dev, T: int = 500, CK: int = 50, reps: int = 1, warm: int = 1, rank: int = 0) -> dict:
    """The adjoint form: 131,072 neurons in 8 partitions over 2 VNs, 500
    synapses per neuron (scale locality mix), T steps forward with membrane
    checkpoints every CK, then the surrogate-gradient backward; against the
    plain step of the same network on the same GPU."""
    import torch
    import synth
    import paper_2205_07125_gb300 as snn

    cfg = synth.NetConfig(name="adjoint-131072n-8p-2vn-k500", M=131072, P=8, n_vn=2, K=500, uniform_all=False,
                          n_part=350, n_vn_t=100, n_remote=50, dmax=8, seed=1004 + rank, steps=T,
                          dyn=synth.Dynamics(drive_lambda=0.8, w_ext=89, drive_seed=2004 + rank))
    t_setup = time.time()
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    part, _ = snn.snn_partition(net, cfg.P, "planted")
    rt = snn.Routing(net, part, cfg.P, cfg.n_vn, "contiguous")
    prm = snn.sim_params(cfg.dyn, raster_cap=cfg.M * T // 10)
    a = snn.Adjoint(net, g.is_exc, rt, prm, snn.adjoint_params(T=T, ckpt_every=CK), device=dev)
    n_pop = a.n_pop
    rng = np.random.default_rng(4000)
    G = np.ones((n_pop, n_pop), np.float32)
    lam = np.full(n_pop, 0.8, np.float32)
    target = (5.0 + 10.0 * rng.random(n_pop)) * 1e-4  # spikes per neuron per step (5-15 Hz)
    setup_s = time.time() - t_setup
    for _ in range(max(1, warm)):
        r = a.forward(G, lam)
        a.backward(2 * (r.astype(np.float64) - target) / n_pop)
    fw = bw = 0.0
    for _ in range(max(1, reps)):
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        r = a.forward(G, lam)
        h1 = time.perf_counter()
        dG, dlam = a.backward(2 * (r.astype(np.float64) - target) / n_pop)
        h2 = time.perf_counter()
        fw += h1 - h0
        bw += h2 - h1
    fw /= max(1, reps)
    bw /= max(1, reps)
    spikes = a.spikes
    a.close()
    # the plain step of the same network (its own Poisson drive), same steps
    sim = snn.Sim(net, rt, snn.sim_params(cfg.dyn, delivery=snn.SNN_DELIVER_AUTO), device=dev)
    sim.autotune(100)
    sim.step(100)
    c0 = sim.read_counts()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(sim.stream)
    sim.step(T)
    e1.record(sim.stream)
    torch.cuda.synchronize()
    pms = e0.elapsed_time(e1)
    pev = sim.read_counts()["events"] - c0["events"]
    sim.close()
    rt.close()
    it = fw + bw
    return {"workload": cfg.name, "neurons": cfg.M, "partitions": cfg.P, "virtual_nodes": cfg.n_vn,
            "synapses": g.E, "steps": T, "checkpoint_every": CK, "populations": n_pop,
            "parameters": "%d gains + %d drive rates" % (n_pop * n_pop, n_pop),
            "surrogate": "1/(1+5|V-theta|)^2, reset detached",
            "timing": "host wall clock of snn_adjoint_forward / _backward (each synchronises), %d run(s)" % reps,
            "forward_ms": fw * 1e3, "backward_ms": bw * 1e3, "forward_spikes": spikes,
            "value": spikes * cfg.K / it, "unit": UNIT,
            "rates_hz": [float(x) * 1e4 for x in r],
            "grad_norm": float(np.sqrt((dG ** 2).sum() + (dlam ** 2).sum())), "setup_s": setup_s,
            "vs_plain": {"what": "plain step of the same network, %d steps, CUDA events" % T,
                         "plain_ms_per_step": pms / T, "plain_events_per_s": pev / (pms * 1e-3),
                         "forward_over_plain_time": fw * 1e3 / pms,
                         "forward_backward_over_plain_time": it * 1e3 / pms}}


def forms_report(args, dev) -> dict:
    """The batched and adjoint forms against the plain step (the metric's
    "batched/adjoint vs plain"), at reduced cost for the default line: the
    first --form-nets networks of the batched workload (seed 3000) for 500
    steps, and the adjoint workload at full size (500 steps, checkpoints
    every 50, one timed forward + backward)."""
    t0 = time.time()
    bf = batch_form(dev, args.form_nets, 500, 20, 500)
    af = adjoint_form(dev, 500, 50, reps=1, warm=1)
    out = {"batched_over_plain": bf["vs_plain"]["batched_over_plain"],
           "adjoint_fwd_bwd_over_plain": af["vs_plain"]["forward_backward_over_plain_time"],
           "batched": bf, "adjoint": af, "seconds": time.time() - t0}
    print("[bench] forms: batched/plain %.2f, adjoint (fwd+bwd)/plain %.1f (%.0f s)"
          % (out["batched_over_plain"], out["adjoint_fwd_bwd_over_plain"], out["seconds"]),
          file=sys.stderr, flush=True)
    return out


def run_batch(args):
    """--config batch: the batched form at the workload's full count of
    networks, one JSON line."""
    import torch
    dist, rank, world = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    wall0 = time.time()
    bf = batch_form(dev, args.batch_nets, args.steps, args.warmup, args.separate_steps, seed=3000 + 100 * rank)
    wall1 = time.time()
    clocks.stop()
    events_all, ms_max, _ = reduce_over_ranks(dist, bf["events_per_step"] * args.steps, bf["ms_per_step"] * args.steps)
    peak, peak_kind = _peaks()
    per_launch = bf["step_bytes"] * (args.steps if bf["gpu_launches"] == 1 else 1)
    t_launch = ms_max if bf["gpu_launches"] == 1 else ms_max / args.steps
    result = {
        "metric": METRIC, "value": events_all / (ms_max * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "steps_per_s": args.steps / (ms_max * 1e-3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+i32",
        "data": "synthetic (seeded generator; independent networks stand in for a batch of models)",
        "config": {"workload": "batch-%dnets-%dn" % (bf["networks"], bf["neurons"]), "networks": bf["networks"],
                   "neurons": bf["neurons"], "synapses": bf["synapses"], "partitions": bf["partitions"],
                   "virtual_nodes": bf["virtual_nodes"], "sizes": "log-uniform 10k-500k",
                   "synapses_per_neuron": "uniform 100-1000", "partitions_per_network": "4-32 (VNs of 2)",
                   "drive": "scale drive x r/10, r ~ U[5, 15] Hz", "parallelism": "replicas x%d" % world,
                   "execution": "autotuned shape %d" % bf["autotune"]["choice"],
                   "l2": "inputs larger than L2: %.1f GB synapse CSR" % (bf["synapses"] * 6 / 1e9)},
        "spikes_per_step": bf["spikes_per_step"], "events_per_step": bf["events_per_step"], "rate_hz": bf["rate_hz"],
        "roofline": {"bound": "hbm", "kernel": "k_persist" if bf["gpu_launches"] == 1 else "k_update+k_route",
                     "achieved": per_launch / (t_launch * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": per_launch / (t_launch * 1e-3) / 1e9 / peak,
                     "peak_source": ("measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                                     else "fallback 6.8 TB/s"),
                     "algorithmic_bytes_per_launch": per_launch, "traffic": None},
        "vs_plain": bf["vs_plain"], "autotune": bf["autotune"], "gpu_launches": bf["gpu_launches"],
        "clocks": clocks.summary(wall0, wall1), "e2e": None, "setup_s": bf["setup_s"],
    }
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_adjoint(args):
    """--config adjoint: the adjoint form, one JSON line."""
    import torch
    dist, rank, world = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    T, CK = 500, 50
    af = adjoint_form(dev, T, CK, reps=max(1, min(args.steps // T, 10)), warm=max(1, args.warmup // 50), rank=rank)
    it = (af["forward_ms"] + af["backward_ms"]) * 1e-3
    result = {
        "metric": METRIC, "value": af["value"], "unit": UNIT, "n_gpus": world, "steps": T, "warmup": args.warmup,
        "ms_per_step": it * 1e3 / T, "steps_per_s": T / it, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (gradients f64)", "data": "synthetic",
        "config": {k: af[k] for k in ("workload", "neurons", "partitions", "virtual_nodes", "synapses", "steps",
                                      "checkpoint_every", "populations", "parameters", "surrogate", "timing")},
        "forward_ms": af["forward_ms"], "backward_ms": af["backward_ms"], "forward_spikes": af["forward_spikes"],
        "rates_hz": af["rates_hz"], "grad_norm": af["grad_norm"], "vs_plain": af["vs_plain"],
        "setup_s": af["setup_s"],
    }
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _permuted(g, seed):
    """The network g with neuron ids relabelled by a seeded permutation (new id
    = perm[old]), so that a partitioner cannot read the planted structure
    off contiguous id ranges."""
    import synth
    rng = np.random.default_rng(seed)
    perm = rng.permutation(g.M).astype(np.int64)
    inv = np.argsort(perm)
    deg = np.diff(g.syn_ptr)[inv]
    syn_ptr = np.zeros(g.M + 1, np.int64)
    syn_ptr[1:] = np.cumsum(deg)
    order = np.concatenate([np.arange(g.syn_ptr[i], g.syn_ptr[i + 1]) for i in inv])
    return synth.Network(g.cfg, syn_ptr, perm[g.tgt[order].astype(np.int64)].astype(np.uint32), g.w[order],
                         g.d[order], g.v0[inv], g.is_exc[inv]), perm


def _route_traffic(g, part, vn_of_part, relay_of, spikes):
    """Messages per partition of the direct route and of the two-level route
    for spike counts `spikes` [M] (messages = one (spike, destination) pair):
    direct: partition p(i) sends one per destination partition q != p(i);
    two-level: p(i) sends one per destination VN g != vn(p(i)) (level 1) and
    one per peer partition of its own VN; relay_of[g, p(i)] forwards one per
    partition of g holding targets other than itself (level 2)."""
    P = int(part.max()) + 1
    src = np.repeat(np.arange(g.M, dtype=np.int64), np.diff(g.syn_ptr))
    q = part[g.tgt.astype(np.int64)].astype(np.int64)
    pairs = np.unique(src * P + q)                       # (neuron, destination partition) with targets
    i, qq = pairs // P, pairs % P
    ps = part[i].astype(np.int64)
    w = spikes[i].astype(np.float64)
    direct = np.bincount(ps[qq != ps], weights=w[qq != ps], minlength=P)
    vq, vp = vn_of_part[qq], vn_of_part[ps]
    peer = (vq == vp) & (qq != ps)
    l1_intra = np.bincount(ps[peer], weights=w[peer], minlength=P)
    n_vn = int(vn_of_part.max()) + 1
    rem = vq != vp
    iv = np.unique(i[rem] * n_vn + vq[rem])              # (neuron, destination VN) level-1 messages
    l1_x = np.bincount(part[iv // n_vn], weights=spikes[iv // n_vn].astype(np.float64), minlength=P)
    r = relay_of[vq[rem], ps[rem]]                        # relay partition of each remote pair
    fwd = qq[rem] != r
    l2 = np.bincount(r[fwd], weights=w[rem][fwd], minlength=P)
    return direct, l1_intra + l1_x + l2, l2


def _relay_policies(vn_of_part, relay_vn, load):
    """Relay maps relay_of[g, p] (destination VN g, source partition p):
    per source VN (the library's: member h mod s of g, h = vn(p)); per source
    partition (member p mod s); load-balanced per source partition (the
    (g, p) pairs in decreasing forwarding load go to the least-loaded member
    of g, longest-processing-time greedy).  load[g, p] = messages."""
    n_vn, P = load.shape
    members = [np.nonzero(vn_of_part == gg)[0] for gg in range(n_vn)]
    by_vn = np.array([[relay_vn[gg, vn_of_part[p_]] for p_ in range(P)] for gg in range(n_vn)])
    by_part = np.array([[members[gg][p_ % len(members[gg])] for p_ in range(P)] for gg in range(n_vn)])
    bal = np.zeros((n_vn, P), np.int64)
    for gg in range(n_vn):
        acc = np.zeros(len(members[gg]))
        for p_ in np.argsort(-load[gg], kind="stable"):
            k = int(np.argmin(acc))
            bal[gg, p_] = members[gg][k]
            acc[k] += load[gg, p_]
    return {"per_source_vn (library)": by_vn, "per_source_partition": by_part, "load_balanced": bal}


def run_partition_study(args):
    """Partition quality (random vs Algorithm 1 vs planted) and relay policy
    (per source VN vs per source partition vs load-balanced) on seeded
    networks with relabelled ids: cut, per-partition traffic of the direct
    and two-level routes per step and the peak (max over partitions) over
    mean ratio, from a GPU run's spikes; for VNs of 4 and of 8 partitions."""
    import synth
    import paper_2205_07125_gb300 as snn

    M, P, K = args.study_neurons, 16, 200
    T = 1000
    out = {"ids": "relabelled by a seeded permutation", "steps": T, "studies": {}}
    for n_vn in (4, 2):
        cfg = synth.NetConfig(name="study-%dn-%dp-%dvn-k%d" % (M, P, n_vn, K), M=M, P=P, n_vn=n_vn, K=K,
                              uniform_all=False, n_part=140, n_vn_t=40, n_remote=20, dmax=8, seed=1005,
                              dyn=synth.Dynamics(drive_lambda=0.8, w_ext=96, drive_seed=2005))
        g0 = synth.make_network(cfg)
        g, perm = _permuted(g0, 77)
        net = snn.Network.from_synth(g)
        src = np.repeat(np.arange(M, dtype=np.int64), np.diff(g.syn_ptr))
        tgt = g.tgt.astype(np.int64)
        study = {}
        for mode in ("random", "greedy", "planted"):
            t0 = time.time()
            if mode == "planted":
                part = oracle_free_planted(M, P)[np.argsort(perm)]  # the generator's partitions, new ids
                stats = {"objective": None}
            else:
                part, stats = snn.snn_partition(net, P, mode, iters=4, seed=11)
            t_part = time.time() - t0
            part = part.astype(np.int64)
            rt = snn.Routing(net, part, P, n_vn, "greedy", iters=4, seed=11)
            vn, relay = rt.groups()
            vn = vn.astype(np.int64)
            cd, ct = rt.connections()
            sim = snn.Sim(net, rt, snn.sim_params(cfg.dyn, raster_cap=M * T // 20, raster_steps=T),
                          device="cuda:0")
            sim.step(T)
            assert sim.sync_status() == 0
            ids, off = sim.read_raster(0, T)
            counts = sim.read_counts()
            sim.close()
            spikes = np.bincount(ids.astype(np.int64), minlength=M)
            lib = _relay_policies(vn, relay.astype(np.int64), np.zeros((n_vn, P)))["per_source_vn (library)"]
            direct, two, _ = _route_traffic(g, part, vn, lib, spikes)
            # forwarding load of each (destination VN, source partition)
            pq = np.unique(src * P + part[tgt])
            i, qq = pq // P, pq % P
            gv, hv = vn[qq], vn[part[i]]
            rem = gv != hv
            load = np.zeros((n_vn, P))
            np.add.at(load, (gv[rem], part[i][rem]), spikes[i[rem]])
            policies = {}
            for name, rmap in _relay_policies(vn, relay.astype(np.int64), load).items():
                _, two_r, l2_r = _route_traffic(g, part, vn, rmap, spikes)
                policies[name] = {"l2_forward_peak_per_step": float(l2_r.max() / T),
                                  "l2_forward_peak_over_mean": float(l2_r.max() / max(1e-9, l2_r.mean())),
                                  "two_level_peak_per_step": float(two_r.max() / T)}
            study[mode] = {
                "partition_s": t_part, "objective": stats.get("objective"),
                "cut_fraction": float((part[src] != part[tgt]).mean()),
                "spikes_per_step": float(spikes.sum() / T),
                "direct_msgs_per_step": {"total": float(direct.sum() / T), "peak": float(direct.max() / T),
                                         "peak_over_mean": float(direct.max() / max(1e-9, direct.mean()))},
                "two_level_msgs_per_step": {"total": float(two.sum() / T), "peak": float(two.max() / T),
                                            "peak_over_mean": float(two.max() / max(1e-9, two.mean()))},
                "library_direct_count_matches": bool(counts["direct"] == int(round(direct.sum()))),
                "static_connections": {"direct_mean": float(cd.mean()), "direct_max": int(cd.max()),
                                       "two_level_mean": float(ct.mean()), "two_level_max": int(ct.max())},
                "relay_policy": policies,
            }
            print("[study] n_vn %d %s: cut %.3f, direct peak/step %.1f, two-level peak/step %.1f"
                  % (n_vn, mode, study[mode]["cut_fraction"], direct.max() / T, two.max() / T),
                  file=sys.stderr, flush=True)
            rt.close()
        out["studies"][cfg.name] = study
    print(json.dumps(out), flush=True)


def _objective(g, part, chunk=1 << 24):
    """Algorithm 1's objective: sum over synapses i -> j with part(i) !=
    part(j) of W_i W_j, W = out-degree (numpy, in chunks of synapses)."""
    W = np.diff(g.syn_ptr).astype(np.int64)
    part = np.asarray(part, np.int64)
    tot = 0
    for i0 in range(0, g.M, max(1, chunk // max(1, int(W.max(initial=1))))):
        i1 = min(g.M, i0 + max(1, chunk // max(1, int(W.max(initial=1)))))
        src = np.repeat(np.arange(i0, i1, dtype=np.int64), W[i0:i1])
        tgt = g.tgt[g.syn_ptr[i0]:g.syn_ptr[i1]].astype(np.int64)
        cut = part[src] != part[tgt]
        tot += int((W[src[cut]] * W[tgt[cut]]).sum())
    return tot


def routing_compare(snn, net, part, P, n_vn, grouping, name):
    """Routing tables (Algorithm 2 grouping + level-1/level-2 tables) built on
    the host (all cores) and on the GPU for the same mapping: times and a
    byte comparison of the tables."""
    import torch
    part = np.ascontiguousarray(part, np.int32)
    t0 = time.perf_counter()
    rt_h = snn.Routing(net, part, P, n_vn, grouping)
    t_h = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rt_d = snn.Routing(net, part, P, n_vn, grouping, build="device", device="cuda:0")
    t_d = time.perf_counter() - t0
    same = all(np.array_equal(rt_h.export(t).view(np.uint8), rt_d.export(t).view(np.uint8))
               for t in ("syn_td", "syn_w", "l2", "l1_vn", "l1_l2", "l1_ptr", "l1_pair", "l2_pair", "csr"))
    r = {"host_s": t_h, "host_threads": os.cpu_count(), "device_s": t_d, "speedup": t_h / t_d,
         "tables_equal": bool(same), "grouping": grouping, "n_l1": rt_d.info()["n_l1"], "n_l2": rt_d.info()["n_l2"]}
    print("[partition] %s routing build: host %.2f s (%d threads), device %.2f s, tables equal %s"
          % (name, t_h, os.cpu_count(), t_d, same), file=sys.stderr, flush=True)
    rt_h.close()
    rt_d.close()
    return r


def run_partition_device(args):
    """Algorithm 1 on the GPU (batched growth, one cooperative launch per
    iteration) against the library's host greedy: wall time of the call
    (synapse lists to the device, in-lists, 4 iterations, labels back),
    objective and balance.  Rounds of one reproduce the host mapping bit for
    bit; the batched rounds are compared by objective with the planted
    partitions the generator used.  On the scale workload also the routing
    tables built by the host (all cores) and by the GPU, checked equal."""
    import torch
    import synth
    import paper_2205_07125_gb300 as snn

    torch.cuda.set_device(0)
    out = {"what": "Algorithm 1 partition time, s (lower is better); objective = sum over cut synapses of "
                   "W_i W_j", "networks": {}}
    # context and module load outside the timings
    tiny = synth.make_edges(64, [(i, (i + 1) % 64, 1, 1) for i in range(64)])
    snn.snn_partition_device(snn.Network.from_synth(tiny), 2, device="cuda:0")

    def device_run(net, P, batch, grow, iters):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        part, st = snn.snn_partition_device(net, P, batch=batch, grow=grow, iters=iters, seed=11,
                                            device="cuda:0")
        return part, st, time.perf_counter() - t0

    # the study network (65,536 neurons, 16 planted partitions, ids relabelled)
    M, P, K = args.study_neurons, 16, 200
    cfg = synth.NetConfig(name="study-%dn-%dp-k%d" % (M, P, K), M=M, P=P, n_vn=4, K=K, uniform_all=False,
                          n_part=140, n_vn_t=40, n_remote=20, dmax=8, seed=1005)
    g, perm = _permuted(synth.make_network(cfg), 77)
    net = snn.Network.from_synth(g)
    planted = oracle_free_planted(M, P)[np.argsort(perm)]
    res = {"neurons": M, "partitions": P, "synapses": int(g.syn_ptr[-1]), "ids": "relabelled",
           "planted_objective": _objective(g, planted)}
    t0 = time.perf_counter()
    part_h, st_h = snn.snn_partition(net, P, "greedy", iters=4, seed=11)
    res["host_greedy"] = {"s": time.perf_counter() - t0, "objective": st_h["objective"], "iters": 4,
                          "threads": 1}
    for batch, grow in ((1, 0), (64, 4), (1024, 4), (2048, 2)):
        part, st, sec = device_run(net, P, batch, grow, 4)
        r = {"s": sec, "objective": st["objective"], "max_over_min_weight": st["max_weight"] / max(1, st["min_weight"]),
             "speedup_vs_host": res["host_greedy"]["s"] / sec}
        if batch == 1:
            r["equals_host_mapping"] = bool(np.array_equal(part, part_h))
        res["device_batch%d_grow%d" % (batch, grow)] = r
        print("[partition] %s batch %d grow %d: %.3f s, objective %d (host %.3f s, %d; planted %d)"
              % (cfg.name, batch, grow, sec, st["objective"], res["host_greedy"]["s"], st_h["objective"],
                 res["planted_objective"]), file=sys.stderr, flush=True)
    res["routing_build"] = routing_compare(snn, net, part, P, 4, "greedy", cfg.name)
    out["networks"][cfg.name] = res

    if args.no_scale:
        print(json.dumps(out), flush=True)
        return
    # the scale workload (1,048,576 neurons, 64 planted partitions, 1.05e9 synapses)
    cfg = workload(0, 0, "scale")
    g = synth.make_network(cfg)
    net = snn.Network.from_synth(g)
    res = {"neurons": cfg.M, "partitions": cfg.P, "synapses": int(g.syn_ptr[-1]), "ids": "generator order",
           "planted_objective": _objective(g, oracle_free_planted(cfg.M, cfg.P))}
    for batch, grow, iters in ((2048, 2, 1), (2048, 2, 4), (1024, 4, 4)):
        part, st, sec = device_run(net, cfg.P, batch, grow, iters)
        res["device_batch%d_grow%d_iters%d" % (batch, grow, iters)] = {
            "s": sec, "objective": st["objective"],
            "objective_over_planted": st["objective"] / max(1, res["planted_objective"]),
            "max_over_min_weight": st["max_weight"] / max(1, st["min_weight"])}
        print("[partition] %s batch %d grow %d iters %d: %.3f s, objective / planted %.4f"
              % (cfg.name, batch, grow, iters, sec, st["objective"] / max(1, res["planted_objective"])),
              file=sys.stderr, flush=True)
    res["routing_build"] = routing_compare(snn, net, part, cfg.P, cfg.n_vn, "contiguous", cfg.name)
    if args.host_scale_iters > 0:
        t0 = time.perf_counter()
        _, st_h = snn.snn_partition(net, cfg.P, "greedy", iters=args.host_scale_iters, seed=11)
        res["host_greedy_iters%d" % args.host_scale_iters] = {
            "s": time.perf_counter() - t0, "objective": st_h["objective"], "threads": 1}
        print("[partition] %s host greedy iters %d: %.1f s" % (cfg.name, args.host_scale_iters,
                                                               time.perf_counter() - t0),
              file=sys.stderr, flush=True)
    out["networks"][cfg.name] = res
    print(json.dumps(out), flush=True)


def oracle_free_planted(M, P):
    """The generator's planted partitions: p owns ids floor(pM/P) .. floor((p+1)M/P)-1."""
    part = np.empty(M, np.int32)
    for p_ in range(P):
        part[M * p_ // P:M * (p_ + 1) // P] = p_
    return part


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--preroll", type=int, default=1500,
                    help="untimed steps from rest before the warm-up, into the steady firing state "
                         "(the paper share's rate settles after about 1,000 steps)")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--neurons", type=int, default=0,
                    help="network size with the workload's per-neuron statistics (profiling cases)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the sim's default launch shape (profiling one shape; SNN_PERSIST_* select it)")
    ap.add_argument("--e2e-steps", type=int, default=10000,
                    help="steps of the end-to-end leg (tables uploaded once, then the steps from rest)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batched and adjoint forms against the plain step")
    ap.add_argument("--form-nets", type=int, default=16,
                    help="networks of the batched form in the default line (--config batch: --batch-nets)")
    ap.add_argument("--defer", action="store_true",
                    help="minimum-delay batching: delay >= 2 synapses delivered during the next step's "
                         "table walk (persistent shared-memory shape)")
    ap.add_argument("--config", choices=("scale", "paper", "tiny", "batch", "adjoint", "partition",
                                         "partition-device"),
                    default="paper",
                    help="paper: the paper-shaped per-GPU share, 5,000,000 neurons / 256 partitions (the "
                         "headline workload); scale: 1,048,576 neurons / 64 partitions; "
                         "tiny: 4,096 neurons; batch: 64 independent networks of uneven sizes; "
                         "adjoint: forward + surrogate-gradient backward of a 131,072-neuron network; "
                         "partition: partition-quality and relay-policy study (JSON report); "
                         "partition-device: Algorithm 1 on the GPU vs the host greedy (JSON report)")
    ap.add_argument("--delivery", choices=tuple(DELIVERY), default="auto",
                    help="ring: every delay at the spike step into the delay ring; arrival: each step "
                         "writes only the next step's input slot (delayed runs queued by arrival step); "
                         "auto: the autotuner picks")
    ap.add_argument("--study-neurons", type=int, default=65536)
    ap.add_argument("--no-scale", action="store_true",
                    help="--config partition-device: the study network only")
    ap.add_argument("--host-scale-iters", type=int, default=1,
                    help="host greedy iterations on the scale workload (--config partition-device; 0: skip)")
    ap.add_argument("--batch-nets", type=int, default=64)
    ap.add_argument("--separate-steps", type=int, default=1000,
                    help="steps per network of the one-sim-per-network comparison (--config batch)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "batch":
        run_batch(args)
    elif args.config == "adjoint":
        run_adjoint(args)
    elif args.config == "partition":
        run_partition_study(args)
    elif args.config == "partition-device":
        run_partition_device(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
