"""Seeded synthetic inputs: network configurations and the network generator.

This package is the only code that both the CPU oracle and the GPU library
tests share.  It makes the *inputs* of a simulation (synapse list, initial
membrane potentials, the planted partition/virtual-node structure and the
scalar parameters of a workload) and holds none of the simulation's own
arithmetic.

The paper (arXiv 2205.07125) simulates a human-brain network built from
medical scans that is not available; the configurations below stand in for
it with random LIF networks whose partition sizes and locality follow the
paper's setting (Sec. V: 10 billion neurons on 2,000 GPUs, i.e. 5 million
neurons per GPU).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_SRC = os.path.join(_HERE, "synth.c")


def build(force: bool = False) -> str:
    """Compile the generator into synth/libsynth.so (gcc, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i64, i32, u64, dbl, vp = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                  ctypes.c_double, ctypes.c_void_p)
        lib.synth_fill.restype = ctypes.c_int
        lib.synth_fill.argtypes = [i64, i32, i32, i32, i32, i32, i32, i32, i32, u64,
                                   dbl, dbl, dbl, dbl, dbl, dbl, dbl,
                                   vp, vp, vp, vp, vp, vp]
        _lib = lib
    return _lib


@dataclasses.dataclass(frozen=True)
class Dynamics:
    """LIF and drive parameters of a workload.

    dt=0.1 ms, tau_m=20 ms, V_th=-50 mV, V_reset=-65 mV, refractory 2 ms
    (20 steps); the resting potential E_L is taken equal to V_reset because
    the workload leaves it open.  Synaptic and drive weights are int16/int32
    fixed point in units of 2^-10 mV.  The Poisson external drive has mean
    `drive_lambda` = nu_ext*dt arrivals per step, each adding `w_ext` units.
    """
    dt_ms: float = 0.1
    tau_ms: float = 20.0
    e_l: float = -65.0
    v_th: float = -50.0
    v_reset: float = -65.0
    t_ref: int = 20
    drive_lambda: float = 0.8
    w_ext: int = 96
    i_bias: int = 0
    drive_seed: int = 2000


@dataclasses.dataclass(frozen=True)
class NetConfig:
    """A synthetic network: sizes, planted structure and generator seed."""
    name: str
    M: int
    P: int                 # planted partitions
    n_vn: int              # planted virtual nodes (P % n_vn == 0)
    K: int                 # out-synapses per neuron
    uniform_all: bool      # targets uniform over all neurons (ignore locality mix)
    n_part: int = 0        # same-partition targets per neuron
    n_vn_t: int = 0        # other partitions of the same VN
    n_remote: int = 0      # partitions of other VNs
    dmax: int = 1
    seed: int = 1000
    steps: int = 1000
    dyn: Dynamics = Dynamics()
    frac_exc: float = 0.8
    mu_e: float = 40.0
    sd_e: float = 8.0
    mu_i: float = 160.0
    sd_i: float = 32.0

    @property
    def vn_size(self) -> int:
        return self.P // self.n_vn

    @property
    def n_synapses(self) -> int:
        return self.M * self.K

    def scaled(self, **kw) -> "NetConfig":
        return dataclasses.replace(self, **kw)


# Tiny plain step: 4,096 neurons, 4 partitions over 2 VNs, 100 uniform
# out-synapses, delay 1, Poisson drive 8 kHz (0.8 arrivals per 0.1 ms step).
TINY = NetConfig(name="tiny-4096n-4p-2vn-k100", M=4096, P=4, n_vn=2, K=100,
                 uniform_all=True, dmax=1, seed=1000, steps=1000,
                 dyn=Dynamics(drive_lambda=0.8, w_ext=96, drive_seed=2000))

# Plain step at scale: 1,048,576 neurons, 64 partitions over 16 VNs of 4,
# 1,000 out-synapses (700 same partition / 200 same VN / 100 remote),
# delays 1..8 steps; drive weight tuned once (oracle runs of 2,000 steps on
# 2^16- and 2^18-neuron networks of the same statistics) for a steady rate
# near 10 Hz.
SCALE = NetConfig(name="scale-1048576n-64p-16vn-k1000", M=1 << 20, P=64, n_vn=16, K=1000,
                  uniform_all=False, n_part=700, n_vn_t=200, n_remote=100, dmax=8,
                  seed=1001, steps=1000,
                  dyn=Dynamics(drive_lambda=0.8, w_ext=89, drive_seed=2001))

# The paper's per-GPU share (10 billion neurons / 2,000 GPUs): 5,000,000
# neurons in 256 partitions over 64 VNs of 4, the same locality mix.
PAPER_SHARE = NetConfig(name="share-5000000n-256p-64vn-k1000", M=5_000_000, P=256, n_vn=64,
                        K=1000, uniform_all=False, n_part=700, n_vn_t=200, n_remote=100,
                        dmax=8, seed=1002, steps=500,
                        dyn=Dynamics(drive_lambda=0.8, w_ext=89, drive_seed=2002))

CONFIGS = {c.name: c for c in (TINY, SCALE, PAPER_SHARE)}


@dataclasses.dataclass
class Network:
    """Source-major synapse list (row i = synapses syn_ptr[i]..syn_ptr[i+1])."""
    cfg: NetConfig
    syn_ptr: np.ndarray    # int64 [M+1]
    tgt: np.ndarray        # uint32 [E] global target ids
    w: np.ndarray          # int16 [E] weights, 2^-10 mV units
    d: np.ndarray          # uint8 [E] delays in steps (>= 1)
    v0: np.ndarray         # float32 [M]
    is_exc: np.ndarray     # uint8 [M]

    @property
    def M(self) -> int:
        return int(self.v0.shape[0])

    @property
    def E(self) -> int:
        return int(self.tgt.shape[0])


def planted_starts(M: int, P: int) -> np.ndarray:
    """Planted partition boundaries start(p) = floor(p*M/P), p = 0..P."""
    p = np.arange(P + 1, dtype=np.int64)
    return (p * M) // P


def make_network(cfg: NetConfig) -> Network:
    """Generate the network of `cfg` (deterministic in cfg.seed)."""
    lib = _load()
    M, K = cfg.M, cfg.K
    E = M * K
    syn_ptr = np.empty(M + 1, np.int64)
    tgt = np.empty(E, np.uint32)
    w = np.empty(E, np.int16)
    d = np.empty(E, np.uint8)
    v0 = np.empty(M, np.float32)
    is_exc = np.empty(M, np.uint8)
    rc = lib.synth_fill(M, cfg.P, cfg.vn_size, K, int(cfg.uniform_all), cfg.n_part, cfg.n_vn_t,
                        cfg.n_remote, cfg.dmax, cfg.seed, cfg.dyn.v_reset, cfg.dyn.v_th,
                        cfg.frac_exc, cfg.mu_e, cfg.sd_e, cfg.mu_i, cfg.sd_i,
                        syn_ptr.ctypes.data, tgt.ctypes.data, w.ctypes.data, d.ctypes.data,
                        v0.ctypes.data, is_exc.ctypes.data)
    if rc != 0:
        raise ValueError("synth_fill rejected config %s" % (cfg,))
    return Network(cfg, syn_ptr, tgt, w, d, v0, is_exc)


def make_edges(M: int, edges, v0=None) -> Network:
    """Hand-built network from an explicit edge list [(src, tgt, w, d), ...]."""
    edges = sorted(edges, key=lambda e: e[0])
    src = np.array([e[0] for e in edges], np.int64)
    syn_ptr = np.zeros(M + 1, np.int64)
    np.add.at(syn_ptr, src + 1, 1)
    syn_ptr = np.cumsum(syn_ptr).astype(np.int64)
    tgt = np.array([e[1] for e in edges], np.uint32)
    w = np.array([e[2] for e in edges], np.int16)
    d = np.array([e[3] for e in edges], np.uint8)
    if v0 is None:
        v0 = np.full(M, -65.0, np.float32)
    cfg = NetConfig(name="edges-%d" % M, M=M, P=1, n_vn=1, K=0, uniform_all=True,
                    dmax=int(d.max()) if len(d) else 1)
    return Network(cfg, syn_ptr, tgt, w, d, np.asarray(v0, np.float32),
                   np.ones(M, np.uint8))


# ---------------------------------------------------------------- batches
@dataclasses.dataclass
class Batch:
    """Independent networks concatenated into one: network k owns ids
    off[k]..off[k+1]-1 and partitions poff[k]..poff[k+1]-1 (planted, VNs of
    `vn_size` partitions inside each network); `net` is the concatenation."""
    cfgs: list
    nets: list
    off: np.ndarray       # [n+1] first id of each network (multiples of 4)
    poff: np.ndarray      # [n+1] first partition label of each network
    net: Network          # the concatenation
    part: np.ndarray      # [M] partition labels of the concatenation
    vn_size: int

    @property
    def P(self) -> int:
        return int(self.poff[-1])

    @property
    def n_vn(self) -> int:
        return self.P // self.vn_size


def batch_configs(n: int = 64, seed: int = 3000, m_lo: int = 10_000, m_hi: int = 500_000,
                  k_lo: int = 100, k_hi: int = 1000, p_lo: int = 4, p_hi: int = 32, vn_size: int = 2,
                  rate_lo: float = 5.0, rate_hi: float = 15.0, w_ext: int = 89) -> list:
    """Configurations of a batch of independent networks: sizes log-uniform
    in [m_lo, m_hi] (multiples of 4), out-degrees uniform in [k_lo, k_hi]
    with the scale workload's locality mix (70 % same partition, 20 % same
    VN, 10 % remote), partitions uniform in [p_lo, p_hi] (multiples of the VN
    size, at least two VNs), delays 1..8, generator seed seed + k.  Network k
    gets a rate r_k uniform in [rate_lo, rate_hi] Hz and drives its neurons
    with r_k / 10 times the scale workload's Poisson drive (0.8 arrivals per
    step): the drive is scaled, the resulting firing rates are measured."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        M = int(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi)))) // 4 * 4
        K = int(rng.integers(k_lo, k_hi + 1))
        P = int(rng.integers(max(p_lo, 2 * vn_size) // vn_size, p_hi // vn_size + 1)) * vn_size
        r = float(rng.uniform(rate_lo, rate_hi))
        n_part = int(round(0.7 * K))
        n_vn_t = int(round(0.2 * K))
        dyn = Dynamics(drive_lambda=0.8 * r / 10.0, w_ext=w_ext, drive_seed=seed + 10_000 + k)
        out.append(NetConfig(name="batch%d-%dn-%dp-k%d" % (k, M, P, K), M=M, P=P, n_vn=P // vn_size, K=K,
                             uniform_all=False, n_part=n_part, n_vn_t=n_vn_t, n_remote=K - n_part - n_vn_t,
                             dmax=8, seed=seed + k, steps=1000, dyn=dyn))
    return out


def make_batch(cfgs: list) -> Batch:
    """Generate every network of `cfgs` and their concatenation."""
    nets = [make_network(c) for c in cfgs]
    vs = cfgs[0].vn_size
    assert all(c.vn_size == vs and c.M % 4 == 0 for c in cfgs)
    off = np.zeros(len(cfgs) + 1, np.int64)
    poff = np.zeros(len(cfgs) + 1, np.int64)
    for k, c in enumerate(cfgs):
        off[k + 1] = off[k] + c.M
        poff[k + 1] = poff[k] + c.P
    M = int(off[-1])
    E = sum(g.E for g in nets)
    syn_ptr = np.empty(M + 1, np.int64)
    tgt = np.empty(E, np.uint32)
    w = np.empty(E, np.int16)
    d = np.empty(E, np.uint8)
    v0 = np.empty(M, np.float32)
    is_exc = np.empty(M, np.uint8)
    part = np.empty(M, np.int32)
    e0 = 0
    for k, (c, g) in enumerate(zip(cfgs, nets)):
        a, b = int(off[k]), int(off[k + 1])
        syn_ptr[a:b] = g.syn_ptr[:-1] + e0
        tgt[e0:e0 + g.E] = g.tgt + np.uint32(a)
        w[e0:e0 + g.E] = g.w
        d[e0:e0 + g.E] = g.d
        v0[a:b] = g.v0
        is_exc[a:b] = g.is_exc
        for p in range(c.P):
            part[a + c.M * p // c.P:a + c.M * (p + 1) // c.P] = poff[k] + p
        e0 += g.E
    syn_ptr[M] = e0
    ucfg = NetConfig(name="batch-%dnets-%dn" % (len(cfgs), M), M=M, P=int(poff[-1]),
                     n_vn=int(poff[-1]) // vs, K=0, uniform_all=False, dmax=max(c.dmax for c in cfgs))
    return Batch(cfgs, nets, off, poff, Network(ucfg, syn_ptr, tgt, w, d, v0, is_exc), part, vs)
