"""CPU oracle — TEST INFRASTRUCTURE ONLY.

A plain sequential simulator (oracle.c) of the partitioned LIF step with
explicit per-partition message queues and the direct all-to-all route, plus
the partitioning (Algorithm 1) and grouping (Algorithm 2) readings as naive
greedy loops.  Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline
leg of `bench.py` may import this package.  It shares no code with the GPU
library (`paper_2205_07125_gb300`), and neither imports the other; the only
code both sides see is the seeded input generator in `synth/`.

Every function here is pinned by tests against closed forms, brute force on
tiny inputs, library routines or published test vectors (tests/test_oracle_*).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

# counter indices (oracle.c enum)
COUNT_NAMES = ("steps", "spikes", "events", "direct", "direct_xvn", "l1_local", "l1_xvn",
               "l2_local", "l2_peer", "l2_relay_local", "l2_relay_remote")


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/liboracle.so (gcc, single thread, no FMA)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared",
                               "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class OrDyn(ctypes.Structure):
    _fields_ = [("dt_ms", ctypes.c_double), ("tau_ms", ctypes.c_double),
                ("e_l", ctypes.c_float), ("v_th", ctypes.c_float), ("v_reset", ctypes.c_float),
                ("t_ref", ctypes.c_int32), ("drive_lambda", ctypes.c_double),
                ("w_ext", ctypes.c_int32), ("i_bias", ctypes.c_int32),
                ("drive_seed", ctypes.c_uint64)]


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_SO)
    vp, i64, i32, u64, dbl = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                              ctypes.c_double)
    L.or_philox4x32_10.argtypes = [vp, vp, vp]
    L.or_philox4x32_10.restype = None
    L.or_poisson_table.argtypes = [dbl, vp, vp]
    L.or_poisson_table.restype = ctypes.c_int
    L.or_mix64.argtypes = [u64]
    L.or_mix64.restype = u64
    L.or_partition_planted.argtypes = [i64, i32, vp]
    L.or_partition_planted.restype = ctypes.c_int
    L.or_cut.argtypes = [i64, vp, vp, vp]
    L.or_cut.restype = i64
    L.or_partition_greedy.argtypes = [i64, vp, vp, i32, i32, u64, vp, vp]
    L.or_partition_greedy.restype = ctypes.c_int
    L.or_partition_greedy_batched.argtypes = [i64, vp, vp, i32, i32, u64, i32, i32, vp, vp]
    L.or_partition_greedy_batched.restype = ctypes.c_int
    L.or_group_greedy.argtypes = [i64, vp, vp, vp, i32, i32, i32, u64, vp, vp]
    L.or_group_greedy.restype = ctypes.c_int
    L.or_create.argtypes = [i64, vp, vp, vp, vp, i32, vp, i32, vp, ctypes.POINTER(OrDyn)]
    L.or_create.restype = vp
    L.or_set_relay_policy.argtypes = [vp, i32, vp]
    L.or_set_relay_policy.restype = ctypes.c_int
    L.or_destroy.argtypes = [vp]
    L.or_destroy.restype = None
    L.or_run.argtypes = [vp, i64, i32, i32, vp, vp, vp, vp, vp, i64, vp, vp, vp, i32, vp, vp,
                         vp, vp, vp, i64, vp]
    L.or_run.restype = ctypes.c_int
    L.or_num_segments.argtypes = [vp]
    L.or_num_segments.restype = i64
    L.or_drive_draws.argtypes = [u64, dbl, i64, i64, i64, vp]
    L.or_drive_draws.restype = ctypes.c_int
    L.or_alpha.argtypes = [dbl, dbl]
    L.or_alpha.restype = ctypes.c_float
    _lib = L
    return L


def _p(a):
    return None if a is None else a.ctypes.data


# ---------------------------------------------------------------- primitives
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of a 4-word counter and a 2-word key (Salmon et al., SC'11)."""
    L = _load()
    c = np.asarray(ctr, np.uint32).copy()
    k = np.asarray(key, np.uint32).copy()
    out = np.zeros(4, np.uint32)
    L.or_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def poisson_table(lam: float) -> np.ndarray:
    """Inverse-CDF thresholds floor(2^32 * P(X <= k)) for X ~ Poisson(lam)."""
    L = _load()
    th = np.zeros(32, np.uint64)
    n = ctypes.c_int32(0)
    if L.or_poisson_table(float(lam), th.ctypes.data, ctypes.byref(n)) != 0:
        raise ValueError("lambda out of range")
    return th[: n.value].copy()


def drive_draws(seed: int, lam: float, j0: int, n: int, t: int) -> np.ndarray:
    """Poisson drive arrivals of neurons j0..j0+n-1 at step t."""
    out = np.zeros(n, np.int32)
    if _load().or_drive_draws(seed, float(lam), j0, n, t, out.ctypes.data) != 0:
        raise ValueError("lambda out of range")
    return out


def mix64(z: int) -> int:
    return int(_load().or_mix64(ctypes.c_uint64(z & 0xFFFFFFFFFFFFFFFF)))


def alpha32(dt_ms: float, tau_ms: float) -> np.float32:
    return np.float32(_load().or_alpha(dt_ms, tau_ms))


def dyn_struct(dyn) -> OrDyn:
    return OrDyn(dt_ms=dyn.dt_ms, tau_ms=dyn.tau_ms, e_l=dyn.e_l, v_th=dyn.v_th,
                 v_reset=dyn.v_reset, t_ref=dyn.t_ref, drive_lambda=dyn.drive_lambda,
                 w_ext=dyn.w_ext, i_bias=dyn.i_bias, drive_seed=dyn.drive_seed)


# ---------------------------------------------------------------- partitions
def partition_planted(M: int, P: int) -> np.ndarray:
    out = np.empty(M, np.int32)
    if _load().or_partition_planted(M, P, out.ctypes.data) != 0:
        raise ValueError("bad planted partition arguments")
    return out


def cut(net, part_of: np.ndarray) -> int:
    po = np.ascontiguousarray(part_of, np.int32)
    return int(_load().or_cut(net.M, net.syn_ptr.ctypes.data, net.tgt.ctypes.data, po.ctypes.data))


def partition_greedy(net, P: int, iters: int = 4, seed: int = 7):
    """Algorithm 1 reading (naive greedy).  Returns (part_of, objective)."""
    out = np.empty(net.M, np.int32)
    best = ctypes.c_int64(0)
    rc = _load().or_partition_greedy(net.M, net.syn_ptr.ctypes.data, net.tgt.ctypes.data, P, iters,
                                     seed, out.ctypes.data, ctypes.byref(best))
    if rc != 0:
        raise ValueError("or_partition_greedy failed: %d" % rc)
    return out, int(best.value)


def partition_greedy_batched(net, P: int, batch: int, grow: int = 0, iters: int = 4, seed: int = 7):
    """Algorithm 1 with batched growth: rounds of min(batch, max(1, n_k //
    grow)) best-gain neurons (grow = 0: batch), ranked by the round's gains,
    n_k the part's size so far.  batch = 1 is partition_greedy.
    Returns (part_of, objective)."""
    out = np.empty(net.M, np.int32)
    best = ctypes.c_int64(0)
    rc = _load().or_partition_greedy_batched(net.M, net.syn_ptr.ctypes.data, net.tgt.ctypes.data, P,
                                             iters, seed, batch, grow, out.ctypes.data, ctypes.byref(best))
    if rc != 0:
        raise ValueError("or_partition_greedy_batched failed: %d" % rc)
    return out, int(best.value)


def group_contiguous(P: int, n_vn: int) -> np.ndarray:
    return (np.arange(P, dtype=np.int32) // (P // n_vn)).astype(np.int32)


def group_greedy(net, part_of, P: int, n_vn: int, iters: int = 4, seed: int = 7):
    """Algorithm 2 reading (naive greedy grouping).  Returns (vn_of_part, cost)."""
    po = np.ascontiguousarray(part_of, np.int32)
    out = np.empty(P, np.int32)
    cost = np.zeros(2, np.uint64)
    rc = _load().or_group_greedy(net.M, net.syn_ptr.ctypes.data, net.tgt.ctypes.data,
                                 po.ctypes.data, P, n_vn, iters, seed, out.ctypes.data,
                                 cost.ctypes.data)
    if rc != 0:
        raise ValueError("or_group_greedy failed: %d" % rc)
    return out, int(cost[0]) + (int(cost[1]) << 64)


# ---------------------------------------------------------------- model file
class ModelFile:
    """A network read from an edge-list file (the library's snn_model_save
    format), with this package's own reader: 8 magic bytes "SNNMODL1", then
    little-endian u64 M, u64 E, u32 max_delay, u32 0, then syn_ptr i64[M+1],
    tgt u32[E], w i16[E], d u8[E], v0 f32[M], is_exc u8[M]."""

    MAGIC = b"SNNMODL1"

    def __init__(self, path: str):
        with open(path, "rb") as f:
            head = f.read(32)
            if len(head) != 32 or head[:8] != self.MAGIC:
                raise ValueError("not a model file: %s" % path)
            M, E = (int(x) for x in np.frombuffer(head[8:24], "<u8"))
            self.max_delay = int(np.frombuffer(head[24:28], "<u4")[0])

            def take(dtype, n):
                a = np.fromfile(f, dtype=dtype, count=n)
                if a.shape[0] != n:
                    raise ValueError("truncated model file: %s" % path)
                return a

            self.syn_ptr = take("<i8", M + 1)
            self.tgt = take("<u4", E)
            self.w = take("<i2", E)
            self.d = take("u1", E)
            self.v0 = take("<f4", M)
            self.is_exc = take("u1", M)
        self.M, self.E = M, E


def load_model(path: str) -> ModelFile:
    return ModelFile(path)


# ---------------------------------------------------------------- simulator
class Oracle:
    """Sequential simulator over a network (borrowed arrays) and a mapping.

    State: V (float32 [M]), ref (uint8 [M]), ring (int32 [D, M]) with
    D = max delay, FP64 shadow v64 (float64 [M]), and the global step t.
    """

    RELAY = {"per_vn": 0, "per_partition": 1, "balanced": 2}

    def __init__(self, net, P, part_of, n_vn, vn_of_part, dyn, relay: str = "per_vn"):
        self._L = _load()
        self.net = net
        self.M = net.M
        self.P, self.n_vn = int(P), int(n_vn)
        self.part_of = np.ascontiguousarray(part_of, np.int32)
        self.vn_of_part = np.ascontiguousarray(vn_of_part, np.int32)
        self.dyn = dyn
        self._dyn = dyn_struct(dyn)
        self.D = max(1, int(net.d.max()) if net.E else 1)
        self._h = self._L.or_create(net.M, net.syn_ptr.ctypes.data, net.tgt.ctypes.data,
                                    net.w.ctypes.data, net.d.ctypes.data, self.P,
                                    self.part_of.ctypes.data, self.n_vn,
                                    self.vn_of_part.ctypes.data, ctypes.byref(self._dyn))
        if not self._h:
            raise ValueError("or_create rejected the network")
        self.relay = np.zeros((self.n_vn, self.P), np.int32)
        if self._L.or_set_relay_policy(self._h, self.RELAY[relay], self.relay.ctypes.data) != 0:
            raise ValueError("unknown relay policy %r" % relay)
        self.V = net.v0.astype(np.float32).copy()
        self.ref = np.zeros(self.M, np.uint8)
        self.ring = np.zeros((self.D, self.M), np.int32)
        self.v64 = net.v0.astype(np.float64)
        self.t = 0
        self.counts = np.zeros(len(COUNT_NAMES), np.uint64)
        self.fp64 = np.zeros(3, np.float64)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.or_destroy(h)
            self._h = None

    @property
    def n_segments(self) -> int:
        return int(self._L.or_num_segments(self._h))

    def run(self, T: int, raster: bool = True, hashes: bool = True, rec_steps=(),
            pairs: bool = False, raster_cap: int | None = None) -> dict:
        M = self.M
        out = {}
        cap = raster_cap if raster_cap is not None else max(1024, M * T // 20)
        ids = np.zeros(cap, np.uint32) if raster else None
        off = np.zeros(T + 1, np.int64) if raster else None
        ch = np.zeros(T, np.uint64) if hashes else None
        vh = np.zeros(T, np.uint64) if hashes else None
        rs = np.asarray(list(rec_steps), np.int64)
        rc_buf = np.zeros((len(rs), M), np.int32)
        pr = np.zeros(max(1, M * self.P), np.uint64) if pairs else None
        npairs = ctypes.c_int64(0)
        rc = self._L.or_run(self._h, self.t, T, self.D, self.V.ctypes.data, self.ref.ctypes.data,
                            self.ring.ctypes.data, self.v64.ctypes.data, _p(ids), cap, _p(off),
                            _p(ch), _p(vh), len(rs), rs.ctypes.data if len(rs) else None,
                            rc_buf.ctypes.data if len(rs) else None, self.counts.ctypes.data,
                            self.fp64.ctypes.data, _p(pr), len(pr) if pairs else 0,
                            ctypes.byref(npairs))
        if rc == -3:
            raise MemoryError("oracle raster capacity exceeded; pass a larger raster_cap")
        if rc != 0:
            raise ValueError("or_run failed: %d" % rc)
        self.t += T
        if raster:
            out["raster_ids"] = ids[: off[-1]].copy()
            out["raster_off"] = off
        if hashes:
            out["cur_hash"], out["v_hash"] = ch, vh
        if len(rs):
            out["currents"] = {int(s): rc_buf[k] for k, s in enumerate(rs)}
        if pairs:
            out["pairs"] = np.sort(pr[: npairs.value])
        return out

    def count_dict(self) -> dict:
        return {k: int(v) for k, v in zip(COUNT_NAMES, self.counts)}

    def fp64_stats(self) -> dict:
        return {"max_rel_err": float(self.fp64[0]), "n_compared": int(self.fp64[1]),
                "n_disagree": int(self.fp64[2])}
