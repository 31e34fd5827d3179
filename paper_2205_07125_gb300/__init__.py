"""Python binding of libsnn.so, the GB300 partitioned spiking-network step.

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of the library (csrc/snn_sim.cu); the host code of the library
(csrc/snn_host.cpp) builds the partition and the two-level routing tables.
PyTorch is used for device memory (the caller-owned workspace) and streams.

The names follow the C ABI in include/snn.h:
    snn_partition(net, P, mode)              -> part_of        (Algorithm 1)
    snn_partition_device(net, P, batch, grow) -> part_of       (Algorithm 1, batched growth, GPU)
    Routing(net, part_of, P, n_vn, grouping)                   (Algorithm 2 + tables)
    Routing(..., build="device")                               (the same tables built on the GPU)
    Sim(net, routing, params).step(T)                          (the hot path)
    Sim.read_raster / read_currents / read_counts / read_hashes / read_state
This module raises ImportError when libsnn.so has not been built; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsnn.so")

if not os.path.exists(_SO):
    raise ImportError("libsnn.so is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = ctypes.CDLL(_SO)

SNN_PART_PLANTED, SNN_PART_GREEDY, SNN_PART_RANDOM = 0, 1, 2
SNN_GROUP_CONTIGUOUS, SNN_GROUP_GREEDY = 0, 1
SNN_DELIVER_RING, SNN_DELIVER_ARRIVAL, SNN_DELIVER_AUTO, SNN_DELIVER_OWNER = 0, 1, 2, 3
SNN_RELAY_PER_VN, SNN_RELAY_PER_PARTITION, SNN_RELAY_BALANCED = 0, 1, 2
RELAY_POLICIES = {"per_vn": SNN_RELAY_PER_VN, "per_partition": SNN_RELAY_PER_PARTITION,
                  "balanced": SNN_RELAY_BALANCED}
SNN_E_CAPACITY = -3

_i32, _i64, _u64, _u32, _f32, _f64, _vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                           ctypes.c_uint32, ctypes.c_float, ctypes.c_double,
                                           ctypes.c_void_p)


class snn_network(ctypes.Structure):
    _fields_ = [("n_neurons", _i64), ("syn_ptr", _vp), ("syn_tgt", _vp), ("syn_w", _vp),
                ("syn_d", _vp), ("v0", _vp)]


class snn_model_params(ctypes.Structure):
    _fields_ = [("n_neurons", _i64), ("n_parts", _i32), ("vn_size", _i32), ("syn_per_neuron", _i32),
                ("uniform", _i32), ("n_same_part", _i32), ("n_same_vn", _i32), ("n_remote", _i32),
                ("max_delay", _i32), ("seed", _u64), ("v_reset", _f64), ("v_th", _f64), ("frac_exc", _f64),
                ("mu_e", _f64), ("sd_e", _f64), ("mu_i", _f64), ("sd_i", _f64)]


class snn_partition_params(ctypes.Structure):
    _fields_ = [("mode", _i32), ("iters", _i32), ("seed", _u64)]


class snn_partition_stats(ctypes.Structure):
    _fields_ = [("objective", _i64), ("min_weight", _i64), ("max_weight", _i64)]


class snn_partition_device_params(ctypes.Structure):
    _fields_ = [("iters", _i32), ("batch", _i32), ("grow", _i32), ("reserved", _i32), ("seed", _u64)]


class snn_routing_params(ctypes.Structure):
    _fields_ = [("grouping", _i32), ("iters", _i32), ("seed", _u64), ("n_threads", _i32),
                ("relay", _i32)]


class snn_routing_info(ctypes.Structure):
    _fields_ = [("n_neurons", _i64), ("n_synapses", _i64), ("n_parts", _i32), ("n_vn", _i32),
                ("vn_size", _i32), ("max_delay", _i32), ("n_l1", _i64), ("n_l2", _i64),
                ("group_cost_lo", _u64), ("group_cost_hi", _u64), ("conn_direct_sum", _i64),
                ("conn_two_level_sum", _i64), ("conn_direct_max", _i32),
                ("conn_two_level_max", _i32), ("identity_order", _i32), ("reserved", _i32)]


class snn_sim_params(ctypes.Structure):
    _fields_ = [("dt_ms", _f64), ("tau_ms", _f64), ("e_l", _f32), ("v_th", _f32), ("v_reset", _f32),
                ("t_ref", _i32), ("drive_lambda", _f64), ("w_ext", _i32), ("i_bias", _i32),
                ("drive_seed", _u64), ("raster_cap", _i64), ("raster_steps", _i64),
                ("hash_steps", _i64), ("cur_every", _i32), ("cur_slots", _i32),
                ("bucket_frac", _f32), ("inbox_frac", _f32), ("steps_per_graph", _i32),
                ("pin_host_tables", _i32), ("defer_delayed", _i32), ("delivery", _i32),
                ("arrival_frac", _f32)]


COUNT_FIELDS = ("steps", "spikes", "events", "direct", "direct_xvn", "l1_local", "l1_xvn",
                "l2_local", "l2_peer", "l2_relay_local", "l2_relay_remote")


class snn_adjoint_params(ctypes.Structure):
    _fields_ = [("T", _i32), ("ckpt_every", _i32), ("sigma", _f32), ("beta", _f32), ("reserved", _i64 * 2)]


class snn_counts(ctypes.Structure):
    _fields_ = [(n, _u64) for n in COUNT_FIELDS]


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_P = ctypes.POINTER
_lib_strerror = _sig("snn_strerror", ctypes.c_char_p, [ctypes.c_int])
_sig("snn_model_params_preset", ctypes.c_int, [_i32, _P(snn_model_params)])
_sig("snn_model_build", ctypes.c_int, [_P(snn_model_params), _P(_vp)])
_sig("snn_model_network", ctypes.c_int, [_vp, _P(snn_network), _P(_vp)])
_sig("snn_model_save", ctypes.c_int, [_vp, ctypes.c_char_p])
_sig("snn_model_load", ctypes.c_int, [ctypes.c_char_p, _P(_vp)])
_sig("snn_model_destroy", None, [_vp])
_sig("snn_partition", ctypes.c_int, [_P(snn_network), _i32, _P(snn_partition_params), _vp,
                                     _P(snn_partition_stats)])
_sig("snn_partition_device_params_default", None, [_P(snn_partition_device_params)])
_sig("snn_partition_device_workspace_bytes", ctypes.c_int, [_P(snn_network), _i32, _P(ctypes.c_size_t)])
_sig("snn_partition_device", ctypes.c_int, [_P(snn_network), _i32, _P(snn_partition_device_params), _vp,
                                            ctypes.c_size_t, _vp, _vp, _P(snn_partition_stats)])
_sig("snn_routing_build", ctypes.c_int, [_P(snn_network), _vp, _i32, _i32, _P(snn_routing_params),
                                         _P(_vp)])
_sig("snn_routing_info_get", ctypes.c_int, [_vp, _P(snn_routing_info)])
_sig("snn_routing_export", ctypes.c_int, [_vp, ctypes.c_char_p, _vp, ctypes.c_size_t, _P(ctypes.c_size_t)])
_sig("snn_routing_build_device_workspace_bytes", ctypes.c_int, [_P(snn_network), _i32, _i32, _P(ctypes.c_size_t)])
_sig("snn_routing_build_device", ctypes.c_int, [_P(snn_network), _vp, _i32, _i32, _P(snn_routing_params), _vp,
                                                ctypes.c_size_t, _vp, _P(_vp)])
_sig("snn_routing_groups", ctypes.c_int, [_vp, _vp, _vp])
_sig("snn_routing_connections", ctypes.c_int, [_vp, _vp, _vp])
_sig("snn_routing_traffic", ctypes.c_int, [_vp, _vp, _i64, _i32, _vp, _vp, _vp, _vp])
_sig("snn_routing_relays", ctypes.c_int, [_vp, _i32, _vp])
_sig("snn_routing_destroy", None, [_vp])
_sig("snn_sim_params_default", None, [_P(snn_sim_params)])
_sig("snn_sim_workspace_bytes", ctypes.c_int, [_vp, _P(snn_sim_params), _P(ctypes.c_size_t)])
_sig("snn_sim_create", ctypes.c_int, [_P(snn_network), _vp, _P(snn_sim_params), _vp, ctypes.c_size_t,
                                      _vp, _P(_vp)])
_sig("snn_batch_workspace_bytes", ctypes.c_int, [_vp, _i32, _vp, _P(ctypes.c_size_t)])
_sig("snn_batch_create", ctypes.c_int, [_P(snn_network), _vp, _i32, _vp, _vp, _vp, ctypes.c_size_t, _vp,
                                        _P(_vp)])
_sig("snn_step", ctypes.c_int, [_vp, _i32])
_sig("snn_autotune", ctypes.c_int, [_vp, _i32, _P(_i32), _P(ctypes.c_double)])
_sig("snn_sync_status", ctypes.c_int, [_vp])
_sig("snn_read_raster", ctypes.c_int, [_vp, _i64, _i64, _vp, _i64, _vp, _P(_i64)])
_sig("snn_read_currents", ctypes.c_int, [_vp, _i64, _vp])
_sig("snn_read_hashes", ctypes.c_int, [_vp, _i64, _i64, _vp, _vp])
_sig("snn_read_counts", ctypes.c_int, [_vp, _P(snn_counts)])
_sig("snn_read_state", ctypes.c_int, [_vp, _vp, _vp, _P(_i64)])
_sig("snn_read_inbox_pairs", ctypes.c_int, [_vp, _vp, _i64, _P(_i64)])
_sig("snn_state_bytes", ctypes.c_int, [_vp, _P(ctypes.c_size_t)])
_sig("snn_save_state", ctypes.c_int, [_vp, _vp, ctypes.c_size_t])
_sig("snn_load_state", ctypes.c_int, [_vp, _vp, ctypes.c_size_t])
_sig("snn_sim_reset", ctypes.c_int, [_vp, _i32])
_sig("snn_launches_per_step", _i64, [_vp])
_sig("snn_launches", _i64, [_vp, _i32])
_sig("snn_profile_phases", ctypes.c_int, [_vp, _i32, _vp])
_sig("snn_deliver_spikes", ctypes.c_int, [_vp, _vp, _i64, _vp, _vp])
_sig("snn_deliver_spikes_static", ctypes.c_int, [_vp, _vp, _i64, _vp, _vp])
_sig("snn_static_scratch_bytes", ctypes.c_size_t, [])
_sig("snn_sim_destroy", None, [_vp])
_sig("snn_adjoint_params_default", None, [_P(snn_adjoint_params)])
_sig("snn_adjoint_workspace_bytes", ctypes.c_int, [_vp, _P(snn_sim_params), _P(snn_adjoint_params),
                                                   _P(ctypes.c_size_t)])
_sig("snn_adjoint_create", ctypes.c_int, [_P(snn_network), _vp, _vp, _P(snn_sim_params), _P(snn_adjoint_params),
                                          _vp, ctypes.c_size_t, _vp, _P(_vp)])
_sig("snn_adjoint_forward", ctypes.c_int, [_vp, _vp, _vp, _vp, _P(_i64)])
_sig("snn_adjoint_backward", ctypes.c_int, [_vp, _vp, _vp, _vp])
_sig("snn_adjoint_read_spikes", ctypes.c_int, [_vp, _vp, _i64, _P(_i64)])
_sig("snn_adjoint_destroy", None, [_vp])

EXPORTS = ("snn_strerror", "snn_model_params_preset", "snn_model_build", "snn_model_network", "snn_model_save",
           "snn_model_load", "snn_model_destroy", "snn_partition", "snn_partition_device_params_default",
           "snn_partition_device_workspace_bytes", "snn_partition_device", "snn_routing_build",
           "snn_routing_export", "snn_routing_build_device_workspace_bytes", "snn_routing_build_device", "snn_routing_info_get",
           "snn_routing_groups", "snn_routing_connections", "snn_routing_traffic", "snn_routing_relays",
           "snn_routing_destroy",
           "snn_sim_params_default", "snn_sim_workspace_bytes", "snn_sim_create", "snn_step",
           "snn_sync_status", "snn_read_raster", "snn_read_currents", "snn_read_hashes",
           "snn_read_counts", "snn_read_state", "snn_read_inbox_pairs", "snn_state_bytes",
           "snn_save_state", "snn_load_state", "snn_sim_reset", "snn_launches_per_step", "snn_launches",
           "snn_profile_phases", "snn_deliver_spikes", "snn_deliver_spikes_static",
           "snn_static_scratch_bytes", "snn_sim_destroy", "snn_batch_workspace_bytes", "snn_batch_create",
           "snn_autotune", "snn_adjoint_params_default", "snn_adjoint_workspace_bytes", "snn_adjoint_create",
           "snn_adjoint_forward", "snn_adjoint_backward", "snn_adjoint_read_spikes", "snn_adjoint_destroy")


class SnnError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, _lib_strerror(code).decode(), code))


def _ck(rc: int, what: str):
    if rc != 0:
        raise SnnError(rc, what)


def library_path() -> str:
    return _SO


class Network:
    """Borrowed view of a source-major synapse list (numpy arrays kept alive here)."""

    def __init__(self, syn_ptr, tgt, w, d, v0):
        self.syn_ptr = np.ascontiguousarray(syn_ptr, np.int64)
        self.tgt = np.ascontiguousarray(tgt, np.uint32)
        self.w = np.ascontiguousarray(w, np.int16)
        self.d = np.ascontiguousarray(d, np.uint8)
        self.v0 = np.ascontiguousarray(v0, np.float32)
        self.M = int(self.v0.shape[0])
        if self.syn_ptr.shape[0] != self.M + 1:
            raise ValueError("syn_ptr must have M+1 entries")
        self.s = snn_network(self.M, self.syn_ptr.ctypes.data, self.tgt.ctypes.data,
                             self.w.ctypes.data, self.d.ctypes.data, self.v0.ctypes.data)

    @classmethod
    def from_synth(cls, net):
        return cls(net.syn_ptr, net.tgt, net.w, net.d, net.v0)


SNN_WORKLOAD_TINY, SNN_WORKLOAD_SCALE, SNN_WORKLOAD_PAPER_SHARE, SNN_WORKLOAD_ADJOINT = 0, 1, 2, 4
_WORKLOADS = {"tiny": SNN_WORKLOAD_TINY, "scale": SNN_WORKLOAD_SCALE, "paper": SNN_WORKLOAD_PAPER_SHARE,
              "adjoint": SNN_WORKLOAD_ADJOINT}


def model_params(workload=None, **kw) -> snn_model_params:
    """snn_model_params of a workload preset ("tiny", "scale", "paper",
    "adjoint" or an SNN_WORKLOAD_* code) with keyword overrides."""
    p = snn_model_params()
    code = _WORKLOADS.get(workload, workload) if workload is not None else SNN_WORKLOAD_TINY
    _ck(_lib.snn_model_params_preset(int(code), ctypes.byref(p)), "snn_model_params_preset")
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Model:
    """A network owned by the library (snn_model_build / snn_model_load); its
    arrays are exposed as numpy views, valid while the model lives."""

    def __init__(self, h):
        self.h = h
        net = snn_network()
        exc = _vp()
        _ck(_lib.snn_model_network(h, ctypes.byref(net), ctypes.byref(exc)), "snn_model_network")
        M = int(net.n_neurons)
        P = ctypes.POINTER

        def view(ptr, ctype, n):
            return np.ctypeslib.as_array(ctypes.cast(ptr, P(ctype)), shape=(n,)) if n else np.zeros(0)

        self.M = M
        self.syn_ptr = view(net.syn_ptr, ctypes.c_int64, M + 1)
        self.E = int(self.syn_ptr[M])
        self.tgt = view(net.syn_tgt, ctypes.c_uint32, self.E)
        self.w = view(net.syn_w, ctypes.c_int16, self.E)
        self.d = view(net.syn_d, ctypes.c_uint8, self.E)
        self.v0 = view(net.v0, ctypes.c_float, M)
        self.is_exc = view(exc, ctypes.c_uint8, M)

    @classmethod
    def build(cls, params: snn_model_params = None, **kw) -> "Model":
        p = params if params is not None else model_params(**kw)
        h = _vp()
        _ck(_lib.snn_model_build(ctypes.byref(p), ctypes.byref(h)), "snn_model_build")
        return cls(h.value)

    @classmethod
    def load(cls, path: str) -> "Model":
        h = _vp()
        _ck(_lib.snn_model_load(os.fsencode(path), ctypes.byref(h)), "snn_model_load")
        return cls(h.value)

    def save(self, path: str):
        _ck(_lib.snn_model_save(self.h, os.fsencode(path)), "snn_model_save")

    def network(self) -> "Network":
        """Network view of the model's arrays (no copy; keeps the model alive)."""
        net = Network(self.syn_ptr, self.tgt, self.w, self.d, self.v0)
        net._model = self
        return net

    def close(self):
        if getattr(self, "h", None):
            _lib.snn_model_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


_PART_MODES = {"planted": SNN_PART_PLANTED, "greedy": SNN_PART_GREEDY, "random": SNN_PART_RANDOM}


def snn_partition(net: Network, n_parts: int, mode: str = "planted", iters: int = 4, seed: int = 7):
    """Algorithm 1 (or a baseline mapping).  Returns (part_of int32[M], stats dict)."""
    out = np.empty(net.M, np.int32)
    prm = snn_partition_params(_PART_MODES[mode], iters, seed)
    st = snn_partition_stats()
    _ck(_lib.snn_partition(ctypes.byref(net.s), n_parts, ctypes.byref(prm), out.ctypes.data,
                           ctypes.byref(st)), "snn_partition")
    return out, {"objective": st.objective, "min_weight": st.min_weight,
                 "max_weight": st.max_weight}


def snn_partition_device(net: Network, n_parts: int, batch: int = 2048, grow: int = 2, iters: int = 4,
                         seed: int = 7, device=None, stream=None):
    """Algorithm 1 with batched growth on the GPU (batch = 1: the sequential
    greedy of snn_partition).  The workspace is a torch tensor on `device`;
    the call returns when the labels are on the host.
    Returns (part_of int32[M], stats dict)."""
    import torch
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    prm = snn_partition_device_params()
    _lib.snn_partition_device_params_default(ctypes.byref(prm))
    prm.iters, prm.batch, prm.grow, prm.seed = iters, batch, grow, seed
    nb = ctypes.c_size_t(0)
    _ck(_lib.snn_partition_device_workspace_bytes(ctypes.byref(net.s), n_parts, ctypes.byref(nb)),
        "snn_partition_device_workspace_bytes")
    out = np.empty(net.M, np.int32)
    st = snn_partition_stats()
    with torch.cuda.device(dev):
        ws = torch.empty(max(256, nb.value), dtype=torch.uint8, device=dev)
        strm = stream if stream is not None else torch.cuda.current_stream(dev)
        _ck(_lib.snn_partition_device(ctypes.byref(net.s), n_parts, ctypes.byref(prm), ws.data_ptr(), nb.value,
                                      strm.cuda_stream, out.ctypes.data, ctypes.byref(st)),
            "snn_partition_device")
        del ws
    return out, {"objective": st.objective, "min_weight": st.min_weight,
                 "max_weight": st.max_weight}


_TABLE_TYPES = {"syn_td": np.uint32, "syn_w": np.int16, "csr": np.int64, "l1_ptr": np.uint32, "l1_vn": np.uint16,
                "l1_l2": np.uint32, "l2": np.uint8, "l1_pair": np.uint32, "l2_pair": np.uint32,
                "bpair_ptr": np.uint32, "bpair_dst": np.uint16, "bpair_cap": np.uint32, "ipair_ptr": np.uint32,
                "ipair_dst": np.uint16, "ipair_cap": np.uint32, "bucket_cap": np.uint64, "inbox_cap": np.uint64,
                "perm_inv": np.uint32, "perm_fwd": np.uint32, "src_part": np.uint16, "pbase": np.int64,
                "v0": np.float32, "vn_of_part": np.int32, "relay": np.int32}


class Routing:
    """Algorithm 2 grouping and the two-level routing tables (host memory).
    build="device" builds the same tables on the GPU (snn_routing_build_device;
    the workspace is a torch tensor on `device`)."""

    def __init__(self, net: Network, part_of, n_parts: int, n_vn: int, grouping: str = "contiguous",
                 iters: int = 4, seed: int = 7, n_threads: int = 0, build: str = "host", device=None,
                 relay: str = "per_vn"):
        self.net = net
        self.part_of = np.ascontiguousarray(part_of, np.int32)
        g = {"contiguous": SNN_GROUP_CONTIGUOUS, "greedy": SNN_GROUP_GREEDY}[grouping]
        prm = snn_routing_params(g, iters, seed, n_threads, RELAY_POLICIES[relay])
        h = _vp()
        if build == "host":
            _ck(_lib.snn_routing_build(ctypes.byref(net.s), self.part_of.ctypes.data, n_parts, n_vn,
                                       ctypes.byref(prm), ctypes.byref(h)), "snn_routing_build")
        elif build == "device":
            import torch
            dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
            nb = ctypes.c_size_t(0)
            _ck(_lib.snn_routing_build_device_workspace_bytes(ctypes.byref(net.s), n_parts, n_vn, ctypes.byref(nb)),
                "snn_routing_build_device_workspace_bytes")
            with torch.cuda.device(dev):
                ws = torch.empty(max(256, nb.value), dtype=torch.uint8, device=dev)
                strm = torch.cuda.current_stream(dev)
                _ck(_lib.snn_routing_build_device(ctypes.byref(net.s), self.part_of.ctypes.data, n_parts, n_vn,
                                                  ctypes.byref(prm), ws.data_ptr(), nb.value, strm.cuda_stream,
                                                  ctypes.byref(h)), "snn_routing_build_device")
                del ws
        else:
            raise ValueError("build must be 'host' or 'device'")
        self.h = h.value
        self.P, self.n_vn = n_parts, n_vn

    def export(self, name: str) -> np.ndarray:
        """A copy of one routing table (snn_routing_export), as a numpy array."""
        nb = ctypes.c_size_t(0)
        _ck(_lib.snn_routing_export(self.h, name.encode(), None, 0, ctypes.byref(nb)), "snn_routing_export")
        out = np.empty(nb.value, np.uint8)
        _ck(_lib.snn_routing_export(self.h, name.encode(), out.ctypes.data, nb.value, ctypes.byref(nb)),
            "snn_routing_export")
        return out.view(_TABLE_TYPES[name])

    def info(self) -> dict:
        i = snn_routing_info()
        _ck(_lib.snn_routing_info_get(self.h, ctypes.byref(i)), "snn_routing_info_get")
        d = {f: getattr(i, f) for f, _ in snn_routing_info._fields_ if f != "reserved"}
        d["group_cost"] = d.pop("group_cost_lo") + (d.pop("group_cost_hi") << 64)
        return d

    def groups(self):
        vn = np.empty(self.P, np.int32)
        relay = np.empty(self.n_vn * self.n_vn, np.int32)
        _ck(_lib.snn_routing_groups(self.h, vn.ctypes.data, relay.ctypes.data), "snn_routing_groups")
        return vn, relay.reshape(self.n_vn, self.n_vn)

    def connections(self):
        a = np.empty(self.P, np.int32)
        b = np.empty(self.P, np.int32)
        _ck(_lib.snn_routing_connections(self.h, a.ctypes.data, b.ctypes.data),
            "snn_routing_connections")
        return a, b

    def relays(self, policy=None) -> np.ndarray:
        """[n_vn, P] relay label of each (destination VN, source partition),
        -1 inside the own VN; policy None: the routing's own (snn_routing_relays)."""
        out = np.empty(self.n_vn * self.P, np.int32)
        code = -1 if policy is None else RELAY_POLICIES.get(policy, policy)
        _ck(_lib.snn_routing_relays(self.h, int(code), out.ctypes.data), "snn_routing_relays")
        return out.reshape(self.n_vn, self.P)

    def traffic(self, ids, policy=None) -> dict:
        """Messages per partition (label order) that the spikes `ids` (global
        ids, repeats count again) cause on the direct and the two-level route,
        sent and received, with the relays of `policy` (None: the routing's
        own; snn_routing_traffic)."""
        ids = np.ascontiguousarray(ids, np.uint32)
        code = -1 if policy is None else RELAY_POLICIES.get(policy, policy)
        out = {k: np.zeros(self.P, np.int64) for k in ("direct_out", "direct_in", "two_level_out", "two_level_in")}
        _ck(_lib.snn_routing_traffic(self.h, ids.ctypes.data, len(ids), int(code), out["direct_out"].ctypes.data,
                                     out["direct_in"].ctypes.data, out["two_level_out"].ctypes.data,
                                     out["two_level_in"].ctypes.data), "snn_routing_traffic")
        return out

    def close(self):
        if getattr(self, "h", None):
            _lib.snn_routing_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def sim_params(dyn=None, **kw) -> snn_sim_params:
    """snn_sim_params from library defaults, a dynamics record (dt_ms, tau_ms,
    e_l, v_th, v_reset, t_ref, drive_lambda, w_ext, i_bias, drive_seed) and
    keyword overrides."""
    p = snn_sim_params()
    _lib.snn_sim_params_default(ctypes.byref(p))
    if dyn is not None:
        for f in ("dt_ms", "tau_ms", "e_l", "v_th", "v_reset", "t_ref", "drive_lambda", "w_ext",
                  "i_bias", "drive_seed"):
            setattr(p, f, getattr(dyn, f))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Sim:
    """A simulation on one GPU; the workspace is a torch uint8 tensor.

    batch=(off, params_list): the network is a concatenation of len(params_list)
    independent networks, network k owning ids off[k]..off[k+1]-1, each with
    its own drive (drive_lambda, drive_seed of params_list[k]); see
    snn_batch_create."""

    def __init__(self, net: Network, routing: Routing, params: snn_sim_params, device=None,
                 stream=None, batch=None):
        import torch
        self.net, self.routing, self.params = net, routing, params
        self.M = net.M
        dev = torch.device(device if device is not None else "cuda")
        self.device = dev
        nb = ctypes.c_size_t(0)
        if batch is not None:
            off, plist = batch
            self._off = np.ascontiguousarray(off, np.int64)
            self._plist = (snn_sim_params * len(plist))(*plist)
            n = len(plist)
            _ck(_lib.snn_batch_workspace_bytes(routing.h, n, self._plist, ctypes.byref(nb)),
                "snn_batch_workspace_bytes")
        else:
            _ck(_lib.snn_sim_workspace_bytes(routing.h, ctypes.byref(params), ctypes.byref(nb)),
                "snn_sim_workspace_bytes")
        self.workspace_bytes = nb.value
        with torch.cuda.device(dev):
            self.workspace = torch.empty(max(256, nb.value), dtype=torch.uint8, device=dev)
            self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
            h = _vp()
            if batch is not None:
                _ck(_lib.snn_batch_create(ctypes.byref(net.s), routing.h, n, self._off.ctypes.data, self._plist,
                                          self.workspace.data_ptr(), nb.value, self.stream.cuda_stream,
                                          ctypes.byref(h)), "snn_batch_create")
            else:
                _ck(_lib.snn_sim_create(ctypes.byref(net.s), routing.h, ctypes.byref(params),
                                        self.workspace.data_ptr(), nb.value, self.stream.cuda_stream,
                                        ctypes.byref(h)), "snn_sim_create")
        self.h = h.value

    def _dev(self):
        import torch
        return torch.cuda.device(self.device)

    def step(self, T: int):
        with self._dev():
            _ck(_lib.snn_step(self.h, int(T)), "snn_step")

    def sync_status(self) -> int:
        with self._dev():
            return int(_lib.snn_sync_status(self.h))

    def read_raster(self, t0: int, t1: int):
        n = ctypes.c_int64(-1)
        off = np.zeros(t1 - t0 + 1, np.int64)
        with self._dev():
            rc = _lib.snn_read_raster(self.h, t0, t1, None, 0, off.ctypes.data, ctypes.byref(n))
            if rc != 0 and not (rc == SNN_E_CAPACITY and n.value >= 0):
                _ck(rc, "snn_read_raster")
            ids = np.zeros(max(1, n.value), np.uint32)
            _ck(_lib.snn_read_raster(self.h, t0, t1, ids.ctypes.data, len(ids), off.ctypes.data,
                                     ctypes.byref(n)), "snn_read_raster")
        return ids[: n.value], off

    def read_currents(self, t: int) -> np.ndarray:
        out = np.empty(self.M, np.int32)
        with self._dev():
            _ck(_lib.snn_read_currents(self.h, t, out.ctypes.data), "snn_read_currents")
        return out

    def read_hashes(self, t0: int, t1: int):
        a = np.zeros(t1 - t0, np.uint64)
        b = np.zeros(t1 - t0, np.uint64)
        with self._dev():
            _ck(_lib.snn_read_hashes(self.h, t0, t1, a.ctypes.data, b.ctypes.data), "snn_read_hashes")
        return a, b

    def read_counts(self) -> dict:
        c = snn_counts()
        with self._dev():
            _ck(_lib.snn_read_counts(self.h, ctypes.byref(c)), "snn_read_counts")
        return {f: int(getattr(c, f)) for f in COUNT_FIELDS}

    def read_state(self):
        V = np.empty(self.M, np.float32)
        ref = np.empty(self.M, np.uint8)
        t = ctypes.c_int64(0)
        with self._dev():
            _ck(_lib.snn_read_state(self.h, V.ctypes.data, ref.ctypes.data, ctypes.byref(t)),
                "snn_read_state")
        return V, ref, int(t.value)

    def read_inbox_pairs(self) -> np.ndarray:
        n = ctypes.c_int64(0)
        with self._dev():
            _ck(_lib.snn_read_inbox_pairs(self.h, None, 0, ctypes.byref(n)), "snn_read_inbox_pairs")
            out = np.zeros(max(1, n.value), np.uint64)
            _ck(_lib.snn_read_inbox_pairs(self.h, out.ctypes.data, len(out), ctypes.byref(n)),
                "snn_read_inbox_pairs")
        return out[: n.value]

    def save_state(self) -> bytes:
        nb = ctypes.c_size_t(0)
        _ck(_lib.snn_state_bytes(self.h, ctypes.byref(nb)), "snn_state_bytes")
        buf = ctypes.create_string_buffer(nb.value)
        with self._dev():
            _ck(_lib.snn_save_state(self.h, buf, nb.value), "snn_save_state")
        return buf.raw

    def load_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        with self._dev():
            _ck(_lib.snn_load_state(self.h, buf, len(blob)), "snn_load_state")

    def reset(self, reupload: bool = False):
        with self._dev():
            _ck(_lib.snn_sim_reset(self.h, int(bool(reupload))), "snn_sim_reset")

    def autotune(self, steps: int = 200):
        """Pick the fastest launch shape (see snn_autotune); returns (choice, ms per step)."""
        c = _i32(0)
        ms = ctypes.c_double(0.0)
        with self._dev():
            _ck(_lib.snn_autotune(self.h, int(steps), ctypes.byref(c), ctypes.byref(ms)), "snn_autotune")
        return int(c.value), float(ms.value)

    def profile_phases(self, T: int) -> np.ndarray:
        """Advance T steps and return the summed ms of the parts of a step
        (snn_profile_phases): persistent path [update, compaction, own-table
        prefetch and queued deliveries, rest of the first barrier wait, routing
        walk, routing deliveries and copies, next step's input-free update and
        the second barrier wait]; graph path [k_update, 0, 0, 0, k_route, 0, 0]."""
        out = np.zeros(7, np.float64)
        with self._dev():
            _ck(_lib.snn_profile_phases(self.h, int(T), out.ctypes.data), "snn_profile_phases")
        return out

    def deliver_spikes(self, ids, out):
        """Route and fan out global spike ids (a torch int32/uint32-compatible CUDA
        tensor of int32) into out (CUDA int32 tensor [max_delay, M], accumulated).
        Returns (level-1 entries, level-2 entries, events)."""
        import torch
        assert ids.is_cuda and out.is_cuda and out.dtype == torch.int32 and ids.dtype == torch.int32
        assert ids.is_contiguous() and out.is_contiguous()
        c = np.zeros(3, np.uint64)
        with self._dev():
            _ck(_lib.snn_deliver_spikes(self.h, ids.data_ptr(), ids.numel(), out.data_ptr(),
                                        c.ctypes.data), "snn_deliver_spikes")
        return tuple(int(x) for x in c)

    def launches(self, T: int) -> int:
        """Kernel launches one step(T) issues."""
        return int(_lib.snn_launches(self.h, int(T)))

    @property
    def launches_per_step(self) -> int:
        return int(_lib.snn_launches_per_step(self.h))

    def close(self):
        if getattr(self, "h", None):
            _lib.snn_sim_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


# ---------------------------------------------------------------- adjoint
def adjoint_params(**kw) -> snn_adjoint_params:
    ap = snn_adjoint_params()
    _lib.snn_adjoint_params_default(ctypes.byref(ap))
    for k, v in kw.items():
        if not hasattr(ap, k):
            raise KeyError(k)
        setattr(ap, k, v)
    return ap


class Adjoint:
    """The surrogate-gradient adjoint of the step (see snn_adjoint_create):
    forward(G, lam) -> population rates, backward(dL/drates) -> (dG, dlam)."""

    def __init__(self, net: Network, is_exc, routing: Routing, params: snn_sim_params,
                 aparams: snn_adjoint_params, device=None, stream=None):
        import torch
        self.net, self.routing, self.params, self.aparams = net, routing, params, aparams
        self.is_exc = np.ascontiguousarray(is_exc, np.uint8)
        self.n_pop = 2 * routing.info()["n_vn"]
        dev = torch.device(device if device is not None else "cuda")
        self.device = dev
        nb = ctypes.c_size_t(0)
        _ck(_lib.snn_adjoint_workspace_bytes(routing.h, ctypes.byref(params), ctypes.byref(aparams),
                                             ctypes.byref(nb)), "snn_adjoint_workspace_bytes")
        with torch.cuda.device(dev):
            self.workspace = torch.empty(max(256, nb.value), dtype=torch.uint8, device=dev)
            self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
            h = _vp()
            _ck(_lib.snn_adjoint_create(ctypes.byref(net.s), self.is_exc.ctypes.data, routing.h,
                                        ctypes.byref(params), ctypes.byref(aparams), self.workspace.data_ptr(),
                                        nb.value, self.stream.cuda_stream, ctypes.byref(h)), "snn_adjoint_create")
        self.h = h.value

    def forward(self, G, lam):
        G = np.ascontiguousarray(G, np.float32).reshape(self.n_pop, self.n_pop)
        lam = np.ascontiguousarray(lam, np.float32)
        rates = np.zeros(self.n_pop, np.float32)
        n = _i64(0)
        with torch_device(self.device):
            _ck(_lib.snn_adjoint_forward(self.h, G.ctypes.data, lam.ctypes.data, rates.ctypes.data,
                                         ctypes.byref(n)), "snn_adjoint_forward")
        self.spikes = int(n.value)
        return rates

    def backward(self, grates):
        g = np.ascontiguousarray(grates, np.float64)
        dG = np.zeros((self.n_pop, self.n_pop), np.float64)
        dlam = np.zeros(self.n_pop, np.float64)
        with torch_device(self.device):
            _ck(_lib.snn_adjoint_backward(self.h, g.ctypes.data, dG.ctypes.data, dlam.ctypes.data),
                "snn_adjoint_backward")
        return dG, dlam

    def spikes_of_last_forward(self):
        """(step, global id) of every spike of the last forward, sorted."""
        n = _i64(0)
        _ck(_lib.snn_adjoint_read_spikes(self.h, None, 0, ctypes.byref(n)), "snn_adjoint_read_spikes")
        out = np.zeros(max(1, n.value), np.uint64)
        _ck(_lib.snn_adjoint_read_spikes(self.h, out.ctypes.data, n.value, ctypes.byref(n)),
            "snn_adjoint_read_spikes")
        out = np.sort(out[:n.value])
        return (out >> np.uint64(32)).astype(np.int64), (out & np.uint64(0xFFFFFFFF)).astype(np.int64)

    def close(self):
        if getattr(self, "h", None):
            _lib.snn_adjoint_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def torch_device(dev):
    import torch
    return torch.cuda.device(dev)


def make_adjoint_function():
    """torch.autograd.Function over an Adjoint: rates = f(G, lam); the
    backward calls the adjoint kernels.  G, lam: CPU or CUDA float tensors."""
    import torch

    class AdjointFunction(torch.autograd.Function):
        @staticmethod
        def forward(ctx, G, lam, adj):
            ctx.adj = adj
            ctx.devs = (G.device, lam.device)
            rates = adj.forward(G.detach().cpu().numpy(), lam.detach().cpu().numpy())
            return torch.from_numpy(rates.astype(np.float64)).to(G.device)

        @staticmethod
        def backward(ctx, grates):
            dG, dlam = ctx.adj.backward(grates.detach().cpu().numpy().astype(np.float64))
            return (torch.from_numpy(dG).to(ctx.devs[0], dtype=torch.float32),
                    torch.from_numpy(dlam).to(ctx.devs[1], dtype=torch.float32), None)

    return AdjointFunction
