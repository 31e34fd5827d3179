"""The model stage of the C ABI (snn_model_*): the network built behind the
ABI is the seeded generator's network array for array, the presets are the
workloads' recipes, the edge-list file written by snn_model_save is read by
the oracle's own reader (and by snn_model_load) into the same arrays, and
malformed files and parameters are rejected.  CPU only."""
import os

import numpy as np
import pytest

import oracle
import synth

FIELDS = ("syn_ptr", "tgt", "w", "d", "v0", "is_exc")


@pytest.fixture(scope="module")
def snn():
    import paper_2205_07125_gb300 as m
    return m


def _same(a, b):
    return all(np.array_equal(getattr(a, k), getattr(b, k)) for k in FIELDS)


def _cfg_params(snn, cfg):
    return snn.model_params(n_neurons=cfg.M, n_parts=cfg.P, vn_size=cfg.vn_size, syn_per_neuron=cfg.K,
                            uniform=int(cfg.uniform_all), n_same_part=cfg.n_part, n_same_vn=cfg.n_vn_t,
                            n_remote=cfg.n_remote, max_delay=cfg.dmax, seed=cfg.seed, v_reset=cfg.dyn.v_reset,
                            v_th=cfg.dyn.v_th, frac_exc=cfg.frac_exc, mu_e=cfg.mu_e, sd_e=cfg.sd_e,
                            mu_i=cfg.mu_i, sd_i=cfg.sd_i)


def test_tiny_preset_is_the_generator_network(snn):
    m = snn.Model.build(workload="tiny")
    assert _same(m, synth.make_network(synth.TINY))


@pytest.mark.parametrize("name", ["scale", "paper"])
def test_presets_are_the_workload_recipes(snn, name):
    cfg = {"scale": synth.SCALE, "paper": synth.PAPER_SHARE}[name]
    p = snn.model_params(name)
    q = _cfg_params(snn, cfg)
    for f, _ in snn.snn_model_params._fields_:
        assert getattr(p, f) == getattr(q, f), f


def test_adjoint_preset(snn):
    p = snn.model_params("adjoint")
    assert (p.n_neurons, p.n_parts, p.vn_size, p.syn_per_neuron) == (131072, 8, 4, 500)
    assert (p.n_same_part, p.n_same_vn, p.n_remote, p.max_delay) == (350, 100, 50, 8)


def test_locality_network_of_any_size(snn):
    cfg = synth.SCALE.scaled(M=20_000, P=20, n_vn=5, K=90, n_part=63, n_vn_t=18, n_remote=9, seed=77, dmax=5)
    m = snn.Model.build(_cfg_params(snn, cfg))
    assert _same(m, synth.make_network(cfg))
    assert m.E == cfg.M * cfg.K


def test_file_round_trip_and_oracle_reader(snn, tmp_path):
    cfg = synth.SCALE.scaled(M=8192, P=8, n_vn=2, K=50, n_part=35, n_vn_t=10, n_remote=5, seed=5)
    m = snn.Model.build(_cfg_params(snn, cfg))
    path = str(tmp_path / "net.snnm")
    m.save(path)
    f = oracle.load_model(path)
    g = synth.make_network(cfg)
    assert _same(f, g) and f.max_delay == cfg.dmax and (f.M, f.E) == (cfg.M, cfg.M * cfg.K)
    assert os.path.getsize(path) == 32 + 8 * (cfg.M + 1) + 7 * f.E + 5 * cfg.M
    assert _same(snn.Model.load(path), g)
    # the oracle simulates the file's network exactly as the generator's
    a = oracle.Oracle(f, cfg.P, oracle.partition_planted(f.M, cfg.P), cfg.n_vn,
                      oracle.group_contiguous(cfg.P, cfg.n_vn), cfg.dyn).run(40)
    b = oracle.Oracle(g, cfg.P, oracle.partition_planted(g.M, cfg.P), cfg.n_vn,
                      oracle.group_contiguous(cfg.P, cfg.n_vn), cfg.dyn).run(40)
    assert np.array_equal(a["raster_ids"], b["raster_ids"]) and np.array_equal(a["v_hash"], b["v_hash"])


def test_malformed_files_and_parameters_are_rejected(snn, tmp_path):
    cfg = synth.TINY.scaled(M=300, K=5, seed=9)
    g = synth.make_network(cfg)

    def write(path, M, E, dmax, arrays):
        with open(path, "wb") as fh:
            fh.write(b"SNNMODL1")
            fh.write(np.array([M, E], "<u8").tobytes())
            fh.write(np.array([dmax, 0], "<u4").tobytes())
            for a in arrays:
                fh.write(np.ascontiguousarray(a).tobytes())

    good = [g.syn_ptr, g.tgt, g.w, g.d, g.v0, g.is_exc]
    p = str(tmp_path / "ok.snnm")
    write(p, g.M, g.E, 1, good)
    assert _same(snn.Model.load(p), g)
    bad_tgt = g.tgt.copy()
    bad_tgt[17] = g.M
    bad_ptr = g.syn_ptr.copy()
    bad_ptr[5], bad_ptr[6] = bad_ptr[6], bad_ptr[5] + 1
    cases = {"target": (g.M, g.E, 1, [g.syn_ptr, bad_tgt] + good[2:]),
             "offsets": (g.M, g.E, 1, [bad_ptr] + good[1:]),
             "delay": (g.M, g.E, 1, good[:3] + [np.full(g.E, 2, np.uint8)] + good[4:]),
             "truncated": (g.M, g.E, 1, good[:4])}
    for name, (M, E, dmax, arrays) in cases.items():
        q = str(tmp_path / (name + ".snnm"))
        write(q, M, E, dmax, arrays)
        with pytest.raises(snn.SnnError) as e:
            snn.Model.load(q)
        assert e.value.code == -1, name
    with open(str(tmp_path / "magic.snnm"), "wb") as fh:
        fh.write(b"NOTAMODL" + bytes(24))
    with pytest.raises(snn.SnnError):
        snn.Model.load(str(tmp_path / "magic.snnm"))
    with pytest.raises(snn.SnnError):
        snn.Model.load(str(tmp_path / "missing.snnm"))
    for kw in ({"n_neurons": 1}, {"n_parts": 0}, {"max_delay": 17}, {"n_parts": 6, "uniform": 0, "vn_size": 4},
               {"uniform": 0, "n_same_part": 1, "n_same_vn": 1, "n_remote": 1}):
        with pytest.raises(snn.SnnError):
            snn.Model.build(snn.model_params("tiny", **kw))
