// The model stage of the C ABI: a seeded synthetic network built, saved as
// an edge-list file and loaded again (host C++).  The paper's statement of
// the problem starts here: a simulation model is generated, then dispersed
// over the GPUs (Sec. I); partitioning and routing (Sec. IV) take the model
// as input.  The network recipe is the seeded generator of synth/synth.c,
// which holds none of the simulation's arithmetic.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>

#include "../../include/snn.h"

extern "C" int synth_fill(int64_t M, int32_t P, int32_t vn_size, int32_t K, int32_t uniform_all, int32_t n_part,
                          int32_t n_vn, int32_t n_remote, int32_t dmax, uint64_t seed, double v_reset, double v_th,
                          double frac_exc, double mu_e, double sd_e, double mu_i, double sd_i, int64_t *syn_ptr,
                          uint32_t *tgt, int16_t *w, uint8_t *d, float *v0, uint8_t *is_exc);

struct snn_model {
    int64_t M = 0, E = 0;
    int32_t max_delay = 1;
    std::unique_ptr<int64_t[]> syn_ptr;
    std::unique_ptr<uint32_t[]> tgt;
    std::unique_ptr<int16_t[]> w;
    std::unique_ptr<uint8_t[]> d;
    std::unique_ptr<float[]> v0;
    std::unique_ptr<uint8_t[]> is_exc;

    bool alloc(int64_t m, int64_t e)
    {
        M = m;
        E = e;
        syn_ptr.reset(new (std::nothrow) int64_t[(size_t)m + 1]);
        tgt.reset(new (std::nothrow) uint32_t[(size_t)(e > 0 ? e : 1)]);
        w.reset(new (std::nothrow) int16_t[(size_t)(e > 0 ? e : 1)]);
        d.reset(new (std::nothrow) uint8_t[(size_t)(e > 0 ? e : 1)]);
        v0.reset(new (std::nothrow) float[(size_t)m]);
        is_exc.reset(new (std::nothrow) uint8_t[(size_t)m]);
        return syn_ptr && tgt && w && d && v0 && is_exc;
    }
};

namespace {

// Edge-list file: the magic, then little-endian u64 M, u64 E, u32 max_delay,
// u32 0, then syn_ptr i64[M+1], tgt u32[E], w i16[E], d u8[E], v0 f32[M],
// is_exc u8[M].
constexpr char kMagic[8] = {'S', 'N', 'N', 'M', 'O', 'D', 'L', '1'};

struct Header {
    char magic[8];
    uint64_t M, E;
    uint32_t max_delay, zero;
};
static_assert(sizeof(Header) == 32, "model file header");

bool params_valid(const snn_model_params *p)
{
    if (!p) return false;
    if (p->n_neurons < 2 || p->n_neurons >= ((int64_t)1 << 28)) return false;
    if (p->n_parts < 1 || p->n_parts > p->n_neurons) return false;
    if (p->syn_per_neuron < 0 || p->max_delay < 1 || p->max_delay > 16) return false;
    if ((double)p->n_neurons * (double)p->syn_per_neuron >= 1099511627776.0) return false;  // E < 2^40
    if (!p->uniform) {
        if (p->vn_size < 1 || p->n_parts % p->vn_size) return false;
        if (p->n_same_part < 0 || p->n_same_vn < 0 || p->n_remote < 0) return false;
        if (p->n_same_part + p->n_same_vn + p->n_remote != p->syn_per_neuron) return false;
    }
    if (!(p->frac_exc >= 0.0 && p->frac_exc <= 1.0)) return false;
    return true;
}

}  // namespace

extern "C" int snn_model_params_preset(int32_t workload, snn_model_params *p)
{
    if (!p) return SNN_E_ARG;
    std::memset(p, 0, sizeof(*p));
    p->v_reset = -65.0;
    p->v_th = -50.0;
    p->frac_exc = 0.8;
    p->mu_e = 40.0;
    p->sd_e = 8.0;
    p->mu_i = 160.0;
    p->sd_i = 32.0;
    // the scale locality mix: 70 % same partition, 20 % the rest of the VN,
    // 10 % outside the VN; delays 1..8
    auto mix = [&](int64_t M, int32_t P, int32_t vn_size, int32_t K, uint64_t seed) {
        p->n_neurons = M;
        p->n_parts = P;
        p->vn_size = vn_size;
        p->syn_per_neuron = K;
        p->uniform = 0;
        p->n_same_part = (int32_t)((7 * K + 5) / 10);
        p->n_same_vn = (int32_t)((2 * K + 5) / 10);
        p->n_remote = K - p->n_same_part - p->n_same_vn;
        p->max_delay = 8;
        p->seed = seed;
    };
    switch (workload) {
    case SNN_WORKLOAD_TINY:
        p->n_neurons = 4096;
        p->n_parts = 4;
        p->vn_size = 2;
        p->syn_per_neuron = 100;
        p->uniform = 1;
        p->max_delay = 1;
        p->seed = 1000;
        return SNN_OK;
    case SNN_WORKLOAD_SCALE: mix(1 << 20, 64, 4, 1000, 1001); return SNN_OK;
    case SNN_WORKLOAD_PAPER_SHARE: mix(5000000, 256, 4, 1000, 1002); return SNN_OK;
    case SNN_WORKLOAD_ADJOINT: mix(131072, 8, 4, 500, 1004); return SNN_OK;
    default: return SNN_E_ARG;
    }
}

extern "C" int snn_model_build(const snn_model_params *p, snn_model **out)
{
    if (!out) return SNN_E_ARG;
    *out = nullptr;
    if (!params_valid(p)) return SNN_E_ARG;
    std::unique_ptr<snn_model> m(new (std::nothrow) snn_model());
    if (!m || !m->alloc(p->n_neurons, p->n_neurons * (int64_t)p->syn_per_neuron)) return SNN_E_NOMEM;
    const int rc = synth_fill(p->n_neurons, p->n_parts, p->uniform ? 1 : p->vn_size, p->syn_per_neuron,
                              p->uniform ? 1 : 0, p->n_same_part, p->n_same_vn, p->n_remote, p->max_delay, p->seed,
                              p->v_reset, p->v_th, p->frac_exc, p->mu_e, p->sd_e, p->mu_i, p->sd_i,
                              m->syn_ptr.get(), m->tgt.get(), m->w.get(), m->d.get(), m->v0.get(), m->is_exc.get());
    if (rc != 0) return SNN_E_ARG;
    m->max_delay = p->max_delay;
    *out = m.release();
    return SNN_OK;
}

extern "C" int snn_model_network(const snn_model *m, snn_network *net, const uint8_t **is_exc)
{
    if (!m || !net) return SNN_E_ARG;
    net->n_neurons = m->M;
    net->syn_ptr = m->syn_ptr.get();
    net->syn_tgt = m->tgt.get();
    net->syn_w = m->w.get();
    net->syn_d = m->d.get();
    net->v0 = m->v0.get();
    if (is_exc) *is_exc = m->is_exc.get();
    return SNN_OK;
}

extern "C" int snn_model_save(const snn_model *m, const char *path)
{
    if (!m || !path) return SNN_E_ARG;
    std::FILE *f = std::fopen(path, "wb");
    if (!f) return SNN_E_ARG;
    Header h;
    std::memcpy(h.magic, kMagic, sizeof(kMagic));
    h.M = (uint64_t)m->M;
    h.E = (uint64_t)m->E;
    h.max_delay = (uint32_t)m->max_delay;
    h.zero = 0;
    const size_t M = (size_t)m->M, E = (size_t)m->E;
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
    ok = ok && std::fwrite(m->syn_ptr.get(), sizeof(int64_t), M + 1, f) == M + 1;
    ok = ok && std::fwrite(m->tgt.get(), sizeof(uint32_t), E, f) == E;
    ok = ok && std::fwrite(m->w.get(), sizeof(int16_t), E, f) == E;
    ok = ok && std::fwrite(m->d.get(), sizeof(uint8_t), E, f) == E;
    ok = ok && std::fwrite(m->v0.get(), sizeof(float), M, f) == M;
    ok = ok && std::fwrite(m->is_exc.get(), sizeof(uint8_t), M, f) == M;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? SNN_OK : SNN_E_ARG;
}

extern "C" int snn_model_load(const char *path, snn_model **out)
{
    if (!out || !path) return SNN_E_ARG;
    *out = nullptr;
    std::FILE *f = std::fopen(path, "rb");
    if (!f) return SNN_E_ARG;
    Header h;
    int rc = SNN_OK;
    std::unique_ptr<snn_model> m(new (std::nothrow) snn_model());
    if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, kMagic, sizeof(kMagic)) != 0 || h.M < 1 ||
        h.M >= ((uint64_t)1 << 28) || h.E >= ((uint64_t)1 << 40) || h.max_delay < 1 || h.max_delay > 16) {
        rc = SNN_E_ARG;
    } else if (!m || !m->alloc((int64_t)h.M, (int64_t)h.E)) {
        rc = SNN_E_NOMEM;
    } else {
        const size_t M = (size_t)h.M, E = (size_t)h.E;
        bool ok = std::fread(m->syn_ptr.get(), sizeof(int64_t), M + 1, f) == M + 1;
        ok = ok && std::fread(m->tgt.get(), sizeof(uint32_t), E, f) == E;
        ok = ok && std::fread(m->w.get(), sizeof(int16_t), E, f) == E;
        ok = ok && std::fread(m->d.get(), sizeof(uint8_t), E, f) == E;
        ok = ok && std::fread(m->v0.get(), sizeof(float), M, f) == M;
        ok = ok && std::fread(m->is_exc.get(), sizeof(uint8_t), M, f) == M;
        // the synapse list must be well formed before any other call sees it
        ok = ok && m->syn_ptr[0] == 0 && (uint64_t)m->syn_ptr[M] == (uint64_t)E;
        for (size_t i = 0; ok && i < M; ++i) ok = m->syn_ptr[i] <= m->syn_ptr[i + 1];
        for (size_t k = 0; ok && k < E; ++k) ok = m->tgt[k] < M && m->d[k] >= 1 && m->d[k] <= h.max_delay;
        m->max_delay = (int32_t)h.max_delay;
        rc = ok ? SNN_OK : SNN_E_ARG;
    }
    std::fclose(f);
    if (rc == SNN_OK) *out = m.release();
    return rc;
}

extern "C" void snn_model_destroy(snn_model *m)
{
    delete m;
}
