/*
 * Seeded synthetic network generator.
 *
 * This module produces the *inputs* of a simulation: the synapse list of a
 * partitioned random LIF network and its initial membrane potentials.  It
 * holds none of the simulation's arithmetic (no neuron update, no routing,
 * no delivery) and is shared by the CPU oracle and the GPU library tests.
 *
 * Network recipe (the paper gives no model; the recipe stands in for its
 * scanned human-brain network, see the workload tables in the design notes):
 *   - M neurons split into P contiguous "planted" partitions,
 *     start(p) = floor(p*M/P); planted virtual nodes (VNs) are runs of
 *     `vn_size` consecutive partitions.
 *   - the first round(0.8*size) ids of each planted partition are excitatory.
 *   - every neuron has exactly K out-synapses (source-major CSR, row i holds
 *     synapses K*i .. K*i+K-1):
 *       uniform mode: targets uniform over all other neurons;
 *       locality mode: n_part targets uniform in the own partition (no
 *       autapse), n_vn uniform over the other partitions of the own VN,
 *       n_remote uniform over neurons outside the own VN.
 *     Targets are drawn with replacement (multapses allowed).
 *   - weights in fixed point (units of 2^-10 mV): excitatory
 *     lround(mu_e + sd_e*z) clamped to [1, 32767], inhibitory
 *     -lround(mu_i + sd_i*z) clamped to [-32768, -1], with z an Irwin-Hall
 *     (sum of 12 uniforms minus 6) approximately standard normal variate,
 *     computed exactly in double so every platform produces the same bits.
 *   - delays uniform in 1..dmax steps.
 *   - V0 = v_reset + u*(v_th - v_reset), u uniform in [0,1).
 *
 * Randomness: splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014) seeded per neuron, so neurons are
 * generated independently and in parallel with bit-identical results for
 * any thread count.
 */
#include <stdint.h>
#include <math.h>

static inline uint64_t sm64_next(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform integer in [0, n) by 64x64->128 multiply-shift */
static inline uint64_t below(uint64_t *s, uint64_t n)
{
    return (uint64_t)(((unsigned __int128)sm64_next(s) * n) >> 64);
}

static inline int64_t pstart(int64_t M, int64_t P, int64_t p)
{
    return (p * M) / P;
}

/* Irwin-Hall(12) - 6, exact in double (the sum of twelve 32-bit fractions
 * needs at most 36 significant bits). */
static inline double irwin_hall(uint64_t *s)
{
    uint64_t acc = 0;
    for (int k = 0; k < 6; ++k) {
        uint64_t r = sm64_next(s);
        acc += (r & 0xFFFFFFFFULL) + (r >> 32);
    }
    return (double)acc * (1.0 / 4294967296.0) - 6.0;
}

int synth_planted_start(int64_t M, int32_t P, int32_t p, int64_t *out)
{
    if (M <= 0 || P <= 0 || p < 0 || p > P) return -1;
    *out = pstart(M, P, p);
    return 0;
}

/*
 * Fill a network.  Arrays are caller-owned:
 *   syn_ptr[M+1] (int64), tgt[M*K] (u32), w[M*K] (i16), d[M*K] (u8),
 *   v0[M] (f32), is_exc[M] (u8).
 * Returns 0, or -1 on invalid arguments.
 */
int synth_fill(int64_t M, int32_t P, int32_t vn_size, int32_t K,
               int32_t uniform_all, int32_t n_part, int32_t n_vn, int32_t n_remote,
               int32_t dmax, uint64_t seed,
               double v_reset, double v_th, double frac_exc,
               double mu_e, double sd_e, double mu_i, double sd_i,
               int64_t *syn_ptr, uint32_t *tgt, int16_t *w, uint8_t *d,
               float *v0, uint8_t *is_exc)
{
    if (M < 2 || P < 1 || P > M || K < 0 || dmax < 1 || dmax > 255) return -1;
    if (M > 0xFFFFFFFFLL) return -1;
    if (!uniform_all) {
        if (vn_size < 1 || P % vn_size) return -1;
        if (M / P < 2) return -1;
        if (n_part + n_vn + n_remote != K || n_part < 0 || n_vn < 0 || n_remote < 0) return -1;
        if (vn_size == 1 && n_vn > 0) return -1;
        if (P == vn_size && n_remote > 0) return -1;
    }
    for (int64_t i = 0; i <= M; ++i) syn_ptr[i] = i * (int64_t)K;

    #pragma omp parallel for schedule(static, 256)
    for (int64_t i = 0; i < M; ++i) {
        uint64_t s = sm64_mix(seed ^ sm64_mix((uint64_t)i + 0x1234567ULL));
        /* planted partition of i: largest p with start(p) <= i */
        int64_t p = ((i + 1) * (int64_t)P - 1) / M;
        while (p > 0 && pstart(M, P, p) > i) --p;
        while (p + 1 < P && pstart(M, P, p + 1) <= i) ++p;
        int64_t ps = pstart(M, P, p), pe = pstart(M, P, p + 1), psz = pe - ps;
        int64_t nexc = (int64_t)floor(frac_exc * (double)psz + 0.5);
        int exc = (i - ps) < nexc;
        is_exc[i] = (uint8_t)exc;
        double u = (double)(sm64_next(&s) >> 11) * (1.0 / 9007199254740992.0);
        v0[i] = (float)(v_reset + u * (v_th - v_reset));

        int64_t g = uniform_all ? 0 : p / vn_size;
        int64_t vs = uniform_all ? 0 : pstart(M, P, g * vn_size);
        int64_t ve = uniform_all ? 0 : pstart(M, P, (g + 1) * vn_size);
        int64_t base = i * (int64_t)K;
        for (int32_t k = 0; k < K; ++k) {
            int64_t t;
            if (uniform_all) {
                t = (int64_t)below(&s, (uint64_t)(M - 1));
                if (t >= i) ++t;
            } else if (k < n_part) {
                t = ps + (int64_t)below(&s, (uint64_t)(psz - 1));
                if (t >= i) ++t;
            } else if (k < n_part + n_vn) {
                t = vs + (int64_t)below(&s, (uint64_t)((ve - vs) - psz));
                if (t >= ps) t += psz;
            } else {
                t = (int64_t)below(&s, (uint64_t)(M - (ve - vs)));
                if (t >= vs) t += (ve - vs);
            }
            tgt[base + k] = (uint32_t)t;
            double z = irwin_hall(&s);
            long q;
            if (exc) {
                q = lround(mu_e + sd_e * z);
                if (q < 1) q = 1;
                if (q > 32767) q = 32767;
            } else {
                q = -lround(mu_i + sd_i * z);
                if (q > -1) q = -1;
                if (q < -32768) q = -32768;
            }
            w[base + k] = (int16_t)q;
            d[base + k] = (uint8_t)(1 + below(&s, (uint64_t)dmax));
        }
    }
    return 0;
}
