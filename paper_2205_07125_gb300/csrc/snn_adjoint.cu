// Surrogate-gradient adjoint of the partitioned LIF step (sm_103a).
//
// No counterpart in the paper (arXiv 2205.07125 simulates, it does not
// train).  The differentiable form keeps the step's routing and integer
// delivery and adds population-pair gains G and per-population drive rates
// lam as parameters:
//   populations  pop(j) = 2 vn(j) + (1 if j is inhibitory), n_pop = 2 n_vn;
//   inputs       A_jb(t) = int32 sum of the weights from population b
//                arriving at j at step t (delivered through the two-level
//                route's tables, kept per source population);
//   current      I_j = (((G[a][0] A_j0 + G[a][1] A_j1) + ...) + w_ext (lam_a
//                + sigma xi_j(t)), fp32, fixed order, no FMA; xi_j(t) =
//                (sum of 12 bytes of Philox4x32-10 (j, t, 0xAD, 0) - 1530) / 256;
//   membrane     as the plain step (hard threshold, reset, refractory).
// Forward: T steps from the initial state with checkpoints of (V, ref, ring)
// every K steps; population spike counts give the rates.  Backward
// (surrogate 1 / (1 + beta |V_pre - theta|)^2, reset detached): segment by
// segment from the last checkpoint, the segment's steps are recomputed with
// their V_pre, spike/refractory flags and inputs recorded, then walked
// backwards: every neuron gathers the adjoints of its targets along its own
// level-2 entries and synapse segments (the transpose of the routed
// delivery), and the parameter gradients accumulate in float64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "snn_internal.h"

using namespace snn;

namespace {

constexpr int kAThreads = 256;
constexpr int kMaxPop = 8;
constexpr uint32_t kNoiseTag = 0xAD;

struct AdjDev {
    long long M;
    int n_pop, D, t_ref;
    float alpha, e_l, v_th, v_reset, w_ext, sigma, beta;
    uint32_t key0, key1;
    // state
    float *V;
    uint8_t *ref;
    int32_t *ring;          // [D][M][n_pop]
    const uint8_t *pop;     // [M] internal order
    const uint32_t *gid;    // internal -> global id (nullptr: identical)
    // tables (internal order)
    const uint2 *row;       // [M+1] {first level-1 entry, first level-2 entry}
    const L2Entry *l2;      // [n_l2]
    const uint32_t *syn_td; // [E] target | (delay - 1) << 28
    const int16_t *syn_w;   // [E]
    // step
    uint32_t *spk;          // [2][M] spikes of a step, by parity
    unsigned int *spk_n;    // [2]
    unsigned long long *pop_cnt;  // [n_pop] spikes per population (forward)
    unsigned long long *raster;   // [raster_cap] (t << 32 | global id)
    unsigned long long *raster_n;
    long long raster_cap;
    // parameters
    const float *G;         // [n_pop][n_pop]
    const float *lam;       // [n_pop]
    // recorded segment
    float *seg_vpre;        // [K][M]
    uint8_t *seg_flag;      // [K][M] bit 0 spike, bit 1 refractory
    int32_t *seg_A;         // [K][M][n_pop]
    // backward
    float *gring;           // [D][n_pop][M] G[pop k][b] * (adjoint of V_pre of k) by step slot and
                            // source population b: a source of population b gathers plane b
    float *gV;              // [M]
    const float *direct;    // [n_pop] dL/dr_a / (T N_a)
    double *dG;             // [n_pop][n_pop]
    double *dlam;           // [n_pop]
};

__device__ __forceinline__ uint4 philox_ctr(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2,
                                            uint32_t c3)
{
    uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = c3;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, x0), lo0 = 0xD2511F53u * x0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, x2), lo1 = 0xCD9E8D57u * x2;
        const uint32_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(x0, x1, x2, x3);
}

__device__ __forceinline__ int byte_sum(uint32_t w)
{
    return (int)(w & 0xFFu) + (int)((w >> 8) & 0xFFu) + (int)((w >> 16) & 0xFFu) + (int)(w >> 24);
}

// xi_j(t): exact multiple of 2^-8
__device__ __forceinline__ float noise_of(const AdjDev &a, uint32_t g, uint32_t t)
{
    const uint4 w = philox_ctr(a.key0, a.key1, g, t, kNoiseTag, 0u);
    const int n = byte_sum(w.x) + byte_sum(w.y) + byte_sum(w.z) - 1530;
    return __fdiv_rn((float)n, 256.0f);
}

// One step t of the forward for every neuron (thread per neuron).  rec >= 0:
// record V_pre, flags and inputs in segment slot rec; count: add the spikes
// to the population counts and the raster.
__global__ void __launch_bounds__(kAThreads) k_adj_update(const AdjDev a, int t, int rec, int count)
{
    __shared__ unsigned long long s_cnt[kMaxPop];
    if (threadIdx.x < kMaxPop) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int par = t & 1;
    const int slot = t % a.D;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.spk_n[par ^ 1] = 0;  // the next step's list
    for (long long k = (long long)blockIdx.x * kAThreads + threadIdx.x; k < a.M;
         k += (long long)gridDim.x * kAThreads) {
        const int p = a.pop[k];
        int32_t *rg = a.ring + ((long long)slot * a.M + k) * a.n_pop;
        float irec = 0.0f;
        for (int b = 0; b < a.n_pop; ++b) {
            const int32_t A = rg[b];
            rg[b] = 0;
            if (rec >= 0) a.seg_A[((long long)rec * a.M + k) * a.n_pop + b] = A;
            const float x = __fmul_rn(a.G[p * a.n_pop + b], (float)A);
            irec = b == 0 ? x : __fadd_rn(irec, x);
        }
        const uint32_t g = a.gid ? a.gid[k] : (uint32_t)k;
        const float x1 = __fmul_rn(a.sigma, noise_of(a, g, (uint32_t)t));
        const float x2 = __fadd_rn(a.lam[p], x1);
        const float drv = __fmul_rn(a.w_ext, x2);
        const float I = __fadd_rn(irec, drv);
        const uint8_t r = a.ref[k];
        const bool refr = r > 0;
        float v = a.V[k];
        const float u = __fsub_rn(v, a.e_l);
        const float au = __fmul_rn(a.alpha, u);
        float vp = __fadd_rn(a.e_l, au);
        vp = __fadd_rn(vp, __fmul_rn(I, 0.0009765625f));
        const bool S = !refr && vp >= a.v_th;
        if (rec >= 0) {
            a.seg_vpre[(long long)rec * a.M + k] = vp;
            a.seg_flag[(long long)rec * a.M + k] = (uint8_t)((S ? 1 : 0) | (refr ? 2 : 0));
        }
        a.V[k] = (refr || S) ? a.v_reset : vp;
        a.ref[k] = refr ? (uint8_t)(r - 1) : (S ? (uint8_t)a.t_ref : (uint8_t)0);
        if (S) {
            const unsigned int pos = atomicAdd(&a.spk_n[par], 1u);
            a.spk[(long long)par * a.M + pos] = (uint32_t)k;
            if (count) {
                atomicAdd(&s_cnt[p], 1ull);
                const unsigned long long rp = atomicAdd(a.raster_n, 1ull);
                if ((long long)rp < a.raster_cap) a.raster[rp] = ((unsigned long long)t << 32) | g;
            }
        }
    }
    __syncthreads();
    if (count && threadIdx.x < a.n_pop && s_cnt[threadIdx.x]) atomicAdd(&a.pop_cnt[threadIdx.x], s_cnt[threadIdx.x]);
}

// Delivery of step t's spikes through the routing tables: one warp per
// spike walks its level-2 entries (one synapse segment each) and adds every
// weight to the ring slot of its delay, column = the source population.
__global__ void __launch_bounds__(kAThreads) k_adj_deliver(const AdjDev a, int t)
{
    const int par = t & 1;
    const unsigned int n = *(volatile unsigned int *)&a.spk_n[par];
    const int lane = threadIdx.x & 31;
    const unsigned int nw = (gridDim.x * kAThreads) >> 5;
    for (unsigned int s = (blockIdx.x * kAThreads + threadIdx.x) >> 5; s < n; s += nw) {
        const uint32_t i = a.spk[(long long)par * a.M + s];
        const int pi = a.pop[i];
        const uint32_t f0 = a.row[i].y, f1 = a.row[i + 1].y;
        for (uint32_t f = f0; f < f1; ++f) {
            const L2Entry l = a.l2[f];
            const unsigned long long o = l.off & kOffMask;
            for (uint32_t x = lane; x < l.len; x += 32) {
                const uint32_t td = a.syn_td[o + x];
                int sl = t + (int)(td >> kTgtBits) + 1;
                sl %= a.D;
                atomicAdd(&a.ring[((long long)sl * a.M + (td & kTgtMask)) * a.n_pop + pi], (int32_t)a.syn_w[o + x]);
            }
        }
    }
}

// One backward step t (segment slot rec) for every neuron, a warp each: the
// gather of the targets' adjoints along the neuron's level-2 entries, the
// neuron's adjoint recursion and its parameter-gradient terms.
__global__ void __launch_bounds__(kAThreads) k_adj_backward(const AdjDev a, int t, int rec)
{
    __shared__ double s_dG[kMaxPop * kMaxPop];
    __shared__ double s_dl[kMaxPop];
    for (int x = threadIdx.x; x < kMaxPop * kMaxPop; x += kAThreads) s_dG[x] = 0.0;
    if (threadIdx.x < kMaxPop) s_dl[threadIdx.x] = 0.0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * kAThreads) >> 5;
    const float c = 0.0009765625f;
    const int tm = t % a.D;
    for (long long j = ((long long)blockIdx.x * kAThreads + threadIdx.x) >> 5; j < a.M; j += nw) {
        const int pj = a.pop[j];
        float acc = 0.0f;
        // the neuron's level-2 entries tile one contiguous run of synapses:
        // walk it with four loads per lane in flight
        const uint32_t f0 = a.row[j].y, f1 = a.row[j + 1].y;
        if (f0 < f1) {
            const unsigned long long b0 = a.l2[f0].off & kOffMask;
            const L2Entry last = a.l2[f1 - 1];
            const unsigned long long b1 = (last.off & kOffMask) + last.len;
            for (unsigned long long x0 = b0 + lane; x0 < b1; x0 += 128) {
                uint32_t td[4];
                int32_t w[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const unsigned long long x = x0 + 32ull * u;
                    td[u] = x < b1 ? a.syn_td[x] : 0u;
                    w[u] = x < b1 ? (int32_t)a.syn_w[x] : 0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t k = td[u] & kTgtMask;
                    int sl = tm + (int)(td[u] >> kTgtBits) + 1;
                    if (sl >= a.D) sl -= a.D;
                    // G[pop k][pj] * gVpre_k(t + d), stored by k when it was computed
                    const float hk = a.gring[((long long)sl * a.n_pop + pj) * a.M + k];
                    acc = __fadd_rn(acc, __fmul_rn((float)w[u], hk));
                }
            }
        }
#pragma unroll
        for (int sft = 16; sft > 0; sft >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, sft));
        if (lane == 0) {
            const float gS = __fadd_rn(a.direct[pj], __fmul_rn(c, acc));
            const uint8_t fl = a.seg_flag[(long long)rec * a.M + j];
            float gvp = 0.0f;
            if (!(fl & 2)) {
                const float x = __fsub_rn(a.seg_vpre[(long long)rec * a.M + j], a.v_th);
                const float den = __fadd_rn(1.0f, __fmul_rn(a.beta, fabsf(x)));
                const float sg = __frcp_rn(__fmul_rn(den, den));
                const float keep = (fl & 1) ? 0.0f : a.gV[j];
                gvp = __fadd_rn(keep, __fmul_rn(gS, sg));
            }
            // the products each source population gathers
            for (int b = 0; b < a.n_pop; ++b)
                a.gring[((long long)tm * a.n_pop + b) * a.M + j] = __fmul_rn(a.G[pj * a.n_pop + b], gvp);
            a.gV[j] = __fmul_rn(a.alpha, gvp);
            if (gvp != 0.0f) {
                const double gd = (double)gvp * (double)c;
                for (int b = 0; b < a.n_pop; ++b)
                    atomicAdd(&s_dG[pj * a.n_pop + b], gd * (double)a.seg_A[((long long)rec * a.M + j) * a.n_pop + b]);
                atomicAdd(&s_dl[pj], gd * (double)a.w_ext);
            }
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < a.n_pop * a.n_pop; x += kAThreads)
        if (s_dG[x] != 0.0) atomicAdd(&a.dG[x], s_dG[x]);
    if (threadIdx.x < a.n_pop && s_dl[threadIdx.x] != 0.0) atomicAdd(&a.dlam[threadIdx.x], s_dl[threadIdx.x]);
}

struct Region {
    size_t off = 0, bytes = 0;
};

struct ALayout {
    Region V, ref, ring, pop, gid, row, l2, syn_td, syn_w, spk, spk_n, pop_cnt, raster, raster_n;
    Region G, lam, seg_vpre, seg_flag, seg_A, gring, gV, direct, dG, dlam;
    Region ck_V, ck_ref, ck_ring;  // [n_ckpt] checkpoints
    size_t total = 0;
    int D = 2, n_pop = 2, n_ckpt = 1;
};

void aplace(ALayout &L, Region &r, size_t bytes)
{
    r.off = L.total;
    r.bytes = bytes;
    L.total += (bytes + 255) & ~(size_t)255;
}

bool adj_params_ok(const snn_adjoint_params *ap)
{
    return ap && ap->T >= 1 && ap->ckpt_every >= 1 && std::isfinite(ap->sigma) && std::isfinite(ap->beta) &&
           ap->beta > 0.0f;
}

int adj_layout(const snn_routing *rt, const snn_sim_params *p, const snn_adjoint_params *ap, ALayout &L)
{
    const int64_t M = rt->M, E = rt->E;
    L = ALayout();
    L.D = rt->max_delay + 1;
    L.n_pop = 2 * rt->n_vn;
    if (L.n_pop > kMaxPop) return SNN_E_RANGE;
    L.n_ckpt = (ap->T + ap->ckpt_every - 1) / ap->ckpt_every;
    const int K = std::min(ap->T, ap->ckpt_every);
    const size_t ring_b = sizeof(int32_t) * (size_t)L.D * M * L.n_pop;
    aplace(L, L.V, sizeof(float) * M);
    aplace(L, L.ref, M);
    aplace(L, L.ring, ring_b);
    aplace(L, L.pop, M);
    aplace(L, L.gid, rt->identity ? 0 : sizeof(uint32_t) * M);
    aplace(L, L.row, sizeof(uint2) * (M + 1));
    aplace(L, L.l2, sizeof(L2Entry) * rt->n_l2);
    aplace(L, L.syn_td, sizeof(uint32_t) * E);
    aplace(L, L.syn_w, sizeof(int16_t) * E);
    aplace(L, L.spk, sizeof(uint32_t) * 2 * M);
    aplace(L, L.spk_n, 2 * sizeof(unsigned int));
    aplace(L, L.pop_cnt, sizeof(unsigned long long) * kMaxPop);
    aplace(L, L.raster, sizeof(unsigned long long) * (size_t)std::max<int64_t>(0, p->raster_cap));
    aplace(L, L.raster_n, sizeof(unsigned long long));
    aplace(L, L.G, sizeof(float) * kMaxPop * kMaxPop);
    aplace(L, L.lam, sizeof(float) * kMaxPop);
    aplace(L, L.seg_vpre, sizeof(float) * (size_t)K * M);
    aplace(L, L.seg_flag, (size_t)K * M);
    aplace(L, L.seg_A, sizeof(int32_t) * (size_t)K * M * L.n_pop);
    aplace(L, L.gring, sizeof(float) * (size_t)L.D * (size_t)L.n_pop * M);
    aplace(L, L.gV, sizeof(float) * M);
    aplace(L, L.direct, sizeof(float) * kMaxPop);
    aplace(L, L.dG, sizeof(double) * kMaxPop * kMaxPop);
    aplace(L, L.dlam, sizeof(double) * kMaxPop);
    aplace(L, L.ck_V, sizeof(float) * M * (size_t)L.n_ckpt);
    aplace(L, L.ck_ref, (size_t)M * L.n_ckpt);
    aplace(L, L.ck_ring, ring_b * L.n_ckpt);
    return SNN_OK;
}

}  // namespace

struct snn_adjoint {
    const snn_routing *rt = nullptr;
    snn_sim_params prm;
    snn_adjoint_params ap;
    ALayout L;
    AdjDev dev;
    char *ws = nullptr;
    cudaStream_t stream = nullptr;
    unsigned grid_n = 1, grid_w = 1;
    std::vector<double> pop_size;
    bool have_forward = false;
};

#define ACK(x)                                    \
    do {                                          \
        cudaError_t e_ = (x);                     \
        if (e_ != cudaSuccess) return SNN_E_CUDA; \
    } while (0)

extern "C" void snn_adjoint_params_default(snn_adjoint_params *ap)
{
    if (!ap) return;
    std::memset(ap, 0, sizeof(*ap));
    ap->T = 500;
    ap->ckpt_every = 50;
    ap->sigma = 0.9f;
    ap->beta = 5.0f;
}

extern "C" int snn_adjoint_workspace_bytes(const snn_routing *rt, const snn_sim_params *p,
                                           const snn_adjoint_params *ap, size_t *bytes)
{
    if (!rt || !p || !bytes || !adj_params_ok(ap)) return SNN_E_ARG;
    ALayout L;
    int rc = adj_layout(rt, p, ap, L);
    if (rc) return rc;
    *bytes = L.total;
    return SNN_OK;
}

extern "C" int snn_adjoint_create(const snn_network *net, const uint8_t *is_exc, const snn_routing *rt,
                                  const snn_sim_params *p, const snn_adjoint_params *ap, void *workspace,
                                  size_t ws_bytes, void *stream, snn_adjoint **out)
{
    if (!out) return SNN_E_ARG;
    *out = nullptr;
    if (!net || !is_exc || !rt || !p || !adj_params_ok(ap) || !workspace || ((uintptr_t)workspace & 255))
        return SNN_E_ARG;
    if (net->n_neurons != rt->M || p->raster_cap < 0) return SNN_E_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return SNN_E_NODEV;
    snn_adjoint *a = new (std::nothrow) snn_adjoint();
    if (!a) return SNN_E_NOMEM;
    a->rt = rt;
    a->prm = *p;
    a->ap = *ap;
    int rc = adj_layout(rt, p, ap, a->L);
    if (rc) {
        delete a;
        return rc;
    }
    if (ws_bytes < a->L.total) {
        delete a;
        return SNN_E_NOMEM;
    }
    a->ws = (char *)workspace;
    a->stream = (cudaStream_t)stream;
    const ALayout &L = a->L;
    const int64_t M = rt->M;
    char *w = a->ws;
    AdjDev &d = a->dev;
    std::memset(&d, 0, sizeof(d));
    d.M = M;
    d.n_pop = L.n_pop;
    d.D = L.D;
    d.t_ref = p->t_ref;
    d.alpha = (float)std::exp(-p->dt_ms / p->tau_ms);
    d.e_l = p->e_l;
    d.v_th = p->v_th;
    d.v_reset = p->v_reset;
    d.w_ext = (float)p->w_ext;
    d.sigma = ap->sigma;
    d.beta = ap->beta;
    d.key0 = (uint32_t)p->drive_seed;
    d.key1 = (uint32_t)(p->drive_seed >> 32);
    d.V = (float *)(w + L.V.off);
    d.ref = (uint8_t *)(w + L.ref.off);
    d.ring = (int32_t *)(w + L.ring.off);
    d.pop = (const uint8_t *)(w + L.pop.off);
    d.gid = rt->identity ? nullptr : (const uint32_t *)(w + L.gid.off);
    d.row = (const uint2 *)(w + L.row.off);
    d.l2 = (const L2Entry *)(w + L.l2.off);
    d.syn_td = (const uint32_t *)(w + L.syn_td.off);
    d.syn_w = (const int16_t *)(w + L.syn_w.off);
    d.spk = (uint32_t *)(w + L.spk.off);
    d.spk_n = (unsigned int *)(w + L.spk_n.off);
    d.pop_cnt = (unsigned long long *)(w + L.pop_cnt.off);
    d.raster = (unsigned long long *)(w + L.raster.off);
    d.raster_n = (unsigned long long *)(w + L.raster_n.off);
    d.raster_cap = p->raster_cap;
    d.G = (const float *)(w + L.G.off);
    d.lam = (const float *)(w + L.lam.off);
    d.seg_vpre = (float *)(w + L.seg_vpre.off);
    d.seg_flag = (uint8_t *)(w + L.seg_flag.off);
    d.seg_A = (int32_t *)(w + L.seg_A.off);
    d.gring = (float *)(w + L.gring.off);
    d.gV = (float *)(w + L.gV.off);
    d.direct = (const float *)(w + L.direct.off);
    d.dG = (double *)(w + L.dG.off);
    d.dlam = (double *)(w + L.dlam.off);
    // populations (internal order) and their sizes
    std::vector<uint8_t> pop((size_t)M);
    const int32_t s = rt->P / rt->n_vn;
    a->pop_size.assign((size_t)L.n_pop, 0.0);
    for (int32_t ip = 0; ip < rt->P; ++ip)
        for (int64_t k = rt->pbase[ip]; k < rt->pbase[ip + 1]; ++k) {
            const uint32_t g = rt->perm_inv[k];
            pop[k] = (uint8_t)(2 * (ip / s) + (is_exc[g] ? 0 : 1));
            a->pop_size[pop[k]] += 1.0;
        }
    std::vector<uint2> row((size_t)M + 1);
    for (int64_t i = 0; i <= M; ++i) row[i] = make_uint2(rt->l1_ptr[i], rt->l1_l2[rt->l1_ptr[i]]);
    auto up = [&](const Region &r, const void *src) -> cudaError_t {
        return r.bytes ? cudaMemcpy(w + r.off, src, r.bytes, cudaMemcpyHostToDevice) : cudaSuccess;
    };
    if (up(L.pop, pop.data()) || up(L.row, row.data()) || up(L.l2, rt->l2.data()) ||
        up(L.syn_td, rt->syn_td.data()) || up(L.syn_w, rt->syn_w.data()) ||
        (!rt->identity && up(L.gid, rt->perm_inv.data()))) {
        delete a;
        return SNN_E_CUDA;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    a->grid_n = (unsigned)std::max<int64_t>(1, std::min<int64_t>((M + kAThreads - 1) / kAThreads, 65535));
    a->grid_w = (unsigned)std::max(1, sms * 8);
    *out = a;
    return SNN_OK;
}

// Initial state (V = v0, ref = 0, empty ring), empty spike lists and counts.
static int adj_reset(snn_adjoint *a)
{
    const ALayout &L = a->L;
    char *w = a->ws;
    cudaStream_t st = a->stream;
    ACK(cudaMemcpyAsync(w + L.V.off, a->rt->v0.data(), L.V.bytes, cudaMemcpyHostToDevice, st));
    ACK(cudaMemsetAsync(w + L.ref.off, 0, L.ref.bytes, st));
    ACK(cudaMemsetAsync(w + L.ring.off, 0, L.ring.bytes, st));
    ACK(cudaMemsetAsync(w + L.spk_n.off, 0, L.spk_n.bytes, st));
    ACK(cudaMemsetAsync(w + L.pop_cnt.off, 0, L.pop_cnt.bytes, st));
    ACK(cudaMemsetAsync(w + L.raster_n.off, 0, L.raster_n.bytes, st));
    return SNN_OK;
}

static void adj_step(snn_adjoint *a, int t, int rec, int count)
{
    k_adj_update<<<a->grid_n, kAThreads, 0, a->stream>>>(a->dev, t, rec, count);
    k_adj_deliver<<<a->grid_w, kAThreads, 0, a->stream>>>(a->dev, t);
}

extern "C" int snn_adjoint_forward(snn_adjoint *a, const float *G, const float *lam, float *rates,
                                   int64_t *spikes)
{
    if (!a || !G || !lam) return SNN_E_ARG;
    const ALayout &L = a->L;
    char *w = a->ws;
    cudaStream_t st = a->stream;
    const int np = L.n_pop;
    ACK(cudaMemcpyAsync(w + L.G.off, G, sizeof(float) * np * np, cudaMemcpyHostToDevice, st));
    ACK(cudaMemcpyAsync(w + L.lam.off, lam, sizeof(float) * np, cudaMemcpyHostToDevice, st));
    int rc = adj_reset(a);
    if (rc) return rc;
    const int T = a->ap.T, K = a->ap.ckpt_every;
    const int64_t M = a->rt->M;
    const size_t ring_b = L.ring.bytes;
    for (int t = 0; t < T; ++t) {
        if (t % K == 0) {
            const int c = t / K;
            ACK(cudaMemcpyAsync(w + L.ck_V.off + (size_t)c * sizeof(float) * M, w + L.V.off, L.V.bytes,
                                cudaMemcpyDeviceToDevice, st));
            ACK(cudaMemcpyAsync(w + L.ck_ref.off + (size_t)c * M, w + L.ref.off, L.ref.bytes,
                                cudaMemcpyDeviceToDevice, st));
            ACK(cudaMemcpyAsync(w + L.ck_ring.off + (size_t)c * ring_b, w + L.ring.off, ring_b,
                                cudaMemcpyDeviceToDevice, st));
        }
        adj_step(a, t, -1, 1);
    }
    ACK(cudaGetLastError());
    unsigned long long cnt[kMaxPop];
    ACK(cudaMemcpyAsync(cnt, w + L.pop_cnt.off, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    ACK(cudaStreamSynchronize(st));
    int64_t tot = 0;
    for (int b = 0; b < np; ++b) {
        if (rates) rates[b] = (float)((double)cnt[b] / ((double)T * a->pop_size[b]));
        tot += (int64_t)cnt[b];
    }
    if (spikes) *spikes = tot;
    a->have_forward = true;
    return SNN_OK;
}

extern "C" int snn_adjoint_backward(snn_adjoint *a, const double *grates, double *dG, double *dlam)
{
    if (!a || !grates || !dG || !dlam) return SNN_E_ARG;
    if (!a->have_forward) return SNN_E_STATE;
    const ALayout &L = a->L;
    char *w = a->ws;
    cudaStream_t st = a->stream;
    const int np = L.n_pop, T = a->ap.T, K = a->ap.ckpt_every;
    const int64_t M = a->rt->M;
    float direct[kMaxPop] = {0};
    for (int b = 0; b < np; ++b) direct[b] = (float)(grates[b] / ((double)T * a->pop_size[b]));
    ACK(cudaMemcpyAsync(w + L.direct.off, direct, sizeof(direct), cudaMemcpyHostToDevice, st));
    ACK(cudaMemsetAsync(w + L.gring.off, 0, L.gring.bytes, st));
    ACK(cudaMemsetAsync(w + L.gV.off, 0, L.gV.bytes, st));
    ACK(cudaMemsetAsync(w + L.dG.off, 0, L.dG.bytes, st));
    ACK(cudaMemsetAsync(w + L.dlam.off, 0, L.dlam.bytes, st));
    const size_t ring_b = L.ring.bytes;
    for (int c = L.n_ckpt - 1; c >= 0; --c) {
        const int t0 = c * K, t1 = std::min(T, t0 + K);
        // the segment's forward again, from its checkpoint, recorded
        ACK(cudaMemcpyAsync(w + L.V.off, w + L.ck_V.off + (size_t)c * sizeof(float) * M, L.V.bytes,
                            cudaMemcpyDeviceToDevice, st));
        ACK(cudaMemcpyAsync(w + L.ref.off, w + L.ck_ref.off + (size_t)c * M, L.ref.bytes, cudaMemcpyDeviceToDevice,
                            st));
        ACK(cudaMemcpyAsync(w + L.ring.off, w + L.ck_ring.off + (size_t)c * ring_b, ring_b, cudaMemcpyDeviceToDevice,
                            st));
        ACK(cudaMemsetAsync(w + L.spk_n.off, 0, L.spk_n.bytes, st));
        for (int t = t0; t < t1; ++t) adj_step(a, t, t - t0, 0);
        for (int t = t1 - 1; t >= t0; --t)
            k_adj_backward<<<a->grid_w, kAThreads, 0, st>>>(a->dev, t, t - t0);
        ACK(cudaGetLastError());
    }
    ACK(cudaMemcpyAsync(dG, w + L.dG.off, sizeof(double) * np * np, cudaMemcpyDeviceToHost, st));
    ACK(cudaMemcpyAsync(dlam, w + L.dlam.off, sizeof(double) * np, cudaMemcpyDeviceToHost, st));
    ACK(cudaStreamSynchronize(st));
    return SNN_OK;
}

extern "C" int snn_adjoint_read_spikes(snn_adjoint *a, uint64_t *out, int64_t cap, int64_t *n)
{
    if (!a || !n) return SNN_E_ARG;
    unsigned long long cnt = 0;
    ACK(cudaStreamSynchronize(a->stream));
    ACK(cudaMemcpy(&cnt, a->ws + a->L.raster_n.off, sizeof(cnt), cudaMemcpyDeviceToHost));
    *n = (int64_t)cnt;
    const int64_t m = std::min<int64_t>((int64_t)cnt, std::min<int64_t>(cap, a->prm.raster_cap));
    if (m > 0 && out) ACK(cudaMemcpy(out, a->ws + a->L.raster.off, sizeof(uint64_t) * m, cudaMemcpyDeviceToHost));
    if ((int64_t)cnt > a->prm.raster_cap) return SNN_E_CAPACITY;
    return SNN_OK;
}

extern "C" void snn_adjoint_destroy(snn_adjoint *a)
{
    delete a;
}
