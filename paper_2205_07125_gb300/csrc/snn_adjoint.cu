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
//
// Backward step t gathers only the newest adjoint plane, that of step t + 1,
// and spreads each synapse's term over the step it belongs to, t + 1 - d, in
// per-delay partial sums (a neuron's sum for step t is complete once step
// t + 1 has been gathered).  So the gather reads one plane of n_pop x M
// floats, and the slice of the source's own partition (most targets) is
// staged in shared memory.  Every segment's steps run as one CUDA graph
// whose kernels read the segment's first step from device memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "snn_internal.h"

using namespace snn;

namespace {

constexpr int kAThreads = 256;
constexpr int kBThreads = 1024;  // backward: one block per SM, up to 64 registers (32 warps hide latency)
constexpr int kBWarps = kBThreads / 32;
constexpr int kBGroups = 2;      // groups of 4 synapses per lane per batch (a run of 256 in one batch)
constexpr int kDWarps = 4;       // forward delivery: warps per spike
constexpr int kDUnroll = 4;
constexpr int kMaxPop = 8;
constexpr uint32_t kNoiseTag = 0xAD;

// A backward block's unit of work: sources j0..j1-1 of one partition, whose
// first n_stage neurons (from base) are staged for planes plane0, plane0+1.
struct BItem {
    uint32_t j0, j1, base, n_stage;
    uint32_t plane0, pad0, pad1, pad2;
};

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
    const unsigned long long *run;  // [M+1] first synapse of each neuron's run: the run its
                                    // level-2 entries tile (one segment per destination partition)
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
    float *hbuf;            // [2][n_pop][M] by step parity: G[pop k][b] * (adjoint of V_pre of k);
                            // a source of population b gathers plane b
    float *part;            // [S][M] partial sums of the gathered terms, by step slot (step mod S)
    int S;                  // step slots = largest delay
    const BItem *items;     // [n_items] backward work units
    int n_items, cap;       // staged neurons per plane (shared memory)
    const int *tb;          // first step of the running segment
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

// One step t = (segment start) + toff of the forward for every neuron
// (thread per neuron).  rec >= 0:
// record V_pre, flags and inputs in segment slot rec; count: add the spikes
// to the population counts and the raster.
template <int NP>
__global__ void __launch_bounds__(kAThreads) k_adj_update(const AdjDev a, int toff, int rec, int count)
{
    const int t = *a.tb + toff;
    __shared__ unsigned long long s_cnt[kMaxPop];
    if (threadIdx.x < kMaxPop) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int par = t & 1;
    const int slot = t % a.D;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.spk_n[par ^ 1] = 0;  // the next step's list
    for (long long k = (long long)blockIdx.x * kAThreads + threadIdx.x; k < a.M;
         k += (long long)gridDim.x * kAThreads) {
        // every load first: the neuron's ring row (NP int32, 8-byte aligned),
        // population, state, id
        int2 *rg = reinterpret_cast<int2 *>(a.ring + ((long long)slot * a.M + k) * NP);
        int32_t A[NP];
#pragma unroll
        for (int b = 0; b < NP / 2; ++b) {
            const int2 v = rg[b];
            A[2 * b] = v.x;
            A[2 * b + 1] = v.y;
        }
        const int p = a.pop[k];
        const uint8_t r = a.ref[k];
        const float v = a.V[k];
        const uint32_t g = a.gid ? a.gid[k] : (uint32_t)k;
#pragma unroll
        for (int b = 0; b < NP / 2; ++b) rg[b] = make_int2(0, 0);
        if (rec >= 0) {
            int2 *sa = reinterpret_cast<int2 *>(a.seg_A + ((long long)rec * a.M + k) * NP);
#pragma unroll
            for (int b = 0; b < NP / 2; ++b) sa[b] = make_int2(A[2 * b], A[2 * b + 1]);
        }
        float irec = __fmul_rn(a.G[p * NP], (float)A[0]);
#pragma unroll
        for (int b = 1; b < NP; ++b) irec = __fadd_rn(irec, __fmul_rn(a.G[p * NP + b], (float)A[b]));
        const float x1 = __fmul_rn(a.sigma, noise_of(a, g, (uint32_t)t));
        const float x2 = __fadd_rn(a.lam[p], x1);
        const float drv = __fmul_rn(a.w_ext, x2);
        const float I = __fadd_rn(irec, drv);
        const bool refr = r > 0;
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
    if (count && threadIdx.x < NP && s_cnt[threadIdx.x]) atomicAdd(&a.pop_cnt[threadIdx.x], s_cnt[threadIdx.x]);
}

// Delivery of step t's spikes through the routing tables: a spike's level-2
// entries tile its synapse run, which kDWarps warps share (a contiguous
// quarter each, kDUnroll loads per lane in flight); every weight is added
// to the ring slot of its delay, column = the source population.
__global__ void __launch_bounds__(kAThreads) k_adj_deliver(const AdjDev a, int toff)
{
    const int t = *a.tb + toff;
    const int par = t & 1;
    const unsigned int n = *(volatile unsigned int *)&a.spk_n[par];
    const int lane = threadIdx.x & 31;
    const unsigned int nw = (gridDim.x * kAThreads) >> 5;
    for (unsigned int wq = (blockIdx.x * kAThreads + threadIdx.x) >> 5; wq < n * kDWarps; wq += nw) {
        const uint32_t i = a.spk[(long long)par * a.M + wq / kDWarps];
        const int q = (int)(wq % kDWarps);
        const int pi = a.pop[i];
        const unsigned long long r0 = a.run[i], len = a.run[i + 1] - r0;
        const unsigned long long b0 = r0 + len * q / kDWarps, b1 = r0 + len * (q + 1) / kDWarps;
        for (unsigned long long x0 = b0 + lane; x0 < b1; x0 += 32 * kDUnroll) {
            uint32_t td[kDUnroll];
            int32_t w[kDUnroll];
#pragma unroll
            for (int u = 0; u < kDUnroll; ++u) {
                const unsigned long long x = x0 + 32ull * u;
                td[u] = x < b1 ? __ldg(a.syn_td + x) : 0u;
                w[u] = x < b1 ? (int32_t)__ldg(a.syn_w + x) : 0;
            }
#pragma unroll
            for (int u = 0; u < kDUnroll; ++u) {
                if (x0 + 32ull * u >= b1) break;
                int sl = t + (int)(td[u] >> kTgtBits) + 1;
                sl %= a.D;
                atomicAdd(&a.ring[((long long)sl * a.M + (td[u] & kTgtMask)) * a.n_pop + pi], w[u]);
            }
        }
    }
}

// A float sum kept as an unevaluated pair hi + lo (Dekker / Knuth two-sum):
// add() takes the exact product gd * x (two-product with one fused
// multiply-add) and keeps the rounding errors in lo, so hi + lo carries about
// 48 significant bits; flush() adds hi + lo in float64 and clears the pair.
// The float64 pipe of this GPU is slow, so the per-neuron terms stay in the
// float pipe.
struct FloatPairSum {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float gd, float x)
    {
        const float p = __fmul_rn(gd, x);
        const float q = __fmaf_rn(gd, x, -p);  // p + q == gd * x exactly
        const float s = __fadd_rn(hi, p);
        const float bp = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(err, q));
    }
    __device__ __forceinline__ void flush(double *dst)
    {
        const double v = (double)hi + (double)lo;
        if (v != 0.0) atomicAdd(dst, v);
        hi = lo = 0.0f;
    }
};

// One backward step t = (segment start) + toff, segment slot rec, for every
// neuron, a warp each.  The warp of source j walks j's synapse run (the
// transpose of the routed delivery) and takes, for every synapse (k, d),
// w * h_k(t + 1) from plane pop(j) of step t + 1: a term of j's input adjoint
// at step t + 1 - d.  The terms collect per lane and delay in shared memory,
// are summed over the warp and added to the partial sums of those steps;
// the sum of step t is then complete (d = 1 is the last term it gets) and
// gives j's adjoint recursion, its plane entries for step t and its
// parameter-gradient terms.  A block works on sources of one partition with
// that partition's slice of the two planes its sources read staged in
// shared memory; a warp's next source has its run bounds and first batch of
// synapses in flight while the current source finishes.
template <int NDL>
__global__ void __launch_bounds__(kBThreads, 1) k_adj_backward(const AdjDev a, int toff, int rec)
{
    extern __shared__ __align__(16) float bsm[];
    __shared__ double s_dG[kMaxPop * kMaxPop];
    __shared__ double s_dl[kMaxPop];
    const int t = *a.tb + toff;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long M = a.M;
    const int np = a.n_pop;
    float *hs = bsm;                                          // [2][cap]
    float *col = bsm + 2 * a.cap + warp * (NDL * 32) + lane;  // this lane's column, stride 32 per delay
    for (int x = threadIdx.x; x < kMaxPop * kMaxPop; x += kBThreads) s_dG[x] = 0.0;
    if (threadIdx.x < kMaxPop) s_dl[threadIdx.x] = 0.0;
#pragma unroll
    for (int dd = 0; dd < NDL; ++dd) col[dd * 32] = 0.0f;
    const float c = 0.0009765625f;
    const float *hn = a.hbuf + (size_t)((t + 1) & 1) * np * M;  // step t + 1
    float *ho = a.hbuf + (size_t)(t & 1) * np * M;              // step t
    // the lanes that hold the warp's sum of delay index dd = lane >> sh
    constexpr int sh = NDL == 8 ? 2 : 1;
    const int dd = lane >> sh;
    const bool holder = (lane & ((1 << sh) - 1)) == 0 && dd < a.S && t - dd >= 0;
    const int slot = (t - dd + a.S) % a.S;  // meaningful where holder
    FloatPairSum acc0, acc1;
    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
        const BItem it = a.items[item];
        __syncthreads();
        {
            const float *s0 = hn + (size_t)it.plane0 * M + it.base;
            const float *s1 = s0 + M;
            for (uint32_t x0 = threadIdx.x; x0 < it.n_stage; x0 += 4 * kBThreads) {
                float v0[4], v1[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t x = x0 + u * kBThreads;
                    v0[u] = x < it.n_stage ? s0[x] : 0.0f;
                    v1[u] = x < it.n_stage ? s1[x] : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t x = x0 + u * kBThreads;
                    if (x < it.n_stage) {
                        hs[x] = v0[u];
                        hs[a.cap + x] = v1[u];
                    }
                }
            }
        }
        __syncthreads();
        uint32_t j = it.j0 + warp;
        // the first source's run and batch.  A batch is kBGroups groups of 4
        // synapses per lane from the run's start rounded down to a multiple
        // of 4 (one 16-byte load of target words and one 8-byte load of
        // weights per group); weights outside the run count as 0.
        unsigned long long r0 = 0, r1 = 0;
        int pj = 0;
        if (j < it.j1) {
            r0 = a.run[j];
            r1 = a.run[j + 1];
            pj = a.pop[j];
        }
        uint4 tv[kBGroups];
        uint2 wv[kBGroups];
        auto load_batch = [&](unsigned long long g0, unsigned long long end) {
#pragma unroll
            for (int u = 0; u < kBGroups; ++u) {
                const unsigned long long e = g0 + 4ull * (lane + 32 * u);
                const bool in = e < end;
                tv[u] = in ? __ldg(reinterpret_cast<const uint4 *>(a.syn_td + e)) : make_uint4(0, 0, 0, 0);
                wv[u] = in ? __ldg(reinterpret_cast<const uint2 *>(a.syn_w + e)) : make_uint2(0, 0);
            }
        };
        load_batch(r0 & ~3ull, r1);
        for (; j < it.j1; j += kBWarps) {
            // the next source's run; this source's epilogue inputs
            const uint32_t jn = j + kBWarps;
            unsigned long long n0 = 0, n1 = 0;
            int pn = 0;
            if (jn < it.j1) {
                n0 = a.run[jn];
                n1 = a.run[jn + 1];
                pn = a.pop[jn];
            }
            const float pin = holder ? a.part[(size_t)slot * M + j] : 0.0f;
            const int32_t Ab = lane < np ? a.seg_A[((long long)rec * M + j) * np + lane] : 0;
            const float Gb = lane < np ? a.G[pj * np + lane] : 0.0f;
            uint8_t fl = 0;
            float vpre = 0.0f, gVj = 0.0f, dir = 0.0f;
            if (lane == 0) {
                fl = a.seg_flag[(long long)rec * M + j];
                vpre = a.seg_vpre[(long long)rec * M + j];
                gVj = a.gV[j];
                dir = a.direct[pj];
            }
            const float *hsp = hs + (pj & 1) * a.cap;
            const float *hgp = hn + (size_t)pj * M;
            for (unsigned long long g0 = r0 & ~3ull;;) {
#pragma unroll
                for (int u = 0; u < kBGroups; ++u) {
                    const unsigned long long e = g0 + 4ull * (lane + 32 * u);
                    const uint32_t tdu[4] = {tv[u].x, tv[u].y, tv[u].z, tv[u].w};
                    const int32_t wu[4] = {(int32_t)(int16_t)(wv[u].x & 0xFFFFu), (int32_t)(int16_t)(wv[u].x >> 16),
                                           (int32_t)(int16_t)(wv[u].y & 0xFFFFu), (int32_t)(int16_t)(wv[u].y >> 16)};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const bool in = e + i >= r0 && e + i < r1;
                        const uint32_t k = tdu[i] & kTgtMask;
                        const uint32_t rel = k - it.base;
                        const float hk = rel < it.n_stage ? hsp[rel] : __ldg(hgp + k);
                        float *cp = col + (tdu[i] >> kTgtBits) * 32;
                        *cp = __fadd_rn(*cp, __fmul_rn((float)(in ? wu[i] : 0), hk));
                    }
                }
                g0 += 4ull * 32 * kBGroups;
                if (g0 >= r1) break;
                load_batch(g0, r1);
            }
            // the next source's first batch, in flight during the epilogue
            load_batch(n0 & ~3ull, n1);
            // the warp's sum per delay: halve the delays held per lane over
            // lane bits 4, 3, ..., then sum the rest of the warp
            float r[NDL];
#pragma unroll
            for (int x = 0; x < NDL; ++x) {
                r[x] = col[x * 32];
                col[x * 32] = 0.0f;
            }
#pragma unroll
            for (int half = NDL / 2, sft = 16; half >= 1; half >>= 1, sft >>= 1) {
                const bool up = (lane & sft) != 0;
#pragma unroll
                for (int q = 0; q < half; ++q) {
                    const float keep = up ? r[half + q] : r[q];
                    const float give = up ? r[q] : r[half + q];
                    r[q] = __fadd_rn(keep, __shfl_xor_sync(0xFFFFFFFFu, give, sft));
                }
            }
#pragma unroll
            for (int sft = (1 << sh) >> 1; sft > 0; sft >>= 1)
                r[0] = __fadd_rn(r[0], __shfl_xor_sync(0xFFFFFFFFu, r[0], sft));
            const float sum = __fadd_rn(pin, r[0]);
            // step t's slot is consumed (and cleared for step t - S); the
            // earlier steps' slots take their terms
            if (holder) a.part[(size_t)slot * M + j] = dd == 0 ? 0.0f : sum;
            float gvp = 0.0f;
            if (lane == 0 && !(fl & 2)) {
                const float gS = __fadd_rn(dir, __fmul_rn(c, sum));
                const float x = __fsub_rn(vpre, a.v_th);
                const float den = __fadd_rn(1.0f, __fmul_rn(a.beta, fabsf(x)));
                const float sg = __frcp_rn(__fmul_rn(den, den));
                const float keep = (fl & 1) ? 0.0f : gVj;
                gvp = __fadd_rn(keep, __fmul_rn(gS, sg));
            }
            gvp = __shfl_sync(0xFFFFFFFFu, gvp, 0);
            // the products each source population gathers at step t - 1
            if (lane < np) ho[(size_t)lane * M + j] = __fmul_rn(Gb, gvp);
            if (lane == 0) a.gV[j] = __fmul_rn(a.alpha, gvp);
            // parameter-gradient terms gvp * c * A_jb (lane b) and gvp * c * w_ext
            // (lane 31): exact products, summed per warp as float pairs
            if (gvp != 0.0f && (lane < np || lane == 31)) {
                const int32_t xi = lane < np ? Ab : 0;
                if (lane == 31 || (xi < (1 << 24) && xi > -(1 << 24))) {
                    const float gd = __fmul_rn(gvp, c);
                    const float x = lane == 31 ? a.w_ext : (float)xi;
                    if (pj & 1) acc1.add(gd, x);
                    else acc0.add(gd, x);
                } else {
                    atomicAdd(&s_dG[pj * np + lane], (double)gvp * (double)c * (double)xi);
                }
            }
            r0 = n0;
            r1 = n1;
            pj = pn;
        }
        // the warp's sums of this item (populations plane0, plane0 + 1)
        if (lane < np) {
            acc0.flush(&s_dG[it.plane0 * np + lane]);
            acc1.flush(&s_dG[(it.plane0 + 1) * np + lane]);
        } else if (lane == 31) {
            acc0.flush(&s_dl[it.plane0]);
            acc1.flush(&s_dl[it.plane0 + 1]);
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < np * np; x += kBThreads)
        if (s_dG[x] != 0.0) atomicAdd(&a.dG[x], s_dG[x]);
    if (threadIdx.x < np && s_dl[threadIdx.x] != 0.0) atomicAdd(&a.dlam[threadIdx.x], s_dl[threadIdx.x]);
}

__global__ void k_adj_set_step(int *tb, int t)
{
    *tb = t;
}

struct Region {
    size_t off = 0, bytes = 0;
};

struct ALayout {
    Region V, ref, ring, pop, gid, run, syn_td, syn_w, spk, spk_n, pop_cnt, raster, raster_n;
    Region G, lam, seg_vpre, seg_flag, seg_A, hbuf, part, items, tb, gV, direct, dG, dlam;
    Region ck_V, ck_ref, ck_ring;  // [n_ckpt] checkpoints
    size_t total = 0;
    int D = 2, n_pop = 2, n_ckpt = 1, S = 1, n_items = 1;
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

int sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        sms = 0;
    cudaGetLastError();
    return std::max(1, sms);
}

// The backward's work units: every partition cut into chunks of sources,
// about one chunk per SM in all (at least one per partition).  Returns the
// count; fills `out` when given (n_stage is capped at create).
int backward_items(const snn_routing *rt, std::vector<BItem> *out)
{
    const int sms = sm_count();
    const int64_t M = rt->M;
    const int32_t s = rt->P / rt->n_vn;
    int n = 0;
    for (int32_t ip = 0; ip < rt->P; ++ip) {
        const int64_t a = rt->pbase[ip], b = rt->pbase[ip + 1];
        if (b <= a) continue;
        const int64_t c = std::max<int64_t>(1, (int64_t)sms * (b - a) / std::max<int64_t>(1, M));
        for (int64_t x = 0; x < c; ++x) {
            if (out) {
                BItem it;
                std::memset(&it, 0, sizeof(it));
                it.j0 = (uint32_t)(a + (b - a) * x / c);
                it.j1 = (uint32_t)(a + (b - a) * (x + 1) / c);
                it.base = (uint32_t)a;
                it.n_stage = (uint32_t)(b - a);
                it.plane0 = (uint32_t)(2 * (ip / s));
                out->push_back(it);
            }
            ++n;
        }
    }
    return std::max(1, n);
}

int adj_layout(const snn_routing *rt, const snn_sim_params *p, const snn_adjoint_params *ap, ALayout &L)
{
    const int64_t M = rt->M, E = rt->E;
    L = ALayout();
    L.D = rt->max_delay + 1;
    L.S = std::max(1, (int)rt->max_delay);
    L.n_items = backward_items(rt, nullptr);
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
    aplace(L, L.run, sizeof(unsigned long long) * (M + 1));
    // the backward reads synapses in aligned groups of 4: up to 3 past the
    // end, zero-filled (target 0, delay 1, weight 0)
    aplace(L, L.syn_td, sizeof(uint32_t) * (E + 4));
    aplace(L, L.syn_w, sizeof(int16_t) * (E + 4));
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
    aplace(L, L.hbuf, sizeof(float) * 2 * (size_t)L.n_pop * M);
    aplace(L, L.part, sizeof(float) * (size_t)L.S * M);
    aplace(L, L.items, sizeof(BItem) * (size_t)L.n_items);
    aplace(L, L.tb, sizeof(int));
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
    cudaStream_t cap_stream = nullptr;  // graph capture
    unsigned grid_n = 1, grid_w = 1, grid_b = 1;
    int ndl = 8;                        // delay columns of the backward (8 or 16)
    size_t bsmem = 0;                   // its dynamic shared memory
    std::vector<double> pop_size;
    bool have_forward = false;
    // one graph per (kind, segment length): 0 forward counted, 1 forward
    // recorded, 2 backward
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;

    ~snn_adjoint()
    {
        for (auto &g : graphs) cudaGraphExecDestroy(g.second);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
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
    d.run = (const unsigned long long *)(w + L.run.off);
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
    d.hbuf = (float *)(w + L.hbuf.off);
    d.part = (float *)(w + L.part.off);
    d.S = L.S;
    d.items = (const BItem *)(w + L.items.off);
    d.tb = (const int *)(w + L.tb.off);
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
    // each neuron's level-2 entries tile its synapse run (one segment per
    // destination partition, partitions ascending): check, keep the bounds
    for (int64_t i = 0; i < M; ++i) {
        uint64_t at = (uint64_t)rt->csr[i];
        for (uint32_t f = rt->l1_l2[rt->l1_ptr[i]]; f < rt->l1_l2[rt->l1_ptr[i + 1]]; ++f) {
            if ((rt->l2[f].off & kOffMask) != at) {
                delete a;
                return SNN_E_STATE;
            }
            at += rt->l2[f].len;
        }
        if (at != (uint64_t)rt->csr[i + 1]) {
            delete a;
            return SNN_E_STATE;
        }
    }
    auto up = [&](const Region &r, const void *src) -> cudaError_t {
        return r.bytes ? cudaMemcpy(w + r.off, src, r.bytes, cudaMemcpyHostToDevice) : cudaSuccess;
    };
    if (up(L.pop, pop.data()) || up(L.run, rt->csr.data()) ||
        cudaMemset(w + L.syn_td.off, 0, L.syn_td.bytes) || cudaMemset(w + L.syn_w.off, 0, L.syn_w.bytes) ||
        cudaMemcpy(w + L.syn_td.off, rt->syn_td.data(), sizeof(uint32_t) * rt->E, cudaMemcpyHostToDevice) ||
        cudaMemcpy(w + L.syn_w.off, rt->syn_w.data(), sizeof(int16_t) * rt->E, cudaMemcpyHostToDevice) ||
        (!rt->identity && up(L.gid, rt->perm_inv.data()))) {
        delete a;
        return SNN_E_CUDA;
    }
    const int sms = sm_count();
    a->grid_n = (unsigned)std::max<int64_t>(1, std::min<int64_t>((M + kAThreads - 1) / kAThreads, 65535));
    a->grid_w = (unsigned)std::max(1, sms * 8);
    // backward: the delay columns, then as much of each partition's two
    // planes as shared memory holds
    {
        std::vector<BItem> items;
        backward_items(rt, &items);
        a->ndl = rt->max_delay <= 8 ? 8 : 16;
        int dev = 0, optin = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
            delete a;
            return SNN_E_CUDA;
        }
        // shared memory: the delay columns, then as much of a partition's two
        // planes as fits
        const size_t cols = sizeof(float) * (size_t)kBWarps * a->ndl * 32;
        const size_t fixed = sizeof(double) * (kMaxPop * kMaxPop + kMaxPop) + 1024;
        int64_t cap = 0;
        if ((size_t)optin > cols + fixed) cap = (int64_t)(((size_t)optin - cols - fixed) / (2 * sizeof(float))) & ~3ll;
        int64_t widest = 0;
        for (const BItem &it : items) widest = std::max<int64_t>(widest, it.n_stage);
        cap = std::min<int64_t>(cap, (widest + 3) & ~3ll);
        for (BItem &it : items) it.n_stage = (uint32_t)std::min<int64_t>(it.n_stage, cap);
        d.cap = (int)cap;
        d.n_items = (int)items.size();
        a->bsmem = cols + 2 * sizeof(float) * (size_t)cap;
        cudaError_t e = a->ndl == 8 ? cudaFuncSetAttribute(k_adj_backward<8>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a->bsmem)
                                    : cudaFuncSetAttribute(k_adj_backward<16>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a->bsmem);
        if (e != cudaSuccess || (int)items.size() != L.n_items ||
            cudaMemcpy(w + L.items.off, items.data(), sizeof(BItem) * items.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaStreamCreateWithFlags(&a->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete a;
            return SNN_E_CUDA;
        }
        a->grid_b = (unsigned)std::min(d.n_items, sms);
    }
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

// The steps of one segment of `len` steps from the step base in device
// memory: kind 0 the counted forward, 1 the recorded forward, 2 the
// backward (last step first).  Captured once per (kind, len) and replayed.
static int adj_segment(snn_adjoint *a, int kind, int len)
{
    cudaGraphExec_t &ex = a->graphs[std::make_pair(kind, len)];
    if (!ex) {
        cudaStream_t cs = a->cap_stream;
        ACK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        for (int i = 0; i < len; ++i) {
            if (kind == 2) {
                const int toff = len - 1 - i;
                if (a->ndl == 8)
                    k_adj_backward<8><<<a->grid_b, kBThreads, a->bsmem, cs>>>(a->dev, toff, toff);
                else
                    k_adj_backward<16><<<a->grid_b, kBThreads, a->bsmem, cs>>>(a->dev, toff, toff);
            } else {
                const int rec = kind == 1 ? i : -1, cnt = kind == 0 ? 1 : 0;
                switch (a->dev.n_pop) {
                case 2: k_adj_update<2><<<a->grid_n, kAThreads, 0, cs>>>(a->dev, i, rec, cnt); break;
                case 4: k_adj_update<4><<<a->grid_n, kAThreads, 0, cs>>>(a->dev, i, rec, cnt); break;
                case 6: k_adj_update<6><<<a->grid_n, kAThreads, 0, cs>>>(a->dev, i, rec, cnt); break;
                default: k_adj_update<8><<<a->grid_n, kAThreads, 0, cs>>>(a->dev, i, rec, cnt); break;
                }
                k_adj_deliver<<<a->grid_w, kAThreads, 0, cs>>>(a->dev, i);
            }
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (e != cudaSuccess || !g) {
            a->graphs.erase(std::make_pair(kind, len));
            return SNN_E_CUDA;
        }
        const cudaError_t e2 = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) {
            a->graphs.erase(std::make_pair(kind, len));
            return SNN_E_CUDA;
        }
    }
    ACK(cudaGraphLaunch(ex, a->stream));
    return SNN_OK;
}

static int adj_set_step(snn_adjoint *a, int t)
{
    k_adj_set_step<<<1, 1, 0, a->stream>>>((int *)a->dev.tb, t);
    ACK(cudaGetLastError());
    return SNN_OK;
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
    for (int t0 = 0; t0 < T; t0 += K) {
        const int c = t0 / K;
        ACK(cudaMemcpyAsync(w + L.ck_V.off + (size_t)c * sizeof(float) * M, w + L.V.off, L.V.bytes,
                            cudaMemcpyDeviceToDevice, st));
        ACK(cudaMemcpyAsync(w + L.ck_ref.off + (size_t)c * M, w + L.ref.off, L.ref.bytes, cudaMemcpyDeviceToDevice,
                            st));
        ACK(cudaMemcpyAsync(w + L.ck_ring.off + (size_t)c * ring_b, w + L.ring.off, ring_b, cudaMemcpyDeviceToDevice,
                            st));
        if ((rc = adj_set_step(a, t0)) != SNN_OK || (rc = adj_segment(a, 0, std::min(K, T - t0))) != SNN_OK)
            return rc;
    }
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
    ACK(cudaMemsetAsync(w + L.hbuf.off, 0, L.hbuf.bytes, st));
    ACK(cudaMemsetAsync(w + L.part.off, 0, L.part.bytes, st));
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
        int rc = adj_set_step(a, t0);
        if (rc == SNN_OK) rc = adj_segment(a, 1, t1 - t0);
        if (rc == SNN_OK) rc = adj_segment(a, 2, t1 - t0);
        if (rc != SNN_OK) return rc;
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
