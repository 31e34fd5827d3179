// Step kernels of one simulation step t (sm_103a), included by snn_sim.cu.
//
// The routing is the paper's two-level route (arXiv 2205.07125, Sec. IV.B);
// the neuron model is LIF (Table I); the arithmetic follows the library's
// documented readings (include/snn.h).  A step has two phases:
//   update_route  a1 consume ring slot t mod D, Poisson drive (Philox4x32-10,
//                    inverse CDF); a2 FP32 LIF update + threshold (no FMA,
//                    fixed order); a3 warp-scan / block-scan compaction of
//                    the spikes into a block buffer and the step's spike
//                    list (4 neurons per thread with 16-byte loads).  The
//                    block that found the spikes routes them, one warp each:
//                 a4 level-1 bucketing: the spike is appended to the bucket of
//                    every destination VN in its level-1 row (one entry per
//                    VN: deduplicated);
//                 a5 level-2 relay expansion: every (spike, VN) entry becomes
//                    an inbox entry of each partition of that VN holding
//                    targets; long segments are also queued as 128-synapse
//                    pieces.
//   deliver       a6 every block takes the inbox prefix sums; pieces of long
//                    segments go one warp per piece with 4 streaming loads in
//                    flight per lane; short segments (<= 8 synapses) are
//                    walked by one lane per inbox entry; every synapse adds
//                    its int16 weight with a 32-bit reduction into
//                    ring[(t+d) mod D][target].  Block 0 closes the step's
//                    bookkeeping (raster offsets, counters).
// The ring has D = max delay + 1 slots, so the slot consumed at step t is
// never written by the deliveries of step t.  Per-step counters are kept
// twice, by step parity: step t fills parity t & 1 and clears the other
// one, which step t - 1 used and step t + 1 will fill, so no block has to
// close a phase.
//
// Two ways to run the phases: k_persist, one cooperative launch for T steps
// with a grid barrier after each phase (bounded waits), and the CUDA-graph
// path, k_update / k_deliver per step with programmatic dependent launch.
#pragma once

#include <cuda_runtime.h>

#include "snn_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPTab = 32;
constexpr int kSpkBuf = 1024;   // spikes a block buffers before flushing
constexpr int kShortSeg = 8;    // segments up to this length are walked by one lane
constexpr int kPiece = 128;     // longer segments are cut into pieces of this many synapses
constexpr int kPreMax = 4097;   // staged prefix entries (P <= 4096)
// Per-VN and per-partition fill counters sit one 128-byte line apart, so
// that their atomics spread over L2 slices instead of queueing on one line.
constexpr int kCntStride = 32;

// status bits
constexpr uint32_t kStBucket = 1u, kStInbox = 2u, kStRaster = 4u, kStTimeout = 8u;

// counter slots
enum { C_STEPS = 0, C_SPIKES, C_EVENTS, C_L1_LOCAL, C_L1_XVN, C_L2_BASE /* + cls (4) */, C_N = 16 };

// The atomically updated words each own a 128-byte line: blocks spinning on
// the barrier generation must not share a line with the hot counters.
struct Ctrl {
    long long t;              // next step to run
    long long head[2];        // raster write head at the start of a step, by step parity
    long long rec_steps;      // steps whose raster offsets are valid
    unsigned int status;
    int rec_on;
    alignas(128) unsigned int S_acc[2];    // spikes of a step, by parity
    alignas(128) unsigned int n_piece[2];  // long-segment pieces queued in a step, by parity
    alignas(128) unsigned int bar_count;   // grid barrier arrivals (k_persist)
    alignas(128) unsigned int bar_gen;     // grid barrier generation (k_persist)
};

struct __align__(16) DevL2 {
    unsigned long long off;
    unsigned int len;
    unsigned short q;
    unsigned char cls;
    unsigned char pad;
};

struct Dev {
    // state
    float *V;
    uint8_t *ref;
    int32_t *ring;
    const uint32_t *gid;  // internal -> global id (nullptr when identical)
    const uint16_t *src_vn;
    // synapses and routing tables
    const uint32_t *syn_td;
    const int16_t *syn_w;
    const uint32_t *l1_ptr;
    const uint16_t *l1_vn;
    const uint32_t *l1_l2;
    const DevL2 *l2;
    // exchange buffers
    uint32_t *bucket;
    const unsigned long long *bucket_base;
    const uint32_t *bucket_capv;
    uint32_t *bucket_cnt;       // [2][n_vn * kCntStride], by step parity
    unsigned long long *inbox;
    const unsigned long long *inbox_base;
    const uint32_t *inbox_capv;
    uint32_t *inbox_cnt;        // [2][P * kCntStride], by step parity
    unsigned long long *piece;  // pieces of long segments: offset << 8 | length
    unsigned int piece_cap;
    // records
    uint32_t *spk;
    long long *raster_off;
    unsigned long long *hash;
    int32_t *cur_rec;
    unsigned long long *counters;
    unsigned long long *phase_ns;  // [2] summed phase times of k_persist (profiling)
    Ctrl *ctrl;
    // scalars
    long long M;
    int P, n_vn, D;
    float alpha, e_l, v_th, v_reset;
    int t_ref, w_ext, i_bias, th_fin;
    uint32_t key0, key1;
    long long raster_cap, raster_steps, hash_steps;
    int cur_every, cur_slots;
    uint32_t th32[kPTab];   // finite Poisson thresholds (the closing 2^32 is implied)
};

__device__ __forceinline__ uint32_t *bucket_cnt_of(const Dev &d, int p)
{
    return d.bucket_cnt + (size_t)p * (size_t)d.n_vn * kCntStride;
}

__device__ __forceinline__ uint32_t *inbox_cnt_of(const Dev &d, int p)
{
    return d.inbox_cnt + (size_t)p * (size_t)d.P * kCntStride;
}

// Philox4x32-10 block of counter (c0, c1, 0, 0): the drive word of neuron j
// at step t is word (j mod 4) of the block (j div 4, t).
__device__ __forceinline__ uint4 philox4(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1)
{
    uint32_t x0 = c0, x1 = c1, x2 = 0u, x3 = 0u;
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

__device__ __forceinline__ uint32_t uint4_word(const uint4 &w, uint32_t k)
{
    return k == 0 ? w.x : k == 1 ? w.y : k == 2 ? w.z : w.w;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Programmatic dependent launch (graph path): wait for the grid before this
// one (all of its writes visible) before touching shared state, and let the
// next grid be scheduled early.  Both are no-ops for a plain launch.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Grid-wide barrier of k_persist (all blocks co-resident: cooperative
// launch).  The wait is bounded: past `limit_ns` the block records
// kStTimeout and gives up.  Returns false when this or any other block gave
// up, after which every block leaves the kernel.
__device__ __forceinline__ bool grid_sync(Ctrl *c, unsigned long long limit_ns, bool arrive = true)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = &c->bar_gen;
        const unsigned int g = *gen;
        __threadfence();
        int ok = 1;
        if (arrive && atomicAdd(&c->bar_count, 1u) == gridDim.x - 1) {
            c->bar_count = 0;
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else {
            const unsigned long long deadline = global_ns() + limit_ns;
            while (*gen == g) {
                if (global_ns() > deadline) {
                    atomicOr(&c->status, kStTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        if (*(volatile unsigned int *)&c->status & kStTimeout) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Index k with pre[k] <= x < pre[k+1] (pre nondecreasing, pre[0] = 0 <= x < pre[n]).
__device__ __forceinline__ int prefix_find(const uint32_t *pre, int n, uint32_t x)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Exclusive prefix of min(cnt[k * kCntStride], cap[k]) into pre[0..n] by one block.
__device__ __forceinline__ void block_prefix(const uint32_t *cnt, const uint32_t *cap, uint32_t *pre, int n)
{
    __shared__ uint32_t s_carry;
    __shared__ uint32_t s_w[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int b = 0; b < n; b += kThreads) {
        const int k = b + threadIdx.x;
        const uint32_t v = k < n ? min(__ldcg(cnt + (size_t)k * kCntStride), cap[k]) : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[wid] = x;
        __syncthreads();
        uint32_t wb = 0;
        for (int w = 0; w < wid; ++w) wb += s_w[w];
        if (k < n) pre[k] = s_carry + wb + x - v;
        __syncthreads();
        if (threadIdx.x == kThreads - 1) s_carry += wb + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) pre[n] = s_carry;
    __syncthreads();
}

// a1 + a2 for one neuron: returns true on a spike.
// th: the Poisson thresholds staged in shared memory (lanes index them
// divergently, which the kernel-parameter bank would serialise).
// u: the neuron's drive word.
__device__ __forceinline__ bool lif_neuron(const Dev &d, const uint32_t *th, uint32_t u, int32_t irec, float &v,
                                           uint32_t &r)
{
    int k = 0;
    while (k < d.th_fin && u >= th[k]) ++k;
    const int32_t I = (int32_t)((uint32_t)irec + (uint32_t)k * (uint32_t)d.w_ext + (uint32_t)d.i_bias);
    if (r > 0) {
        r -= 1;
        v = d.v_reset;
        return false;
    }
    const float uu = __fsub_rn(v, d.e_l);
    const float au = __fmul_rn(d.alpha, uu);
    v = __fadd_rn(d.e_l, au);
    const float x = __fmul_rn(__int2float_rn(I), 0.0009765625f);
    v = __fadd_rn(v, x);
    if (v >= d.v_th) {
        v = d.v_reset;
        r = (uint32_t)d.t_ref;
        return true;
    }
    return false;
}

// Per-thread tallies of the routing done by one block.
struct RouteTally {
    unsigned int l1_loc = 0, l1_xvn = 0, ovf = 0;
    unsigned int cls[4] = {0, 0, 0, 0};
};

// a4 + a5 for the n spikes buffered in s_spk, one warp per spike (all
// threads of the block call this); counters of step parity p.
__device__ __forceinline__ void route_spikes(const Dev &d, int p, const uint32_t *s_spk, unsigned int n,
                                             RouteTally &rt)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t *bcnt = bucket_cnt_of(d, p);
    uint32_t *icnt = inbox_cnt_of(d, p);
    for (unsigned int s = wid; s < n; s += kThreads / 32) {
        const uint32_t i = s_spk[s];
        const uint16_t h = d.src_vn[i];
        const uint32_t e0 = d.l1_ptr[i], e1 = d.l1_ptr[i + 1];
        // a4: one level-1 entry per destination VN, appended to that VN's bucket
        for (uint32_t e = e0 + lane; e < e1; e += 32u) {
            const uint16_t g = d.l1_vn[e];
            const unsigned int pos = atomicAdd(&bcnt[(int)g * kCntStride], 1u);
            if (pos < d.bucket_capv[g]) d.bucket[d.bucket_base[g] + pos] = e;
            else rt.ovf |= kStBucket;
            if (g == h) ++rt.l1_loc;
            else ++rt.l1_xvn;
        }
        // a5: the relay of each destination VN expands the spike's entry into
        // the inboxes of the VN's partitions that hold targets; the level-2
        // rows of one spike's VNs are contiguous
        const uint32_t f0 = d.l1_l2[e0], f1 = d.l1_l2[e1];
        for (uint32_t fb = f0; fb < f1; fb += 32u) {
            const uint32_t f = fb + lane;
            DevL2 l;
            l.off = 0;
            l.len = 0;
            l.q = 0;
            if (f < f1) l = d.l2[f];
            // long segments are also cut into pieces for an even delivery;
            // their reservation is issued next to the inbox one
            const unsigned int np = l.len > (unsigned int)kShortSeg ? (l.len + kPiece - 1) / kPiece : 0u;
            unsigned int incl = np;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned int ptot = __shfl_sync(0xFFFFFFFFu, incl, 31);
            unsigned int pos = 0, pb = 0;
            if (f < f1) pos = atomicAdd(&icnt[(int)l.q * kCntStride], 1u);
            if (ptot && lane == 0) pb = atomicAdd(&d.ctrl->n_piece[p], ptot);
            if (f < f1) {
                if (pos < d.inbox_capv[l.q])
                    d.inbox[d.inbox_base[l.q] + pos] = (l.off << kLenBits) | (unsigned long long)l.len;
                else
                    rt.ovf |= kStInbox;
                // per-class tallies without a dynamically indexed (local-memory) array
                rt.cls[0] += l.cls == 0;
                rt.cls[1] += l.cls == 1;
                rt.cls[2] += l.cls == 2;
                rt.cls[3] += l.cls == 3;
            }
            if (ptot) {
                pb = __shfl_sync(0xFFFFFFFFu, pb, 0) + incl - np;
                for (unsigned int k = 0; k < np; ++k, ++pb) {
                    const unsigned int len = min((unsigned int)kPiece, l.len - k * kPiece);
                    if (pb < d.piece_cap) d.piece[pb] = ((l.off + (unsigned long long)k * kPiece) << 8) | len;
                    else rt.ovf |= kStInbox;
                }
            }
        }
    }
}

// Route the block's buffered spikes and append them to the step's spike
// list (all threads call).
__device__ __forceinline__ void flush_spikes(const Dev &d, int p, long long head, uint32_t *s_spk,
                                             unsigned int &s_n, unsigned int &s_gbase, int &s_routed,
                                             RouteTally &rt)
{
    __syncthreads();
    const unsigned int n = s_n;
    if (n == 0) return;
    route_spikes(d, p, s_spk, n, rt);
    if (threadIdx.x == 0) {
        s_gbase = atomicAdd(&d.ctrl->S_acc[p], n);
        s_routed = 1;
    }
    __syncthreads();
    const unsigned int gb = s_gbase;
    for (unsigned int k = threadIdx.x; k < n; k += kThreads) d.spk[head + gb + k] = s_spk[k];
    __syncthreads();
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
}

// ---------------------------------------------------------------- a1-a5
template <bool VEC>
__device__ __forceinline__ void update_route(const Dev &d, long long t)
{
    __shared__ uint32_t s_spk[kSpkBuf];
    __shared__ unsigned int s_wsum[kThreads / 32];
    __shared__ unsigned int s_n, s_tot, s_gbase;
    __shared__ int s_flush, s_routed;
    __shared__ unsigned long long s_h[2][kThreads / 32];
    __shared__ unsigned int s_tally[kThreads / 32][6];
    __shared__ uint32_t s_th[kPTab];

    Ctrl *c = d.ctrl;
    const int p = (int)(t & 1);
    const long long head = c->head[p];
    const int slot = (int)(t % d.D);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool do_hash = t < d.hash_steps;
    const bool do_cur = d.cur_every > 0 && (t % d.cur_every) == 0 && (t / d.cur_every) < d.cur_slots;
    int32_t *ring = d.ring + (long long)slot * d.M;
    int32_t *cur = do_cur ? d.cur_rec + (t / d.cur_every) * d.M : nullptr;
    constexpr int NPT = VEC ? 4 : 1;
    const long long nitem = VEC ? d.M / 4 : d.M;
    if (blockIdx.x == 0) {
        // clear the other parity: step t - 1 is done with it, step t + 1 fills it
        uint32_t *b1 = bucket_cnt_of(d, p ^ 1), *i1 = inbox_cnt_of(d, p ^ 1);
        for (int x = threadIdx.x; x < d.n_vn; x += kThreads) b1[x * kCntStride] = 0;
        for (int x = threadIdx.x; x < d.P; x += kThreads) i1[x * kCntStride] = 0;
        if (threadIdx.x == 0) {
            c->S_acc[p ^ 1] = 0;
            c->n_piece[p ^ 1] = 0;
        }
    }
    if (threadIdx.x < kPTab) s_th[threadIdx.x] = d.th32[threadIdx.x];
    if (threadIdx.x == 0) {
        s_n = 0;
        s_routed = 0;
    }
    __syncthreads();

    RouteTally rt;
    unsigned long long hc = 0, hv = 0;
    for (long long b0 = (long long)blockIdx.x * kThreads; b0 < nitem; b0 += (long long)gridDim.x * kThreads) {
        const long long q = b0 + threadIdx.x;
        const long long j0 = q * NPT;
        unsigned int m = 0;
        if (q < nitem) {
            float vv[NPT];
            int32_t ii[NPT];
            uint32_t r4;
            if constexpr (VEC) {
                const float4 v4 = *reinterpret_cast<const float4 *>(d.V + j0);
                const int4 i4 = *reinterpret_cast<const int4 *>(ring + j0);
                r4 = *reinterpret_cast<const uint32_t *>(d.ref + j0);
                *reinterpret_cast<int4 *>(ring + j0) = make_int4(0, 0, 0, 0);
                if (cur) *reinterpret_cast<int4 *>(cur + j0) = i4;
                vv[0] = v4.x;
                vv[1] = v4.y;
                vv[2] = v4.z;
                vv[3] = v4.w;
                ii[0] = i4.x;
                ii[1] = i4.y;
                ii[2] = i4.z;
                ii[3] = i4.w;
            } else {
                vv[0] = d.V[j0];
                ii[0] = ring[j0];
                r4 = d.ref[j0];
                ring[j0] = 0;
                if (cur) cur[j0] = ii[0];
            }
            uint32_t r_out = 0;
#pragma unroll
            // one Philox block serves the four neurons of a quad in the
            // global order; a reordering map needs a block per neuron
            uint4 wq = make_uint4(0u, 0u, 0u, 0u);
            if (VEC && !d.gid) wq = philox4(d.key0, d.key1, (uint32_t)(j0 >> 2), (uint32_t)t);
            for (int k = 0; k < NPT; ++k) {
                const uint32_t g = d.gid ? d.gid[j0 + k] : (uint32_t)(j0 + k);
                uint32_t u;
                if (VEC && !d.gid) u = uint4_word(wq, (uint32_t)k);
                else u = uint4_word(philox4(d.key0, d.key1, g >> 2, (uint32_t)t), g & 3u);
                uint32_t r = (r4 >> (8 * k)) & 0xFFu;
                if (lif_neuron(d, s_th, u, ii[k], vv[k], r)) m |= 1u << k;
                r_out |= r << (8 * k);
                if (do_hash) {
                    hc += mix64(((unsigned long long)g << 32) | (uint32_t)ii[k]);
                    hv += mix64(((unsigned long long)g << 32) | __float_as_uint(vv[k]));
                }
            }
            if constexpr (VEC) {
                *reinterpret_cast<float4 *>(d.V + j0) = make_float4(vv[0], vv[1], vv[2], vv[3]);
                *reinterpret_cast<uint32_t *>(d.ref + j0) = r_out;
            } else {
                d.V[j0] = vv[0];
                d.ref[j0] = (uint8_t)r_out;
            }
        }
        // a3: compaction of this pass (blocks without spikes skip it)
        const unsigned int cnt = __popc(m);
        if (__syncthreads_or(cnt)) {
            unsigned int x = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_wsum[wid] = x;
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned int tot = 0;
                for (int w = 0; w < kThreads / 32; ++w) {
                    const unsigned int cw = s_wsum[w];
                    s_wsum[w] = tot;
                    tot += cw;
                }
                s_tot = tot;
                s_flush = (s_n + tot > (unsigned int)kSpkBuf);
            }
            __syncthreads();
            if (s_flush) flush_spikes(d, p, head, s_spk, s_n, s_gbase, s_routed, rt);
            unsigned int pos = s_n + s_wsum[wid] + x - cnt;
            for (unsigned int mm = m; mm; mm &= mm - 1u) s_spk[pos++] = (uint32_t)(j0 + __ffs(mm) - 1);
            __syncthreads();
            if (threadIdx.x == 0) s_n += s_tot;
        }
    }
    flush_spikes(d, p, head, s_spk, s_n, s_gbase, s_routed, rt);
    if (do_hash) {
        hc = warp_sum(hc);
        hv = warp_sum(hv);
        if (lane == 0) {
            s_h[0][wid] = hc;
            s_h[1][wid] = hv;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long a = 0, b = 0;
            for (int w = 0; w < kThreads / 32; ++w) {
                a += s_h[0][w];
                b += s_h[1][w];
            }
            atomicAdd(&d.hash[2 * t], a);
            atomicAdd(&d.hash[2 * t + 1], b);
        }
    }
    __syncthreads();
    if (s_routed) {
        // message tallies of the routed spikes
        unsigned int v[6] = {rt.l1_loc, rt.l1_xvn, rt.cls[0], rt.cls[1], rt.cls[2], rt.cls[3]};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            v[k] = warp_sum(v[k]);
            if (lane == 0) s_tally[wid][k] = v[k];
        }
        if (rt.ovf) atomicOr(&c->status, rt.ovf);
        __syncthreads();
        if (threadIdx.x < 6) {
            unsigned long long a = 0;
            for (int w = 0; w < kThreads / 32; ++w) a += s_tally[w][threadIdx.x];
            // slots C_L1_LOCAL, C_L1_XVN, C_L2_BASE + 0..3 are consecutive
            if (a) atomicAdd(&d.counters[C_L1_LOCAL + threadIdx.x], a);
        }
    }
}

__device__ __forceinline__ void deliver_one(const Dev &d, int tm, unsigned long long o)
{
    const uint32_t td = __ldcs(d.syn_td + o);
    const int32_t w = __ldcs(d.syn_w + o);
    int sl = tm + (int)(td >> kTgtBits) + 1;
    if (sl >= d.D) sl -= d.D;
    atomicAdd(&d.ring[(long long)sl * d.M + (td & kTgtMask)], w);
}

// Close step t (one thread): raster offsets, the next step's write head,
// step and spike counters.
__device__ __forceinline__ void close_step(const Dev &d, long long t)
{
    Ctrl *c = d.ctrl;
    const int p = (int)(t & 1);
    const unsigned int S = *(volatile unsigned int *)&c->S_acc[p];
    long long h = c->head[p];
    if (c->rec_on) {
        if (t < d.raster_steps && h + S <= d.raster_cap) {
            h += S;
            d.raster_off[t + 1] = h;
            c->rec_steps = t + 1;
        } else {
            c->rec_on = 0;
            c->status |= kStRaster;
        }
    }
    c->head[p ^ 1] = h;
    d.counters[C_STEPS] += 1ull;
    d.counters[C_SPIKES] += S;
}

// ---------------------------------------------------------------- a6
// Work items: the pieces of long segments (one warp each, 4 synapses per
// lane, all loads in flight before the reductions), then chunks of 32 inbox
// entries whose short segments are walked by their lane.
__device__ __forceinline__ void deliver(const Dev &d, long long t)
{
    __shared__ uint32_t s_pre[kPreMax];
    __shared__ unsigned long long s_ev;
    const int p = (int)(t & 1);
    block_prefix(inbox_cnt_of(d, p), d.inbox_capv, s_pre, d.P);
    if (threadIdx.x == 0) s_ev = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) close_step(d, t);
    __syncthreads();
    const int np = d.P + 1;
    const uint32_t n2 = s_pre[d.P];
    const unsigned int npc = min(*(volatile unsigned int *)&d.ctrl->n_piece[p], d.piece_cap);
    const uint32_t items = npc + (n2 + 31u) / 32u;
    const int tm = (int)(t % d.D);
    const int lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * kThreads) >> 5;
    unsigned long long ev = 0;
    for (uint32_t it = (blockIdx.x * kThreads + threadIdx.x) >> 5; it < items; it += nw) {
        if (it < npc) {
            const unsigned long long e = d.piece[it];
            const unsigned long long o = e >> 8;
            const unsigned int n = (unsigned int)(e & 0xFFu);
            uint32_t td[kPiece / 32];
            int32_t w[kPiece / 32];
#pragma unroll
            for (int u = 0; u < kPiece / 32; ++u) {
                const unsigned int k = (unsigned int)u * 32u + (unsigned int)lane;
                if (k < n) {
                    td[u] = __ldcs(d.syn_td + o + k);
                    w[u] = __ldcs(d.syn_w + o + k);
                }
            }
#pragma unroll
            for (int u = 0; u < kPiece / 32; ++u) {
                const unsigned int k = (unsigned int)u * 32u + (unsigned int)lane;
                if (k < n) {
                    int sl = tm + (int)(td[u] >> kTgtBits) + 1;
                    if (sl >= d.D) sl -= d.D;
                    atomicAdd(&d.ring[(long long)sl * d.M + (td[u] & kTgtMask)], w[u]);
                }
            }
            if (lane == 0) ev += n;
        } else {
            const uint32_t x = (it - npc) * 32u + lane;
            if (x < n2) {
                const int q = prefix_find(s_pre, np, x);
                const unsigned long long ent = d.inbox[d.inbox_base[q] + (x - s_pre[q])];
                const unsigned long long off = ent >> kLenBits;
                const unsigned int len = (unsigned int)(ent & kLenMask);
                if (len <= (unsigned int)kShortSeg) {
                    ev += len;
                    for (unsigned int l = 0; l < len; ++l) deliver_one(d, tm, off + l);
                }
            }
        }
    }
    ev = warp_sum(ev);
    if (lane == 0 && ev) atomicAdd(&s_ev, ev);
    __syncthreads();
    if (threadIdx.x == 0 && s_ev) atomicAdd(&d.counters[C_EVENTS], s_ev);
}

// ---------------------------------------------------------------- graph path
// Step t = ctrl->t + k of a captured graph; k_advance moves ctrl->t past the
// graph's steps at its end.
template <bool VEC>
__global__ void __launch_bounds__(kThreads) k_update(const Dev d, int k)
{
    pdl_enter();
    update_route<VEC>(d, d.ctrl->t + k);
}

__global__ void __launch_bounds__(kThreads) k_deliver(const Dev d, int k)
{
    pdl_enter();
    deliver(d, d.ctrl->t + k);
}

__global__ void k_advance(Ctrl *c, int steps)
{
    c->t += steps;
}

// ---------------------------------------------------------------- persistent
// T steps in one cooperative launch: update_route, barrier, deliver, barrier.
// Every wait is bounded (limit_ns per barrier); a timeout ends the run with
// kStTimeout in the status word.  With phase_ns set, block 0 sums the time of
// each phase (from the start of a phase to the end of the barrier after it).
// skip_arrival (tests of the bounded wait only): block 0 waits at the first
// barrier without arriving, so every block's wait runs out.
template <bool VEC>
__global__ void __launch_bounds__(kThreads, 4) k_persist(const Dev d, int T, unsigned long long limit_ns,
                                                         int skip_arrival)
{
    Ctrl *c = d.ctrl;
    const long long t0 = c->t;
    int done = 0;
    unsigned long long ns[2] = {0, 0};
    const bool prof = d.phase_ns != nullptr && blockIdx.x == 0 && threadIdx.x == 0;
    for (int s = 0; s < T; ++s) {
        const long long t = t0 + s;
        const unsigned long long a = prof ? global_ns() : 0;
        update_route<VEC>(d, t);
        if (!grid_sync(c, limit_ns, !(skip_arrival && s == 0 && blockIdx.x == 0))) break;
        const unsigned long long b = prof ? global_ns() : 0;
        deliver(d, t);
        if (!grid_sync(c, limit_ns)) break;
        if (prof) {
            const unsigned long long e = global_ns();
            ns[0] += b - a;
            ns[1] += e - b;
        }
        ++done;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->t = t0 + done;
        if (prof) {
            d.phase_ns[0] += ns[0];
            d.phase_ns[1] += ns[1];
        }
    }
}

}  // namespace
