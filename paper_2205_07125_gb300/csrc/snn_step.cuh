// Step kernel of one simulation step t (sm_103a), included by snn_sim.cu.
//
// The routing is the paper's two-level route (arXiv 2205.07125, Sec. IV.B);
// the neuron model is LIF (Table I); the arithmetic follows the library's
// documented readings (include/snn.h).  Every block runs the whole step on
// its share of the neurons:
//   a1 consume ring slot t mod D, Poisson drive (Philox4x32-10, inverse CDF);
//   a2 FP32 LIF update + threshold (no FMA, fixed order);
//   a3 warp-scan / block-scan compaction of the spikes into a block buffer
//      and the step's spike list (4 neurons per thread, 16-byte loads);
//   a4 level-1 bucketing, one warp per spike: the spike's entry is appended
//      to the bucket of every destination VN in its level-1 row (one entry per
//      VN: deduplicated);
//   a5 level-2 relay expansion: every (spike, VN) entry becomes an inbox
//      entry of each partition of that VN holding targets;
//   a6 delivery of the block's spikes: the level-2 segments are staged in
//      shared memory (long segments cut into 128-synapse pieces, one warp
//      each; short ones walked by one lane) and every synapse adds its int16
//      weight with a 32-bit reduction into ring[(t + d) mod D][target].
// Delivery of step t writes only slots t+1 .. t+D-1 (D = max delay + 1), so
// it may overlap the updates of step t; one grid-wide synchronisation per
// step orders it before step t + 1 reads its slot.  Exchange fill counters
// are kept twice, by step parity: step t fills parity t & 1 and clears the
// other one, which only step t - 1 used.  The spike counts and raster heads
// of steps rotate through three slots (a step's slot is read during the
// next step, cleared during the one after).
//
// Two ways to run: k_persist, one cooperative launch for T steps with a
// bounded grid barrier after each step, and the CUDA-graph path, one k_step
// launch per step with programmatic dependent launch.
#pragma once

#include <cuda_runtime.h>

#include "snn_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kPTab = 32;
constexpr int kSpkBuf = 1024;   // spikes a block buffers before routing them
constexpr int kLongCap = 512;   // staged pieces of one routing round
constexpr int kShortCap = 1024; // staged short segments of one routing round
// Exchange fill counters are keyed by (source partition, destination) pair
// and sit 32 bytes apart, so each sees only the spikes of one source
// partition.
constexpr int kPairStride = 8;

// status bits
constexpr uint32_t kStBucket = 1u, kStInbox = 2u, kStRaster = 4u, kStTimeout = 8u;

// counter slots: steps and spikes in Dev::counters (closing thread), the
// others in each block's tally row
enum { C_STEPS = 0, C_SPIKES, C_EVENTS, C_L1_LOCAL, C_L1_XVN, C_L2_BASE /* + cls (4) */, C_N = 16 };
constexpr int kTally = 7;  // slots C_EVENTS .. C_L2_BASE + 3, consecutive

struct Ctrl {
    long long t;              // next step to run
    long long head[3];        // raster write head of step t at slot t mod 3 (-1: recording stopped)
    long long rec_steps;      // steps whose raster offsets are valid
    unsigned int status;
    int pad;
    alignas(128) unsigned int S_acc[3];   // spikes of step t at slot t mod 3
    alignas(128) unsigned long long bar;  // grid-barrier arrivals of the running k_persist launch
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
    const uint32_t *gid;       // internal -> global id (nullptr when identical)
    const uint16_t *src_part;  // internal partition of each internal neuron
    // synapses and routing tables
    const uint32_t *syn_td;
    const int16_t *syn_w;
    const uint32_t *l1_ptr;
    const uint16_t *l1_vn;
    const uint32_t *l1_l2;
    const DevL2 *l2;
    const uint32_t *l1_pair;  // exchange pair (source partition, VN) of each level-1 entry
    const uint32_t *l2_pair;  // exchange pair (source partition, partition) of each level-2 entry
    // exchange buffers, one region per pair (source partition p, destination)
    uint32_t *bucket;                        // level-1 entry ids, region (p, VN g)
    const unsigned long long *bucket_base;   // [n_bpair]
    const uint32_t *bucket_capv;             // [n_bpair]
    uint32_t *bucket_cnt;                    // [2][n_bpair * kPairStride], by step parity
    unsigned long long *inbox;               // segments offset << 24 | length, region (p, q)
    const unsigned long long *inbox_base;    // [n_ipair]
    const uint32_t *inbox_capv;              // [n_ipair]
    uint32_t *inbox_cnt;                     // [2][n_ipair * kPairStride], by step parity
    // records
    uint32_t *spk;
    long long *raster_off;
    unsigned long long *hash;
    int32_t *cur_rec;
    unsigned long long *counters;  // [C_N] steps and spikes
    unsigned long long *tally;     // [tally_rows][C_N] per-block event and message tallies
    unsigned long long *phase_ns;  // [2] k_persist: block 0's work and barrier wait (profiling)
    Ctrl *ctrl;
    // scalars
    long long M;
    int P, n_vn, vn_size, D;
    int n_bpair, n_ipair;
    float alpha, e_l, v_th, v_reset;
    int t_ref, w_ext, i_bias, th_fin;
    uint32_t key0, key1;
    long long raster_cap, raster_steps, hash_steps;
    int cur_every, cur_slots;
    uint32_t th32[kPTab];   // finite Poisson thresholds (the closing 2^32 is implied)
};

// Counter arrays of step parity par.
__device__ __forceinline__ uint32_t *bucket_cnt_of(const Dev &d, int par)
{
    return d.bucket_cnt + (size_t)par * (size_t)d.n_bpair * kPairStride;
}

__device__ __forceinline__ uint32_t *inbox_cnt_of(const Dev &d, int par)
{
    return d.inbox_cnt + (size_t)par * (size_t)d.n_ipair * kPairStride;
}

// Rotation slot of step x (x >= -1).
__device__ __forceinline__ int slot3(long long x)
{
    return (int)((x + 3) % 3);
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

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release(unsigned long long *p, unsigned long long x)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(x) : "memory");
}

// Programmatic dependent launch (graph path): wait for the grid before this
// one (all of its writes visible) before touching shared state, and let the
// next grid be scheduled early.  Both are no-ops for a plain launch.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Grid-wide barrier number k of a k_persist launch (all blocks co-resident:
// cooperative launch).  Each block adds one arrival to Ctrl::bar, which the
// host zeroes before the launch; barrier k is complete when the count reaches
// (k + 1) * gridDim.x.  A block-wide barrier, then a release add and acquire
// loads at GPU scope make every write of every block before the barrier
// visible to every block after it.  The wait is bounded: past limit_ns the
// block records kStTimeout and gives up, and a block that sees another one's
// timeout gives up too.  Returns false when the block gave up.
__device__ __forceinline__ bool grid_sync(Ctrl *c, unsigned long long k, unsigned long long limit_ns,
                                          bool arrive = true)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long target = (k + 1ull) * gridDim.x;
        if (arrive) red_release(&c->bar, 1ull);
        const unsigned long long deadline = global_ns() + limit_ns;
        unsigned int spins = 0;
        while (ld_acquire(&c->bar) < target) {
            if ((++spins & 15u) == 0u) {
                if (*(volatile unsigned int *)&c->status & kStTimeout) {
                    ok = 0;
                    break;
                }
                if (global_ns() > deadline) {
                    atomicOr(&c->status, kStTimeout);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(64);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
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

// Raster write head of step t + 1 from step t's head h and spike count S:
// recording continues while t is within the recorded steps and the spikes
// fit; -1 once it stopped.
__device__ __forceinline__ long long next_head(const Dev &d, long long h, unsigned int S, long long t)
{
    if (h < 0) return -1;
    if (t < d.raster_steps && h + (long long)S <= d.raster_cap) return h + (long long)S;
    return -1;
}

// Shared-memory state of one block's step (declared by run_step).
struct Stage {
    uint32_t *spk;             // [kSpkBuf] buffered spikes (internal ids)
    unsigned long long *lng;   // [kLongCap] pieces: offset << 8 | length (<= kPiece)
    unsigned long long *sht;   // [kShortCap] short segments: offset << 8 | length (<= kShortSeg)
    unsigned int *n, *gbase, *nl, *ns;
    int *routed;
    unsigned int (*ty)[kTally];  // [kWarps][kTally] tallies: events, l1 local, l1 cross-VN, l2 by class
};

// Add a warp's per-lane tally v into slot k of its shared tally row.
__device__ __forceinline__ void tally_add(const Stage &sg, int k, unsigned int v)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sg.ty[threadIdx.x >> 5][k] += v;
}

// a6 for n consecutive synapses from offset o by one thread (the rare
// overflow of a staging list).
__device__ __forceinline__ unsigned int deliver_run(const Dev &d, int tm, unsigned long long o, unsigned int n)
{
    for (unsigned int k = 0; k < n; ++k) {
        const uint32_t td = __ldcs(d.syn_td + o + k);
        const int32_t w = __ldcs(d.syn_w + o + k);
        int sl = tm + (int)(td >> kTgtBits) + 1;
        if (sl >= d.D) sl -= d.D;
        atomicAdd(&d.ring[(long long)sl * d.M + (td & kTgtMask)], w);
    }
    return n;
}

// a4 + a5 for spike i by one warp, with its delivery work staged in shared
// memory; counters of step parity par.
__device__ __forceinline__ void route_spike(const Dev &d, int par, int tm, uint32_t i, const Stage &sg)
{
    unsigned int ev = 0, l1_loc = 0, l1_xvn = 0, ovf = 0;
    unsigned int cls[4] = {0, 0, 0, 0};
    const int lane = threadIdx.x & 31;
    uint32_t *bcnt = bucket_cnt_of(d, par);
    uint32_t *icnt = inbox_cnt_of(d, par);
    const int p = d.src_part[i];
    const int h = p / d.vn_size;
    const uint32_t e0 = d.l1_ptr[i], e1 = d.l1_ptr[i + 1];
    const uint32_t f0 = d.l1_l2[e0], f1 = d.l1_l2[e1];
    // a4: one level-1 entry per destination VN, appended to bucket (p, g)
    for (uint32_t e = e0 + lane; e < e1; e += 32u) {
        const int g = d.l1_vn[e];
        const uint32_t k = d.l1_pair[e];
        const unsigned int pos = atomicAdd(&bcnt[(size_t)k * kPairStride], 1u);
        if (pos < d.bucket_capv[k]) d.bucket[d.bucket_base[k] + pos] = e;
        else ovf |= kStBucket;
        if (g == h) ++l1_loc;
        else ++l1_xvn;
    }
    // a5: the relay of each destination VN expands the spike's entry into
    // inbox (p, q) of every partition q of that VN holding targets (the
    // level-2 rows of one spike's VNs are contiguous)
    for (uint32_t fb = f0; fb < f1; fb += 32u) {
        const uint32_t f = fb + lane;
        const bool a = f < f1;
        DevL2 l;
        l.off = 0;
        l.len = 0;
        l.q = 0;
        l.cls = 0;
        uint32_t kq = 0;
        if (a) {
            l = d.l2[f];
            kq = d.l2_pair[f];
            const unsigned int pos = atomicAdd(&icnt[(size_t)kq * kPairStride], 1u);
            if (pos < d.inbox_capv[kq])
                d.inbox[d.inbox_base[kq] + pos] = (l.off << kLenBits) | (unsigned long long)l.len;
            else
                ovf |= kStInbox;
            // per-class tallies without a dynamically indexed (local-memory) array
            cls[0] += l.cls == 0;
            cls[1] += l.cls == 1;
            cls[2] += l.cls == 2;
            cls[3] += l.cls == 3;
        }
        // stage the delivery: long segments as pieces, short ones whole
        const bool shrt = a && l.len <= kShortSeg;
        const unsigned int np = (a && !shrt) ? (l.len + kPiece - 1u) / kPiece : 0u;
        unsigned int incl = np;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        const unsigned int ptot = __shfl_sync(0xFFFFFFFFu, incl, 31);
        const unsigned int sm = __ballot_sync(0xFFFFFFFFu, shrt);
        unsigned int pb = 0, sb = 0;
        if (lane == 0) {
            if (ptot) pb = atomicAdd(sg.nl, ptot);
            if (sm) sb = atomicAdd(sg.ns, (unsigned int)__popc(sm));
        }
        pb = __shfl_sync(0xFFFFFFFFu, pb, 0) + incl - np;
        sb = __shfl_sync(0xFFFFFFFFu, sb, 0) + (unsigned int)__popc(sm & ((1u << lane) - 1u));
        for (unsigned int k = 0; k < np; ++k, ++pb) {
            const unsigned long long o = l.off + (unsigned long long)k * kPiece;
            const unsigned int n = min(kPiece, l.len - k * kPiece);
            if (pb < (unsigned int)kLongCap) sg.lng[pb] = (o << 8) | n;
            else ev += deliver_run(d, tm, o, n);  // list full: this lane delivers it
        }
        if (shrt) {
            if (sb < (unsigned int)kShortCap) sg.sht[sb] = (l.off << 8) | l.len;
            else ev += deliver_run(d, tm, l.off, l.len);
        }
    }
    if (ovf) atomicOr(&d.ctrl->status, ovf);
    tally_add(sg, 0, ev);
    tally_add(sg, 1, l1_loc);
    tally_add(sg, 2, l1_xvn);
#pragma unroll
    for (int k = 0; k < 4; ++k) tally_add(sg, 3 + k, cls[k]);
}

// a6 for the staged work of one routing round, all warps of the block: a
// piece per warp (4 synapses per lane, every load in flight before the
// reductions), then short segments a lane each.
__device__ __forceinline__ void deliver_staged(const Dev &d, int tm, const Stage &sg, unsigned int nl,
                                               unsigned int ns)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned int ev = 0;
    const unsigned int units = nl + (ns + 31u) / 32u;
    for (unsigned int u = (unsigned int)wid; u < units; u += kWarps) {
        if (u < nl) {
            const unsigned long long e = sg.lng[u];
            const unsigned long long o = e >> 8;
            const unsigned int n = (unsigned int)(e & 0xFFu);
            uint32_t td[kPiece / 32];
            int32_t w[kPiece / 32];
#pragma unroll
            for (int k = 0; k < (int)(kPiece / 32); ++k) {
                const unsigned int x = (unsigned int)k * 32u + (unsigned int)lane;
                if (x < n) {
                    td[k] = __ldcs(d.syn_td + o + x);
                    w[k] = __ldcs(d.syn_w + o + x);
                }
            }
#pragma unroll
            for (int k = 0; k < (int)(kPiece / 32); ++k) {
                const unsigned int x = (unsigned int)k * 32u + (unsigned int)lane;
                if (x < n) {
                    int sl = tm + (int)(td[k] >> kTgtBits) + 1;
                    if (sl >= d.D) sl -= d.D;
                    atomicAdd(&d.ring[(long long)sl * d.M + (td[k] & kTgtMask)], w[k]);
                }
            }
            if (lane == 0) ev += n;
        } else {
            const unsigned int x = (u - nl) * 32u + (unsigned int)lane;
            if (x < ns) {
                const unsigned long long e = sg.sht[x];
                const unsigned long long o = e >> 8;
                const unsigned int n = (unsigned int)(e & 0xFFu);
                // 4 loads in flight, then their reductions
                for (unsigned int k0 = 0; k0 < n; k0 += 4u) {
                    uint32_t td[4];
                    int32_t w[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (k0 + k < n) {
                            td[k] = __ldcs(d.syn_td + o + k0 + k);
                            w[k] = __ldcs(d.syn_w + o + k0 + k);
                        }
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (k0 + k < n) {
                            int sl = tm + (int)(td[k] >> kTgtBits) + 1;
                            if (sl >= d.D) sl -= d.D;
                            atomicAdd(&d.ring[(long long)sl * d.M + (td[k] & kTgtMask)], w[k]);
                        }
                }
                ev += n;
            }
        }
    }
    tally_add(sg, 0, ev);
}

// Route and deliver the block's buffered spikes in rounds of one spike per
// warp, and append them to the step's spike list at raster head `head`
// (all threads call).
__device__ __forceinline__ void flush_spikes(const Dev &d, long long t, long long head, const Stage &sg)
{
    __syncthreads();
    const unsigned int n = *sg.n;
    if (n == 0) return;
    const int par = (int)(t & 1);
    const int tm = (int)(t % d.D);
    const int wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        *sg.gbase = atomicAdd(&d.ctrl->S_acc[slot3(t)], n);
        *sg.routed = 1;
    }
    for (unsigned int b = 0; b < n; b += kWarps) {
        if (threadIdx.x == 0) {
            *sg.nl = 0;
            *sg.ns = 0;
        }
        __syncthreads();
        if (b + (unsigned int)wid < n) route_spike(d, par, tm, sg.spk[b + wid], sg);
        __syncthreads();
        deliver_staged(d, tm, sg, min(*sg.nl, (unsigned int)kLongCap), min(*sg.ns, (unsigned int)kShortCap));
        __syncthreads();
    }
    if (head >= 0) {
        const unsigned int gb = *sg.gbase;
        for (unsigned int k = threadIdx.x; k < n; k += kThreads) d.spk[head + gb + k] = sg.spk[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) *sg.n = 0;
    __syncthreads();
}

// ---------------------------------------------------------------- a1-a6
// One step t on this block's share of the neurons (all threads call).
template <bool VEC>
__device__ __forceinline__ void run_step(const Dev &d, long long t)
{
    __shared__ uint32_t s_spk[kSpkBuf];
    __shared__ unsigned long long s_lng[kLongCap];
    __shared__ unsigned long long s_sht[kShortCap];
    __shared__ unsigned int s_wsum[kWarps];
    __shared__ unsigned int s_n, s_tot, s_gbase, s_nl, s_ns;
    __shared__ int s_flush, s_routed;
    __shared__ unsigned long long s_h[2][kWarps];
    __shared__ unsigned int s_tally[kWarps][kTally];
    __shared__ uint32_t s_th[kPTab];
    const Stage sg{s_spk, s_lng, s_sht, &s_n, &s_gbase, &s_nl, &s_ns, &s_routed, s_tally};

    Ctrl *c = d.ctrl;
    const int par = (int)(t & 1);
    const int slot = (int)(t % d.D);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool do_hash = t < d.hash_steps;
    const bool do_cur = d.cur_every > 0 && (t % d.cur_every) == 0 && (t / d.cur_every) < d.cur_slots;
    int32_t *ring = d.ring + (long long)slot * d.M;
    int32_t *cur = do_cur ? d.cur_rec + (t / d.cur_every) * d.M : nullptr;
    constexpr int NPT = VEC ? 4 : 1;
    const long long nitem = VEC ? d.M / 4 : d.M;
    // this step's raster head, from the previous step's head and spike count
    const long long head = next_head(d, *(volatile long long *)&c->head[slot3(t - 1)],
                                     *(volatile unsigned int *)&c->S_acc[slot3(t - 1)], t - 1);
    {
        // clear the other parity (used by step t - 1 only; step t + 1 fills
        // it) and the spike count of step t + 1
        uint32_t *b1 = bucket_cnt_of(d, par ^ 1), *i1 = inbox_cnt_of(d, par ^ 1);
        const int nb = d.n_bpair, ni = nb + d.n_ipair;
        for (int x = blockIdx.x * kThreads + threadIdx.x; x < ni; x += gridDim.x * kThreads) {
            if (x < nb) b1[(size_t)x * kPairStride] = 0;
            else i1[(size_t)(x - nb) * kPairStride] = 0;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) c->S_acc[slot3(t + 1)] = 0;
    }
    if (threadIdx.x < kPTab) s_th[threadIdx.x] = d.th32[threadIdx.x];
    if (threadIdx.x == 0) {
        s_n = 0;
        s_routed = 0;
    }
    if (threadIdx.x < kWarps * kTally) (&s_tally[0][0])[threadIdx.x] = 0u;
    __syncthreads();

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
            // one Philox block serves the four neurons of a quad in the
            // global order; a reordering map needs a block per neuron
            uint4 wq = make_uint4(0u, 0u, 0u, 0u);
            if (VEC && !d.gid) wq = philox4(d.key0, d.key1, (uint32_t)(j0 >> 2), (uint32_t)t);
#pragma unroll
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
                for (int w = 0; w < kWarps; ++w) {
                    const unsigned int cw = s_wsum[w];
                    s_wsum[w] = tot;
                    tot += cw;
                }
                s_tot = tot;
                s_flush = (s_n + tot > (unsigned int)kSpkBuf);
            }
            __syncthreads();
            if (s_flush) flush_spikes(d, t, head, sg);
            unsigned int pos = s_n + s_wsum[wid] + x - cnt;
            for (unsigned int mm = m; mm; mm &= mm - 1u) s_spk[pos++] = (uint32_t)(j0 + __ffs(mm) - 1);
            __syncthreads();
            if (threadIdx.x == 0) s_n += s_tot;
        }
    }
    flush_spikes(d, t, head, sg);
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
            for (int w = 0; w < kWarps; ++w) {
                a += s_h[0][w];
                b += s_h[1][w];
            }
            atomicAdd(&d.hash[2 * t], a);
            atomicAdd(&d.hash[2 * t + 1], b);
        }
    }
    __syncthreads();
    if (s_routed) {
        // tallies of the routed spikes into this block's row (no other block
        // writes it, so plain adds)
        if (threadIdx.x < kTally) {
            unsigned long long a = 0;
            for (int w = 0; w < kWarps; ++w) a += s_tally[w][threadIdx.x];
            d.tally[(size_t)blockIdx.x * C_N + C_EVENTS + threadIdx.x] += a;
        }
    }
}

// Close step t (one thread, once every block has finished the step): the
// next step's raster head and offset, step and spike counters.
__device__ __forceinline__ void close_step(const Dev &d, long long t)
{
    Ctrl *c = d.ctrl;
    const unsigned int S = *(volatile unsigned int *)&c->S_acc[slot3(t)];
    const long long h = *(volatile long long *)&c->head[slot3(t)];
    const long long hn = next_head(d, h, S, t);
    c->head[slot3(t + 1)] = hn;
    if (hn >= 0) {
        d.raster_off[t + 1] = hn;
        c->rec_steps = t + 1;
    } else if (h >= 0) {
        atomicOr(&c->status, kStRaster);
    }
    d.counters[C_STEPS] += 1ull;
    d.counters[C_SPIKES] += S;
}

// ---------------------------------------------------------------- graph path
// Step t = ctrl->t + k of a captured graph.  Block 0 closes step t - 1 (the
// graph's first step was closed by the graph before); k_advance closes the
// graph's last step and moves ctrl->t past its steps.
template <bool VEC>
__global__ void __launch_bounds__(kThreads) k_step(const Dev d, int k)
{
    pdl_enter();
    const long long t = *(volatile long long *)&d.ctrl->t + k;
    if (k > 0 && blockIdx.x == 0 && threadIdx.x == 0) close_step(d, t - 1);
    run_step<VEC>(d, t);
}

__global__ void k_advance(const Dev d, int steps)
{
    pdl_enter();
    const long long t = d.ctrl->t;
    if (steps > 0) close_step(d, t + steps - 1);
    d.ctrl->t = t + steps;
}

// ---------------------------------------------------------------- persistent
// T steps in one cooperative launch, a grid barrier after each.  Block 0
// closes step t - 1 while step t runs and the last step after the final
// barrier.  Every wait is bounded (limit_ns per barrier); a timeout ends the
// run with kStTimeout in the status word.  With phase_ns set, block 0 sums
// its own work and its wait at the barrier.  skip_arrival (tests of the
// bounded wait only): block 0 waits at the first barrier without arriving, so
// every block's wait runs out.
template <bool VEC>
__global__ void __launch_bounds__(kThreads, 4) k_persist(const Dev d, int T, unsigned long long limit_ns,
                                                         int skip_arrival)
{
    Ctrl *c = d.ctrl;
    const long long t0 = *(volatile long long *)&c->t;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const bool prof = d.phase_ns != nullptr && lead;
    int done = 0;
    long long closed = t0 - 1;
    unsigned long long ns[2] = {0, 0};
    for (int s = 0; s < T; ++s) {
        const long long t = t0 + s;
        const unsigned long long a = prof ? global_ns() : 0;
        if (s > 0 && lead) {
            close_step(d, t - 1);
            closed = t - 1;
        }
        run_step<VEC>(d, t);
        const unsigned long long b = prof ? global_ns() : 0;
        if (!grid_sync(c, (unsigned long long)s, limit_ns, !(skip_arrival && s == 0 && blockIdx.x == 0))) break;
        if (prof) {
            const unsigned long long e = global_ns();
            ns[0] += b - a;
            ns[1] += e - b;
        }
        ++done;
    }
    if (lead) {
        if (t0 + done - 1 > closed) close_step(d, t0 + done - 1);
        c->t = t0 + done;
        if (prof) {
            d.phase_ns[0] += ns[0];
            d.phase_ns[1] += ns[1];
        }
    }
}

}  // namespace
