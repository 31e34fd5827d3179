// Host side of the simulation: device layout in the caller's workspace, table
// upload, CUDA-graph capture and replay of the step kernels (snn_step.cuh),
// the spike fan-out entry points, and the read-out and checkpoint calls of
// the C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <new>
#include <vector>

#include "snn_internal.h"

using namespace snn;

#include "snn_step.cuh"

namespace {

// ---------------------------------------------------------------- spike fan-out
// Route and fan out a caller-given spike list (snn_deliver_spikes): the same
// level-1 -> level-2 -> segment path as a step, with flat scratch lists and
// the result accumulated into a caller buffer out[d-1][global id].
struct FoArgs {
    const uint32_t *ids;
    long long n;
    const uint32_t *fwd;  // global -> internal (nullptr when identical)
    const uint32_t *gid;  // internal -> global (nullptr when identical)
    const uint32_t *l1_ptr;
    const uint32_t *l1_l2;
    const DevL2 *l2;
    const uint32_t *syn_td;
    const int16_t *syn_w;
    uint32_t *bucket;              // scratch: level-1 entry ids
    unsigned long long cap1;
    unsigned long long *inbox;     // scratch: packed segments
    unsigned long long cap2;
    unsigned int *cnt;             // scratch: [0] bucket fill, [1] inbox fill, [2] status
    unsigned long long *ev;        // scratch: events delivered
    int32_t *out;
    long long M;
};

constexpr unsigned int kFoStBucket = 1u, kFoStInbox = 2u, kFoStId = 4u;

__global__ void __launch_bounds__(kThreads) k_fo_level1(const FoArgs a)
{
    unsigned int st = 0;
    for (long long s = (long long)blockIdx.x * kThreads + threadIdx.x; s < a.n;
         s += (long long)gridDim.x * kThreads) {
        const uint32_t g = a.ids[s];
        if ((long long)g >= a.M) {
            st |= kFoStId;
            continue;
        }
        const uint32_t i = a.fwd ? a.fwd[g] : g;
        for (uint32_t e = a.l1_ptr[i]; e < a.l1_ptr[i + 1]; ++e) {
            const unsigned int pos = atomicAdd(&a.cnt[0], 1u);
            if (pos < a.cap1) a.bucket[pos] = e;
            else st |= kFoStBucket;
        }
    }
    if (st) atomicOr(&a.cnt[2], st);
}

__global__ void __launch_bounds__(kThreads) k_fo_level2(const FoArgs a)
{
    unsigned int st = 0;
    const unsigned long long n1 = min((unsigned long long)a.cnt[0], a.cap1);
    for (unsigned long long x = (unsigned long long)blockIdx.x * kThreads + threadIdx.x; x < n1;
         x += (unsigned long long)gridDim.x * kThreads) {
        const uint32_t e = a.bucket[x];
        for (uint32_t f = a.l1_l2[e]; f < a.l1_l2[e + 1]; ++f) {
            const DevL2 l = a.l2[f];
            const unsigned int pos = atomicAdd(&a.cnt[1], 1u);
            if (pos < a.cap2) a.inbox[pos] = ((l.off & kOffMask) << kLenBits) | (unsigned long long)l.len;
            else st |= kFoStInbox;
        }
    }
    if (st) atomicOr(&a.cnt[2], st);
}

__global__ void __launch_bounds__(kThreads) k_fo_deliver(const FoArgs a)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long n2 = min((unsigned long long)a.cnt[1], a.cap2);
    const unsigned long long nw = ((unsigned long long)gridDim.x * kThreads) >> 5;
    unsigned long long ev = 0;
    for (unsigned long long x = ((unsigned long long)blockIdx.x * kThreads + threadIdx.x) >> 5; x < n2;
         x += nw) {
        const unsigned long long ent = a.inbox[x];
        const unsigned long long off = ent >> kLenBits;
        const unsigned int len = (unsigned int)(ent & kLenMask);
        for (unsigned int l = lane; l < len; l += 32) {
            const uint32_t td = a.syn_td[off + l];
            const uint32_t tgt = td & kTgtMask;
            const long long j = a.gid ? (long long)a.gid[tgt] : (long long)tgt;
            atomicAdd(&a.out[(long long)(td >> kTgtBits) * a.M + j], (int32_t)a.syn_w[off + l]);
        }
        ev += len;
    }
    if (lane == 0 && ev) atomicAdd(a.ev, ev);
}

// ---------------------------------------------------------------- delivery by arrival step
// Delay counts of every level-2 segment (the segment's synapses are sorted by
// delay): dcnt[f] holds c[k] = synapses of delay <= k + 1, k = 0..7, as 16-bit
// fields (segments of at most 65535 synapses, delays up to 8).
__global__ void __launch_bounds__(kThreads) k_delay_counts(const DevL2 *l2, const uint32_t *syn_td, long long n_l2,
                                                           uint4 *dcnt)
{
    for (long long f = (long long)blockIdx.x * kThreads + threadIdx.x; f < n_l2;
         f += (long long)gridDim.x * kThreads) {
        const DevL2 l = l2[f];
        const unsigned long long o = l.off & kOffMask;
        // a segment is sorted by (delay, target): the count of delay <= x + 1
        // is where the delay first exceeds it (a binary search per delay, so
        // that the long own-partition segments do not hold up their warps)
        uint32_t c[kMaxArr];
#pragma unroll
        for (int x = 0; x < kMaxArr; ++x) {
            uint32_t lo = 0, hi = l.len;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if ((syn_td[o + mid] >> kTgtBits) <= (uint32_t)x) lo = mid + 1;
                else hi = mid;
            }
            c[x] = lo;
        }
        dcnt[f] = make_uint4(c[0] | (c[1] << 16), c[2] | (c[3] << 16), c[4] | (c[5] << 16), c[6] | (c[7] << 16));
    }
}

// Checkpoint of a sim with delivery by arrival step, next step t: move the
// state into the delay-ring form a checkpoint holds.  Step t's input slot
// goes into ring slot t mod D; every run still queued (lists of steps t ..
// t + n_arr - 2, arriving at step s + 1) is added into ring slot (s + 1) mod
// D.  The caller then clears the lists and lets steps < t + D consume their
// ring slots (Ctrl::inject_until), so the sim continues unchanged.
__global__ void __launch_bounds__(kThreads) k_materialize(const Dev d, long long t)
{
    const long long stride = (long long)gridDim.x * kThreads;
    const long long x0 = (long long)blockIdx.x * kThreads + threadIdx.x;
    int32_t *in = d.acc + (size_t)(t & 1) * (size_t)d.M;
    int32_t *slot = d.ring + (size_t)(t % d.D) * (size_t)d.M;
    for (long long j = x0; j < d.M; j += stride) {
        slot[j] = (int32_t)((uint32_t)slot[j] + (uint32_t)in[j]);
        in[j] = 0;
    }
    for (int k = 0; k + 1 < d.n_arr; ++k) {
        const long long s = t + k;
        const int li = (int)(s % d.n_arr);
        const unsigned long long n =
            min((unsigned long long)d.arr_cnt[(size_t)li * kPairStride], d.arr_cap);
        int32_t *dst = d.ring + (size_t)((s + 1) % d.D) * (size_t)d.M;
        const unsigned long long *recs = d.arr + (size_t)li * d.arr_cap;
        for (long long r = x0; r < (long long)n; r += stride) {
            const unsigned long long rec = recs[r];
            const unsigned long long o = rec >> kLenBits;
            const unsigned int len = (unsigned int)(rec & kLenMask);
            for (unsigned int y = 0; y < len; ++y)
                atomicAdd(dst + (d.syn_td[o + y] & kTgtMask), (int32_t)d.syn_w[o + y]);
        }
    }
}

// The same for partition-owned delivery, next step t: every list (q, li)
// holds runs arriving at step s = the step in t .. t + n_own - 1 with
// s mod n_own = li, added into ring slot s mod D.
__global__ void __launch_bounds__(kThreads) k_materialize_owner(const Dev d, long long t)
{
    for (int q = blockIdx.x; q < d.P; q += gridDim.x) {
        const ulonglong2 sl = d.inb_slot[q];
        for (int li = 0; li < d.n_own; ++li) {
            const long long s = t + ((li - (int)(t % d.n_own)) % d.n_own + d.n_own) % d.n_own;
            int32_t *dst = d.ring + (size_t)(s % d.D) * (size_t)d.M;
            const unsigned long long n =
                min((unsigned long long)d.inb_cnt[((size_t)q * d.n_own + li) * kPairStride], sl.y);
            const unsigned long long *recs = d.inb + sl.x + (unsigned long long)li * sl.y;
            for (unsigned long long r = threadIdx.x; r < n; r += kThreads) {
                const unsigned long long rec = recs[r];
                const unsigned long long o = rec >> kLenBits;
                const unsigned int len = (unsigned int)(rec & kLenMask);
                for (unsigned int y = 0; y < len; ++y)
                    atomicAdd(dst + (d.syn_td[o + y] & kTgtMask), (int32_t)d.syn_w[o + y]);
            }
        }
    }
}

// ---------------------------------------------------------------- host helpers
struct Region {
    size_t off = 0, bytes = 0;
};

struct Layout {
    Region V, ref, ring, gid, src_part, syn_td, syn_w, l1_ptr, l1_vn, l1_l2, l2, row, csr, l1_pair, l2_pair;
    Region bucket, bucket_slot, bucket_cnt, inbox, inbox_slot, inbox_cnt;
    Region tally;  // per-block tally rows
    Region net_of, net_drive;  // batches: network of each quad, drive of each network
    Region spk, spk_step, raster_off, hash, cur_rec, counters, ctrl;
    Region fwd, fo_cnt;  // snn_deliver_spikes: global -> internal map, scratch counters
    Region phase_ns;
    Region acc, arr, arr_cnt, dcnt;  // delivery by arrival step (absent with SNN_DELIVER_RING)
    Region inb, inb_slot, inb_cnt, pbase;  // partition-owned delivery
    size_t total = 0;
    int n_arr = 0;                   // arrival lists (the largest delay); 0: no arrival regions
    uint64_t arr_cap = 0;            // runs per arrival list
    int n_own = 0;                   // lists per partition of owned delivery; 0: no owner regions
    int64_t own_max = 0;             // neurons of the largest partition
    std::vector<uint64_t> inb_base_h, inb_cap_h;  // per internal partition: first record, list capacity
    std::vector<uint64_t> bucket_base_h, inbox_base_h;
    std::vector<uint32_t> bucket_cap_h, inbox_cap_h;
    int64_t tally_rows = 0;
    int32_t n_net = 0;  // networks of a batch (0: a single network)
    int D = 2;
};

static void place(Layout &L, Region &r, size_t bytes)
{
    r.off = L.total;
    r.bytes = bytes;
    L.total += (bytes + 255) & ~(size_t)255;
}

// Blocks of one k_step launch: one pass over the neurons, 4 per thread when
// M % 4 == 0.
static int64_t step_grid(int64_t M)
{
    const int64_t items = (M % 4) == 0 ? M / 4 : M;
    return std::max<int64_t>(1, (items + kThreads - 1) / kThreads);
}

// Tally rows: one per block of either launch shape (a persistent grid is
// capped to the rows there are).
constexpr int64_t kMinTallyRows = 2048;

// Level-2 statistics of delivery by arrival step (cached in the routing):
// the longest segment, the segments holding a synapse of delay >= 2 and the
// sum over segments of min(max_delay - 1, synapses of delay >= 2).
static void arrival_stats(const snn_routing *rt)
{
    if (rt->seg_runs.load() >= 0) return;
    const int nt = resolve_threads(0);
    std::vector<int64_t> mx((size_t)nt, 0), dl((size_t)nt, 0), rn((size_t)nt, 0);
    const int64_t lim = std::max(0, rt->max_delay - 1);
    parallel_for(rt->n_l2, nt, [&](int64_t lo, int64_t hi, int k) {
        int64_t a = 0, b = 0, c = 0;
        for (int64_t f = lo; f < hi; ++f) {
            const L2Entry &e = rt->l2[f];
            const int64_t n1 = (int64_t)(e.off >> kOffBits), late = (int64_t)e.len - n1;
            a = std::max<int64_t>(a, e.len);
            b += late > 0;
            c += std::min(lim, late);
        }
        mx[k] = a;
        dl[k] = b;
        rn[k] = c;
    });
    int64_t a = 0, b = 0, c = 0;
    for (int k = 0; k < nt; ++k) {
        a = std::max(a, mx[k]);
        b += dl[k];
        c += rn[k];
    }
    rt->seg_maxlen.store(a);
    rt->seg_delayed.store(b);
    rt->seg_runs.store(c);
}

// Whether the routing allows delivery by arrival step: delays up to
// kMaxArr and segments short enough for the 16-bit delay counts.
static bool arrival_possible(const snn_routing *rt)
{
    arrival_stats(rt);
    return rt->max_delay <= kMaxArr && rt->seg_maxlen.load() <= 0xFFFF;
}

// Per internal destination partition: the level-2 segments into it and the
// sum over them of min(max_delay, length) (cached in the routing).
static void owner_stats(const snn_routing *rt)
{
    std::call_once(rt->own_once, [rt]() {
        const int32_t P = rt->P;
        const int nt = resolve_threads(0);
        std::vector<std::vector<int64_t>> sg((size_t)nt), rn((size_t)nt);
        const int64_t lim = std::max(1, rt->max_delay);
        parallel_for(rt->n_l2, nt, [&](int64_t lo, int64_t hi, int k) {
            sg[k].assign((size_t)P, 0);
            rn[k].assign((size_t)P, 0);
            for (int64_t f = lo; f < hi; ++f) {
                const L2Entry &e = rt->l2[f];
                sg[k][e.q] += 1;
                rn[k][e.q] += std::min<int64_t>(lim, e.len);
            }
        });
        rt->own_segs.assign((size_t)P, 0);
        rt->own_runs.assign((size_t)P, 0);
        for (int k = 0; k < nt; ++k)
            if (!sg[k].empty())
                for (int32_t q = 0; q < P; ++q) {
                    rt->own_segs[q] += sg[k][q];
                    rt->own_runs[q] += rn[k][q];
                }
    });
}

// The largest accumulator a block of k_owner may hold in shared memory.
constexpr int64_t kOwnerSmemMax = 200 * 1024;

// The delivery a sim uses: the parameter, or SNN_DELIVERY=0|1|2|3 from the
// environment (tests of every path).
static int effective_delivery(const snn_sim_params *p)
{
    int delivery = p->delivery;
    if (const char *e = std::getenv("SNN_DELIVERY"))
        if (e[0] >= '0' && e[0] <= '3' && e[1] == 0) delivery = e[0] - '0';
    return delivery;
}

static int make_layout(const snn_routing *rt, const snn_sim_params *p, Layout &L, int32_t n_net = 0)
{
    const int64_t M = rt->M, E = rt->E;
    L = Layout();
    L.n_net = n_net;
    L.D = rt->max_delay + 1;
    auto cap = [](uint64_t exact, float frac) -> uint64_t {
        double c = std::ceil((double)exact * (double)frac);
        if (c < 0) c = 0;
        if (c > (double)exact) c = (double)exact;
        return (uint64_t)c;
    };
    // one region per exchange pair and per source partition's work list,
    // each sized by its exact worst case times the capacity fraction
    auto regions = [&](const uint64_t *exact, size_t n, float frac, std::vector<uint64_t> &base,
                       std::vector<uint32_t> *capv, uint64_t &tot) -> bool {
        base.resize(n);
        tot = 0;
        for (size_t k = 0; k < n; ++k) {
            const uint64_t c = cap(exact[k], frac);
            if (c > 0xFFFFFFFFull) return false;
            base[k] = tot;
            if (capv) capv->push_back((uint32_t)c);
            tot += c;
        }
        return true;
    };
    const int32_t P = rt->P;
    const size_t n_bp = rt->bpair_cap.size(), n_ip = rt->ipair_cap.size();
    std::vector<uint64_t> ex(rt->bpair_cap.begin(), rt->bpair_cap.end());
    uint64_t nb = 0, ni = 0;
    if (!regions(ex.data(), n_bp, p->bucket_frac, L.bucket_base_h, &L.bucket_cap_h, nb)) return SNN_E_RANGE;
    ex.assign(rt->ipair_cap.begin(), rt->ipair_cap.end());
    if (!regions(ex.data(), n_ip, p->inbox_frac, L.inbox_base_h, &L.inbox_cap_h, ni)) return SNN_E_RANGE;
    (void)P;
    L.tally_rows = std::max<int64_t>(step_grid(rt->M), kMinTallyRows);
    place(L, L.ctrl, sizeof(Ctrl));
    place(L, L.counters, sizeof(unsigned long long) * C_N);
    place(L, L.V, sizeof(float) * (size_t)M);
    place(L, L.ref, (size_t)M);
    place(L, L.ring, sizeof(int32_t) * (size_t)M * (size_t)L.D);
    place(L, L.gid, rt->identity ? 0 : sizeof(uint32_t) * (size_t)M);
    place(L, L.src_part, sizeof(uint16_t) * (size_t)M);
    place(L, L.syn_td, sizeof(uint32_t) * (size_t)E);
    place(L, L.syn_w, sizeof(int16_t) * (size_t)E);
    place(L, L.l1_ptr, sizeof(uint32_t) * (size_t)(M + 1));
    place(L, L.l1_vn, sizeof(uint16_t) * (size_t)rt->n_l1);
    place(L, L.l1_l2, sizeof(uint32_t) * (size_t)(rt->n_l1 + 1));
    place(L, L.l2, sizeof(L2Entry) * (size_t)rt->n_l2);
    place(L, L.row, sizeof(uint2) * (size_t)(M + 1));
    place(L, L.csr, sizeof(unsigned long long) * (size_t)(M + 1));
    place(L, L.l1_pair, sizeof(uint32_t) * (size_t)rt->n_l1);
    place(L, L.l2_pair, sizeof(uint32_t) * (size_t)rt->n_l2);
    place(L, L.bucket, sizeof(uint32_t) * (size_t)nb);
    place(L, L.bucket_slot, sizeof(ulonglong2) * n_bp);
    place(L, L.bucket_cnt, 2 * sizeof(uint32_t) * kPairStride * n_bp);  // by step parity
    place(L, L.inbox, sizeof(uint64_t) * (size_t)ni);
    place(L, L.inbox_slot, sizeof(ulonglong2) * n_ip);
    place(L, L.inbox_cnt, 2 * sizeof(uint32_t) * kPairStride * n_ip);  // by step parity
    place(L, L.tally, sizeof(unsigned long long) * C_N * (size_t)L.tally_rows);
    if (n_net > 0) {
        place(L, L.net_of, sizeof(uint16_t) * (size_t)(M / 4));
        place(L, L.net_drive, sizeof(NetDrive) * (size_t)n_net);
    }
    place(L, L.spk, sizeof(uint32_t) * (size_t)(p->raster_cap + M));
    place(L, L.spk_step, sizeof(uint32_t) * (size_t)M);
    place(L, L.raster_off, sizeof(long long) * (size_t)(p->raster_steps + 1));
    place(L, L.hash, sizeof(unsigned long long) * 2 * (size_t)p->hash_steps);
    place(L, L.cur_rec, sizeof(int32_t) * (size_t)M * (size_t)p->cur_slots);
    place(L, L.fwd, rt->identity ? 0 : sizeof(uint32_t) * (size_t)M);
    place(L, L.fo_cnt, 64);
    place(L, L.phase_ns, kPhases * sizeof(unsigned long long));
    const int delivery = effective_delivery(p);
    const bool want_arr = (delivery == SNN_DELIVER_ARRIVAL || delivery == SNN_DELIVER_AUTO) && !p->defer_delayed;
    const bool want_own = (delivery == SNN_DELIVER_OWNER || delivery == SNN_DELIVER_AUTO) && !p->defer_delayed;
    if (want_own) {
        int64_t mx = 0;
        for (int32_t q = 0; q < P; ++q) mx = std::max(mx, rt->pbase[q + 1] - rt->pbase[q]);
        // (quads of 4 ids with 16-byte accesses: M % 4 == 0)
        if (!arrival_possible(rt) || mx * 4 > kOwnerSmemMax || rt->M % 4 != 0) {
            if (delivery == SNN_DELIVER_OWNER) return SNN_E_RANGE;
        } else {
            // each list's exact worst case: with t_ref >= max_delay - 1 a neuron
            // spikes at most once in the max_delay steps that feed a list (one run
            // per segment into q), else one run per delay present in a segment
            owner_stats(rt);
            L.n_own = rt->max_delay;
            L.own_max = mx;
            L.inb_base_h.assign((size_t)P, 0);
            L.inb_cap_h.assign((size_t)P, 0);
            uint64_t tot = 0;
            for (int32_t q = 0; q < P; ++q) {
                const int64_t worst = p->t_ref >= L.n_own - 1 ? rt->own_segs[q] : rt->own_runs[q];
                const uint64_t c = cap((uint64_t)worst, p->arrival_frac);
                if (c > 0xFFFFFFFFull) return SNN_E_RANGE;  // 32-bit fill counters
                L.inb_base_h[q] = tot;
                L.inb_cap_h[q] = c;
                tot += c * (uint64_t)L.n_own;
            }
            place(L, L.inb, sizeof(unsigned long long) * (size_t)tot);
            place(L, L.inb_slot, sizeof(ulonglong2) * (size_t)P);
            place(L, L.inb_cnt, sizeof(uint32_t) * kPairStride * (size_t)P * (size_t)L.n_own);
            place(L, L.pbase, sizeof(long long) * (size_t)(P + 1));
        }
    }
    if (want_arr) {
        if (!arrival_possible(rt)) {
            if (delivery == SNN_DELIVER_ARRIVAL) return SNN_E_RANGE;
        } else {
            // each arrival list's exact worst case: with t_ref >= max_delay - 2 a
            // neuron spikes at most once in the max_delay - 1 steps that feed a
            // list (at most one run per segment), else one run per delay >= 2
            // present in the segment
            L.n_arr = rt->max_delay;
            const int64_t worst = p->t_ref >= L.n_arr - 2 ? rt->seg_delayed.load() : rt->seg_runs.load();
            double c = std::ceil((double)worst * (double)p->arrival_frac);
            if (c > (double)worst) c = (double)worst;
            if (c > 4294967295.0) return SNN_E_RANGE;  // 32-bit fill counters
            L.arr_cap = (uint64_t)c;
            place(L, L.acc, 2 * sizeof(int32_t) * (size_t)M);
            place(L, L.arr, sizeof(unsigned long long) * (size_t)L.n_arr * (size_t)L.arr_cap);
            place(L, L.arr_cnt, sizeof(uint32_t) * kPairStride * (size_t)L.n_arr);
        }
    }
    if (L.n_arr > 0 || L.n_own > 0) place(L, L.dcnt, sizeof(uint4) * (size_t)rt->n_l2);
    return SNN_OK;
}

static bool params_ok(const snn_sim_params *p)
{
    if (!p) return false;
    if (!(p->dt_ms > 0) || !(p->tau_ms > 0)) return false;
    if (p->t_ref < 0 || p->t_ref > 255) return false;
    if (!(p->drive_lambda >= 0.0) || p->drive_lambda > 16.0) return false;
    if (p->raster_cap < 0 || p->raster_steps < 0 || p->hash_steps < 0) return false;
    if (p->cur_every < 0 || p->cur_slots < 0) return false;
    if (!(p->bucket_frac >= 0.0f) || !(p->inbox_frac >= 0.0f)) return false;
    if (p->steps_per_graph < 1 || p->steps_per_graph > 256) return false;
    if (p->defer_delayed != 0 && p->defer_delayed != 1) return false;
    if (p->delivery < SNN_DELIVER_RING || p->delivery > SNN_DELIVER_OWNER) return false;
    if (!(p->arrival_frac >= 0.0f)) return false;
    if (p->defer_delayed && (p->delivery == SNN_DELIVER_ARRIVAL || p->delivery == SNN_DELIVER_OWNER)) return false;
    return true;
}

// Poisson inverse-CDF thresholds floor(2^32 * CDF(k)), closed by 2^32 at the
// first threshold that reaches 2^32 - 1 (pmf by p_k = p_{k-1} lambda / k).
static int poisson_thresholds(double lambda, unsigned long long *th, int *len)
{
    double pmf = std::exp(-lambda), cdf = pmf;
    int n = 0;
    for (int k = 0; k < kPTab; ++k) {
        if (k > 0) {
            pmf = pmf * lambda / (double)k;
            cdf = cdf + pmf;
        }
        double x = std::floor(cdf * 4294967296.0);
        unsigned long long v = x >= 4294967295.0 ? 4294967296ULL : (unsigned long long)x;
        th[k] = v;
        n = k + 1;
        if (v >= 4294967296ULL) break;
    }
    for (int k = n; k < kPTab; ++k) th[k] = 4294967296ULL;
    *len = n;
    return SNN_OK;
}

// The finite thresholds of the inverse-CDF table (every one but the closing
// 2^32 fits in 32 bits) and their count.
static void finite_thresholds(double lambda, uint32_t *th32, int *fin)
{
    unsigned long long th[kPTab];
    int len = 0;
    poisson_thresholds(lambda, th, &len);
    *fin = len - 1;
    for (int k = 0; k < kPTab; ++k) th32[k] = k < len - 1 ? (uint32_t)th[k] : 0xFFFFFFFFu;
}

}  // namespace

struct snn_sim {
    const snn_routing *rt = nullptr;
    snn_sim_params prm;
    Layout L;
    Dev dev;
    char *ws = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t g1 = nullptr, gU = nullptr;
    int U = 32;
    int device = 0;
    cudaGraphExec_t gP = nullptr;  // instrumented graph (snn_profile_phases)
    int UP = 0;
    std::vector<cudaEvent_t> pev;
    int64_t static_row_l1 = -1, static_row_l2 = -1;  // snn_deliver_spikes_static sizing
    unsigned grid_update = 1, grid_route = 1;
    bool vec = false;  // 4 neurons per thread with 16-byte loads (M % 4 == 0)
    int pmode = kModeScalar;  // neuron-state access of k_persist
    size_t persist_smem = 0;  // dynamic shared memory of k_persist (kModeSmem)
    int64_t chunk_q = 0;      // quads per block of k_persist (kModeSmem)
    int sms = 0;              // SMs of the device
    bool coop = false;        // cooperative launch available
    int persist_bps = 0;      // blocks per SM of k_persist
    bool allow_persist = true, allow_smem = true;  // SNN_PERSIST / SNN_PERSIST_SMEM
    bool pdl = true;       // programmatic dependent launch between step kernels
    bool persist = false;  // one cooperative launch per snn_step (k_persist)
    bool defer = false;    // k_persist with minimum-delay batching (shared-memory state only)
    bool arrival = false;  // delivery by arrival step active (the workspace holds its regions)
    bool owner = false;    // partition-owned delivery active (k_owner; the workspace holds its regions)
    size_t owner_smem = 0; // dynamic shared memory of k_owner: the largest partition's accumulator
    unsigned grid_persist = 1;
    // bound on one grid-barrier wait of k_persist: a healthy barrier takes
    // microseconds; past this the kernel records a timeout and returns
    unsigned long long barrier_limit_ns = 1000000000ull;
    int test_skip_arrival = 0;  // tests of the bounded wait (SNN_TEST_SKIP_BARRIER)
    std::vector<uint2> row_h;   // the uploaded per-neuron rows (host copy, kept for re-uploads)
    std::vector<void *> pinned;
    // batches: the network of each quad and each network's drive (host copies)
    std::vector<uint16_t> net_of_h;
    std::vector<NetDrive> net_drive_h;
};

#define CK(x)                                     \
    do {                                          \
        cudaError_t e_ = (x);                     \
        if (e_ != cudaSuccess) return SNN_E_CUDA; \
    } while (0)

extern "C" void snn_sim_params_default(snn_sim_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->dt_ms = 0.1;
    p->tau_ms = 20.0;
    p->e_l = -65.0f;
    p->v_th = -50.0f;
    p->v_reset = -65.0f;
    p->t_ref = 20;
    p->drive_lambda = 0.8;
    p->w_ext = 96;
    p->i_bias = 0;
    p->drive_seed = 2000;
    p->bucket_frac = 1.0f;
    p->inbox_frac = 1.0f;
    p->steps_per_graph = 32;
    p->delivery = SNN_DELIVER_RING;
    p->arrival_frac = 1.0f;
}

extern "C" int snn_sim_workspace_bytes(const snn_routing *rt, const snn_sim_params *p, size_t *bytes)
{
    if (!rt || !bytes || !params_ok(p)) return SNN_E_ARG;
    Layout L;
    int rc = make_layout(rt, p, L);
    if (rc) return rc;
    *bytes = L.total;
    return SNN_OK;
}

static int upload_tables(snn_sim *s)
{
    const snn_routing *rt = s->rt;
    const Layout &L = s->L;
    char *w = s->ws;
    cudaStream_t st = s->stream;
    auto up = [&](const Region &r, const void *src) -> cudaError_t {
        if (!r.bytes) return cudaSuccess;
        return cudaMemcpyAsync(w + r.off, src, r.bytes, cudaMemcpyHostToDevice, st);
    };
    CK(up(L.syn_td, rt->syn_td.data()));
    CK(up(L.syn_w, rt->syn_w.data()));
    CK(up(L.l1_ptr, rt->l1_ptr.data()));
    CK(up(L.l1_vn, rt->l1_vn.data()));
    CK(up(L.l1_l2, rt->l1_l2.data()));
    CK(up(L.l2, rt->l2.data()));
    CK(up(L.src_part, rt->src_part.data()));
    if (L.n_net > 0) {
        CK(up(L.net_of, s->net_of_h.data()));
        CK(up(L.net_drive, s->net_drive_h.data()));
    }
    CK(up(L.l1_pair, rt->l1_pair.data()));
    {
        // first level-1 and level-2 entry of each neuron, read together (built
        // once per sim)
        if (s->row_h.size() != (size_t)rt->M + 1) {
            s->row_h.resize((size_t)rt->M + 1);
            for (int64_t i = 0; i <= rt->M; ++i)
                s->row_h[i] = make_uint2(rt->l1_ptr[i], rt->l1_l2[rt->l1_ptr[i]]);
        }
        CK(cudaMemcpyAsync(w + L.row.off, s->row_h.data(), L.row.bytes, cudaMemcpyHostToDevice, st));
    }
    CK(up(L.l2_pair, rt->l2_pair.data()));
    CK(up(L.csr, rt->csr.data()));
    if (L.n_own > 0) {
        // partition bounds and each partition's list region
        CK(cudaMemcpyAsync(w + L.pbase.off, rt->pbase.data(), L.pbase.bytes, cudaMemcpyHostToDevice, st));
        std::vector<ulonglong2> v((size_t)rt->P);
        for (int32_t q = 0; q < rt->P; ++q) v[q] = make_ulonglong2(L.inb_base_h[q], L.inb_cap_h[q]);
        CK(cudaMemcpy(w + L.inb_slot.off, v.data(), L.inb_slot.bytes, cudaMemcpyHostToDevice));
    }
    if (L.dcnt.bytes && rt->n_l2 > 0) {
        // delay counts of every segment, from the uploaded tables
        const long long g = std::min<long long>((rt->n_l2 + kThreads - 1) / kThreads, (long long)s->sms * 8);
        k_delay_counts<<<(unsigned)std::max(1ll, g), kThreads, 0, st>>>(
            (const DevL2 *)(w + L.l2.off), (const uint32_t *)(w + L.syn_td.off), (long long)rt->n_l2,
            (uint4 *)(w + L.dcnt.off));
        CK(cudaGetLastError());
    }
    if (!rt->identity) CK(up(L.gid, rt->perm_inv.data()));
    if (!rt->identity) CK(up(L.fwd, rt->perm_fwd.data()));
    {
        // exchange regions {first entry, capacity} of every pair
        auto slots = [&](const Region &r, const std::vector<uint64_t> &base, const std::vector<uint32_t> &cap) {
            std::vector<ulonglong2> v(base.size());
            for (size_t k = 0; k < v.size(); ++k) v[k] = make_ulonglong2(base[k], cap[k]);
            return r.bytes ? cudaMemcpy(w + r.off, v.data(), r.bytes, cudaMemcpyHostToDevice) : cudaSuccess;
        };
        CK(slots(L.bucket_slot, L.bucket_base_h, L.bucket_cap_h));
        CK(slots(L.inbox_slot, L.inbox_base_h, L.inbox_cap_h));
    }
    return SNN_OK;
}

static int reset_state(snn_sim *s)
{
    const Layout &L = s->L;
    char *w = s->ws;
    cudaStream_t st = s->stream;
    CK(cudaMemcpyAsync(w + L.V.off, s->rt->v0.data(), L.V.bytes, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(w + L.ref.off, 0, L.ref.bytes, st));
    CK(cudaMemsetAsync(w + L.ring.off, 0, L.ring.bytes, st));
    CK(cudaMemsetAsync(w + L.counters.off, 0, L.counters.bytes, st));
    CK(cudaMemsetAsync(w + L.bucket_cnt.off, 0, L.bucket_cnt.bytes, st));
    CK(cudaMemsetAsync(w + L.inbox_cnt.off, 0, L.inbox_cnt.bytes, st));
    CK(cudaMemsetAsync(w + L.tally.off, 0, L.tally.bytes, st));
    if (L.raster_off.bytes) CK(cudaMemsetAsync(w + L.raster_off.off, 0, L.raster_off.bytes, st));
    if (L.hash.bytes) CK(cudaMemsetAsync(w + L.hash.off, 0, L.hash.bytes, st));
    if (L.cur_rec.bytes) CK(cudaMemsetAsync(w + L.cur_rec.off, 0, L.cur_rec.bytes, st));
    if (L.acc.bytes) CK(cudaMemsetAsync(w + L.acc.off, 0, L.acc.bytes, st));
    if (L.arr_cnt.bytes) CK(cudaMemsetAsync(w + L.arr_cnt.off, 0, L.arr_cnt.bytes, st));
    if (L.inb_cnt.bytes) CK(cudaMemsetAsync(w + L.inb_cnt.off, 0, L.inb_cnt.bytes, st));
    Ctrl c;
    std::memset(&c, 0, sizeof(c));
    const bool rec = s->prm.raster_cap > 0 && s->prm.raster_steps > 0;
    for (int k = 0; k < 3; ++k) c.head[k] = rec ? 0 : -1;  // step 0 (and the step before it) write at 0
    CK(cudaMemcpyAsync(w + L.ctrl.off, &c, sizeof(c), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    return SNN_OK;
}

// Launch kernel `half` (0: k_update, 1: k_route) of step ctrl->t + k.  With
// programmatic dependent launch each kernel may be scheduled while the one
// before it drains; it waits (griddepcontrol.wait) before reading.
static cudaError_t launch_half(snn_sim *s, int half, int k, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(half == 0 ? s->grid_update : s->grid_route);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    if (s->pdl) {
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    if (s->arrival) {
        if (half == 0)
            cudaLaunchKernelEx(&cfg, s->vec ? k_update<kModeVec, true> : k_update<kModeScalar, true>, s->dev, k);
        else cudaLaunchKernelEx(&cfg, k_route<true>, s->dev, k);
    } else {
        if (half == 0)
            cudaLaunchKernelEx(&cfg, s->vec ? k_update<kModeVec, false> : k_update<kModeScalar, false>, s->dev, k);
        else cudaLaunchKernelEx(&cfg, k_route<false>, s->dev, k);
    }
    return cudaGetLastError();
}

static cudaError_t launch_step(snn_sim *s, int k, cudaStream_t st)
{
    cudaError_t e = launch_half(s, 0, k, st);
    return e == cudaSuccess ? launch_half(s, 1, k, st) : e;
}

static int capture(snn_sim *s, int steps, cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < steps && le == cudaSuccess; ++k) le = launch_step(s, k, s->cap_stream);
    if (le == cudaSuccess) {
        k_advance<<<1, 1, 0, s->cap_stream>>>(s->dev, steps);
        le = cudaGetLastError();
    }
    cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return SNN_E_CUDA;
    }
    cudaError_t ie = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return ie == cudaSuccess ? SNN_OK : SNN_E_CUDA;
}

extern "C" void snn_sim_destroy(snn_sim *s)
{
    if (!s) return;
    if (s->g1) cudaGraphExecDestroy(s->g1);
    if (s->gU) cudaGraphExecDestroy(s->gU);
    if (s->gP) cudaGraphExecDestroy(s->gP);
    for (cudaEvent_t e : s->pev) cudaEventDestroy(e);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    for (void *p : s->pinned) cudaHostUnregister(p);
    delete s;
}

// Checks of a batch (networks k = 0..n-1 own ids [off[k], off[k+1])): the
// offsets are multiples of 4, no synapse leaves its network, and no
// partition or VN mixes networks.
static int batch_check(const snn_network *net, const snn_routing *rt, int32_t n, const int64_t *off,
                       const snn_sim_params *params)
{
    const int64_t M = rt->M;
    if (n < 1 || n > 65535 || !off || !params || off[0] != 0 || off[n] != M) return SNN_E_ARG;
    for (int32_t k = 0; k < n; ++k) {
        if (off[k + 1] <= off[k] || (off[k] & 3)) return SNN_E_ARG;
        if (!(params[k].drive_lambda >= 0.0) || params[k].drive_lambda > 16.0) return SNN_E_ARG;
    }
    auto net_of = [&](int64_t i) { return (int32_t)(std::upper_bound(off, off + n + 1, i) - off - 1); };
    std::atomic<int> bad{0};
    parallel_for(M, resolve_threads(0), [&](int64_t lo, int64_t hi, int) {
        int32_t k = net_of(lo);
        for (int64_t i = lo; i < hi && !bad.load(std::memory_order_relaxed); ++i) {
            while (i >= off[k + 1]) ++k;
            for (int64_t e = net->syn_ptr[i]; e < net->syn_ptr[i + 1]; ++e)
                if ((int64_t)net->syn_tgt[e] < off[k] || (int64_t)net->syn_tgt[e] >= off[k + 1]) {
                    bad = 1;
                    break;
                }
        }
    });
    if (bad) return SNN_E_ARG;
    // every partition and every VN within one network
    std::vector<int32_t> pnet((size_t)rt->P, -1);
    for (int32_t ip = 0; ip < rt->P; ++ip)
        for (int64_t k = rt->pbase[ip]; k < rt->pbase[ip + 1]; ++k) {
            const int32_t x = net_of((int64_t)rt->perm_inv[k]);
            if (pnet[ip] < 0) pnet[ip] = x;
            else if (pnet[ip] != x) return SNN_E_ARG;
        }
    const int32_t vs = rt->P / rt->n_vn;
    for (int32_t ip = 0; ip < rt->P; ++ip)
        if (pnet[ip] != pnet[(ip / vs) * vs]) return SNN_E_ARG;
    return SNN_OK;
}

static int sim_create(const snn_network *net, const snn_routing *rt, const snn_sim_params *p, int32_t n_net,
                      const int64_t *off, const snn_sim_params *params, void *workspace, size_t ws_bytes,
                      void *stream, snn_sim **out);

extern "C" int snn_sim_create(const snn_network *net, const snn_routing *rt, const snn_sim_params *p,
                              void *workspace, size_t ws_bytes, void *stream, snn_sim **out)
{
    return sim_create(net, rt, p, 0, nullptr, nullptr, workspace, ws_bytes, stream, out);
}

extern "C" int snn_batch_workspace_bytes(const snn_routing *rt, int32_t n, const snn_sim_params *params,
                                         size_t *bytes)
{
    if (!rt || !bytes || n < 1 || !params || !params_ok(&params[0]) || rt->M % 4) return SNN_E_ARG;
    Layout L;
    int rc = make_layout(rt, &params[0], L, n);
    if (rc) return rc;
    *bytes = L.total;
    return SNN_OK;
}

extern "C" int snn_batch_create(const snn_network *net, const snn_routing *rt, int32_t n, const int64_t *off,
                                const snn_sim_params *params, void *workspace, size_t ws_bytes, void *stream,
                                snn_sim **out)
{
    if (!out) return SNN_E_ARG;
    *out = nullptr;
    if (!net || !rt || !params || !params_ok(&params[0]) || net->n_neurons != rt->M) return SNN_E_ARG;
    int rc = batch_check(net, rt, n, off, params);
    if (rc) return rc;
    return sim_create(net, rt, &params[0], n, off, params, workspace, ws_bytes, stream, out);
}

// The k_persist instance of a state-access mode; the minimum-delay
// batching one exists for the shared-memory mode.
static const void *persist_fn(int mode, bool defer, bool arr, int b = 2)
{
    // global neuron state: the instance built for 3 blocks per SM when that
    // many are asked for, else the one for 2
    const bool three = b >= 3;
    if (arr) {
        if (mode == kModeSmem) return (const void *)k_persist<kModeSmem, false, true, 3>;
        if (mode == kModeVec)
            return three ? (const void *)k_persist<kModeVec, false, true, 3> : (const void *)k_persist<kModeVec, false, true, 2>;
        return three ? (const void *)k_persist<kModeScalar, false, true, 3> : (const void *)k_persist<kModeScalar, false, true, 2>;
    }
    if (mode == kModeSmem)
        return defer ? (const void *)k_persist<kModeSmem, true, false, 3> : (const void *)k_persist<kModeSmem, false, false, 3>;
    if (mode == kModeVec)
        return three ? (const void *)k_persist<kModeVec, false, false, 3> : (const void *)k_persist<kModeVec, false, false, 2>;
    return three ? (const void *)k_persist<kModeScalar, false, false, 3> : (const void *)k_persist<kModeScalar, false, false, 2>;
}

// Select the partition-owned kernel with b blocks per SM if that many stay
// resident with the largest partition's accumulator in shared memory.
// Returns whether it was selected (the persistent path then runs k_owner).
static bool shape_owner(snn_sim *s, int b)
{
    if (s->L.n_own == 0 || !s->coop || !s->allow_persist) return false;
    const size_t dyn = (size_t)((s->L.own_max * 4 + 15) / 16 * 16);
    if (cudaFuncSetAttribute((const void *)k_owner, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) !=
        cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int op = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&op, (const void *)k_owner, kThreads, dyn) != cudaSuccess ||
        op < b) {
        cudaGetLastError();
        return false;
    }
    s->persist = true;
    s->owner = true;
    s->persist_bps = b;
    s->grid_persist = (unsigned)std::min<int64_t>((int64_t)s->sms * b, s->L.tally_rows);
    s->owner_smem = dyn;
    return true;
}

// Select the persistent kernel in neuron-state mode `mode` with b blocks per
// SM if that many stay resident (kModeSmem: and the block's quads fit in its
// shared memory).  Returns whether it was selected.
static bool shape_persist(snn_sim *s, int mode, int b)
{
    const snn_routing *rt = s->rt;
    const int64_t grid = std::min<int64_t>((int64_t)s->sms * b, s->L.tally_rows);
    size_t dyn = 0;
    int64_t cq = 0;
    const void *fn = persist_fn(mode, s->defer, s->arrival, b);
    if (mode != kModeScalar && !s->vec) return false;
    if (mode == kModeSmem) {
        int smax = 0;
        cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
        cq = (rt->M / 4 + grid - 1) / grid;
        dyn = (size_t)cq * 52;  // V, ring slot, drive (16 B per quad each), refractory counters (4)
        if (dyn > (size_t)smax ||
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    }
    int op = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&op, fn, kThreads, dyn) != cudaSuccess || op < b) {
        cudaGetLastError();
        return false;
    }
    s->persist = true;
    s->owner = false;
    s->pmode = mode;
    s->persist_bps = b;
    s->grid_persist = (unsigned)grid;
    s->persist_smem = dyn;
    s->chunk_q = cq;
    s->dev.chunk_q = cq;
    return true;
}

static int sim_create(const snn_network *net, const snn_routing *rt, const snn_sim_params *p, int32_t n_net,
                      const int64_t *off, const snn_sim_params *params, void *workspace, size_t ws_bytes,
                      void *stream, snn_sim **out)
{
    if (!out) return SNN_E_ARG;
    *out = nullptr;
    if (!net || !rt || !params_ok(p) || !workspace) return SNN_E_ARG;
    if (net->n_neurons != rt->M || net->syn_ptr[net->n_neurons] != rt->E) return SNN_E_ARG;
    if (((uintptr_t)workspace) & 255) return SNN_E_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return SNN_E_NODEV;
    snn_sim *s = new (std::nothrow) snn_sim();
    if (!s) return SNN_E_NOMEM;
    s->rt = rt;
    s->prm = *p;
    if (n_net > 0) {
        // the network of each quad of ids, each network's drive
        try {
            s->net_of_h.resize((size_t)(rt->M / 4));
            for (int32_t k = 0; k < n_net; ++k)
                for (int64_t q = off[k] / 4; q < off[k + 1] / 4; ++q) s->net_of_h[q] = (uint16_t)k;
            s->net_drive_h.assign((size_t)n_net, NetDrive{});
            for (int32_t k = 0; k < n_net; ++k) {
                NetDrive &nd = s->net_drive_h[k];
                finite_thresholds(params[k].drive_lambda, nd.th, &nd.fin);
                nd.key0 = (uint32_t)params[k].drive_seed;
                nd.key1 = (uint32_t)(params[k].drive_seed >> 32);
                nd.off = off[k];
            }
        } catch (const std::bad_alloc &) {
            delete s;
            return SNN_E_NOMEM;
        }
    }
    int rc = make_layout(rt, p, s->L, n_net);
    if (rc) { delete s; return rc; }
    if (ws_bytes < s->L.total) { delete s; return SNN_E_NOMEM; }
    s->ws = (char *)workspace;
    s->stream = (cudaStream_t)stream;
    s->U = p->steps_per_graph;
    if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return SNN_E_CUDA; }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
        delete s;
        return SNN_E_CUDA;
    }
    s->vec = (rt->M % 4) == 0;
    {
        // SNN_PDL=0 launches the step kernels with plain stream order
        const char *e = std::getenv("SNN_PDL");
        s->pdl = !(e && e[0] == '0');
    }
    {
        // fan-out grids: as many blocks as stay resident together
        int o3 = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o3, k_fo_deliver, kThreads, 0) != cudaSuccess) {
            snn_sim_destroy(s);
            return SNN_E_CUDA;
        }
        s->grid_update = (unsigned)step_grid(rt->M);  // one pass over the neurons
        s->grid_route = (unsigned)(sms * std::max(1, o3));
        // persistent path: one cooperative launch, every block resident
        // (SNN_PERSIST=0 selects the CUDA-graph path).  With M % 4 == 0 each
        // block keeps its quads' state in shared memory when that fits at
        // the most blocks per SM that do (SNN_PERSIST_SMEM=0: global state).
        s->sms = sms;
        int coop = 0;
        const char *e = std::getenv("SNN_PERSIST");
        const char *esm = std::getenv("SNN_PERSIST_SMEM");
        // SNN_PERSIST_BLOCKS_PER_SM lowers the resident blocks per SM (tuning)
        const char *bps = std::getenv("SNN_PERSIST_BLOCKS_PER_SM");
        const int bmax = (bps && std::atoi(bps) > 0) ? std::min(4, std::atoi(bps)) : 4;
        s->coop = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->device) == cudaSuccess && coop;
        // minimum-delay batching on the shared-memory persistent shape
        // (SNN_PERSIST_DEFER=1 turns it on as the parameter does: tests)
        const char *edf = std::getenv("SNN_PERSIST_DEFER");
        s->defer = p->defer_delayed != 0 || (edf && edf[0] == '1');
        s->allow_persist = !(e && e[0] == '0') && s->coop;
        s->allow_smem = !(esm && esm[0] == '0');
        if (s->allow_persist) {
            if (s->allow_smem)
                for (int b = bmax; b >= 1 && !s->persist; --b) shape_persist(s, kModeSmem, b);
            for (int b = bmax; b >= 1 && !s->persist; --b) shape_persist(s, s->vec ? kModeVec : kModeScalar, b);
        }
        cudaGetLastError();
        // tests of the bounded barrier wait: a shorter bound, and block 0
        // skipping its first arrival so that the others' wait runs out
        const char *lim = std::getenv("SNN_BARRIER_LIMIT_NS");
        if (lim && std::strtoull(lim, nullptr, 10) > 0) s->barrier_limit_ns = std::strtoull(lim, nullptr, 10);
        const char *skip = std::getenv("SNN_TEST_SKIP_BARRIER");
        s->test_skip_arrival = (skip && skip[0] == '1') ? 1 : 0;
    }
    if (cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return SNN_E_CUDA;
    }
    if (p->pin_host_tables) {
        auto pin = [&](const void *ptr, size_t bytes) {
            if (ptr && bytes && cudaHostRegister((void *)ptr, bytes, cudaHostRegisterDefault) == cudaSuccess)
                s->pinned.push_back((void *)ptr);
            else
                cudaGetLastError();
        };
        pin(rt->syn_td.data(), s->L.syn_td.bytes);
        pin(rt->syn_w.data(), s->L.syn_w.bytes);
        pin(rt->l2.data(), s->L.l2.bytes);
        pin(rt->l2_pair.data(), s->L.l2_pair.bytes);
        pin(rt->l1_vn.data(), s->L.l1_vn.bytes);
        pin(rt->l1_l2.data(), s->L.l1_l2.bytes);
        pin(rt->l1_pair.data(), s->L.l1_pair.bytes);
        pin(rt->l1_ptr.data(), s->L.l1_ptr.bytes);
        pin(rt->csr.data(), s->L.csr.bytes);
    }
    // device view
    const Layout &L = s->L;
    char *w = s->ws;
    Dev &d = s->dev;
    std::memset(&d, 0, sizeof(d));
    d.V = (float *)(w + L.V.off);
    d.ref = (uint8_t *)(w + L.ref.off);
    d.ring = (int32_t *)(w + L.ring.off);
    d.gid = rt->identity ? nullptr : (const uint32_t *)(w + L.gid.off);
    d.src_part = (const uint16_t *)(w + L.src_part.off);
    d.row = (const uint2 *)(w + L.row.off);
    d.csr = (const unsigned long long *)(w + L.csr.off);
    d.l1_pair = (const uint32_t *)(w + L.l1_pair.off);
    d.l2_pair = (const uint32_t *)(w + L.l2_pair.off);
    d.syn_td = (const uint32_t *)(w + L.syn_td.off);
    d.syn_w = (const int16_t *)(w + L.syn_w.off);
    d.l1_ptr = (const uint32_t *)(w + L.l1_ptr.off);
    d.l1_vn = (const uint16_t *)(w + L.l1_vn.off);
    d.l1_l2 = (const uint32_t *)(w + L.l1_l2.off);
    d.l2 = (const DevL2 *)(w + L.l2.off);
    d.bucket = (uint32_t *)(w + L.bucket.off);
    d.bucket_slot = (const ulonglong2 *)(w + L.bucket_slot.off);
    d.bucket_cnt = (uint32_t *)(w + L.bucket_cnt.off);
    d.inbox = (unsigned long long *)(w + L.inbox.off);
    d.inbox_slot = (const ulonglong2 *)(w + L.inbox_slot.off);
    d.inbox_cnt = (uint32_t *)(w + L.inbox_cnt.off);
    d.tally = (unsigned long long *)(w + L.tally.off);
    d.spk = (uint32_t *)(w + L.spk.off);
    d.spk_step = (uint32_t *)(w + L.spk_step.off);
    d.raster_off = (long long *)(w + L.raster_off.off);
    d.hash = (unsigned long long *)(w + L.hash.off);
    d.cur_rec = (int32_t *)(w + L.cur_rec.off);
    d.counters = (unsigned long long *)(w + L.counters.off);
    d.ctrl = (Ctrl *)(w + L.ctrl.off);
    d.M = rt->M;
    d.P = rt->P;
    d.n_vn = rt->n_vn;
    d.vn_size = rt->P / rt->n_vn;
    d.chunk_q = s->chunk_q;
    d.n_bpair = (int)rt->bpair_cap.size();
    d.n_ipair = (int)rt->ipair_cap.size();
    d.D = L.D;
    d.alpha = (float)std::exp(-p->dt_ms / p->tau_ms);
    d.e_l = p->e_l;
    d.v_th = p->v_th;
    d.v_reset = p->v_reset;
    d.t_ref = p->t_ref;
    d.w_ext = p->w_ext;
    d.i_bias = p->i_bias;
    d.key0 = (uint32_t)p->drive_seed;
    d.key1 = (uint32_t)(p->drive_seed >> 32);
    d.raster_cap = p->raster_cap;
    d.raster_steps = p->raster_steps;
    d.hash_steps = p->hash_steps;
    d.cur_every = p->cur_every;
    d.cur_slots = p->cur_slots;
    {
        // SNN_VEC_PIECES=1: staged pieces delivered with 16-byte / 8-byte loads
        const char *e = std::getenv("SNN_VEC_PIECES");
        d.vec_pieces = (e && e[0] == '1') ? 1 : 0;
        // SNN_BAR_GROUPS=G (2..16): two-level grid-barrier arrival over G groups
        const char *eb = std::getenv("SNN_BAR_GROUPS");
        const int g = eb ? std::atoi(eb) : 0;
        d.bar_groups = (g > 1) ? std::min(g, kBarGroups) : 0;
        // SNN_PREFETCH_STATE=0 turns off the next-step state prefetch (global state)
        const char *ep = std::getenv("SNN_PREFETCH_STATE");
        d.prefetch_state = (ep && ep[0] == '0') ? 0 : 1;
        // queued runs delivered through asynchronous copies (SNN_ASYNC_RECORDS=0: plain loads)
        const char *ea = std::getenv("SNN_ASYNC_RECORDS");
        d.async_rec = (ea && ea[0] == '0') ? 0 : 1;
    }
    if (L.n_arr > 0 || L.n_own > 0) d.dcnt = (const uint4 *)(w + L.dcnt.off);
    if (L.n_own > 0) {
        d.inb = (unsigned long long *)(w + L.inb.off);
        d.inb_slot = (const ulonglong2 *)(w + L.inb_slot.off);
        d.inb_cnt = (uint32_t *)(w + L.inb_cnt.off);
        d.pbase = (const long long *)(w + L.pbase.off);
        d.n_own = L.n_own;
    }
    if (L.n_arr > 0) {
        d.acc = (int32_t *)(w + L.acc.off);
        d.arr = (unsigned long long *)(w + L.arr.off);
        d.arr_cnt = (uint32_t *)(w + L.arr_cnt.off);
        d.arr_cap = L.arr_cap;
        // SNN_DELIVER_AUTO starts with delivery by arrival step (snn_autotune
        // may switch); minimum-delay batching (SNN_PERSIST_DEFER) keeps the ring
        s->arrival = !s->defer;
    }
    d.n_arr = s->arrival ? L.n_arr : 0;
    if (s->arrival && s->persist) {
        // the persistent shape again, for its instance with delivery by arrival step
        const int m = s->pmode, b = s->persist_bps;
        s->persist = false;
        for (int bb = b; bb >= 1 && !s->persist; --bb) shape_persist(s, m, bb);
        cudaGetLastError();
    }
    if (effective_delivery(p) == SNN_DELIVER_OWNER && !s->defer) {
        // partition-owned delivery asked for: its persistent kernel, or an error
        const bool prev = s->persist;
        s->persist = false;
        if (!shape_owner(s, 2) && !shape_owner(s, 1)) {
            s->persist = prev;
            snn_sim_destroy(s);
            return SNN_E_RANGE;
        }
    }
    finite_thresholds(p->drive_lambda, d.th32, &d.th_fin);
    if (L.n_net > 0) {
        d.net_of = (const uint16_t *)(w + L.net_of.off);
        d.net_drive = (const NetDrive *)(w + L.net_drive.off);
    }

    {
        // the worst case per spike of snn_deliver_spikes_static: the longest
        // level-1 row and the most level-2 entries of a neuron
        int64_t m1 = 0, m2 = 0;
        for (int64_t k = 0; k < rt->M; ++k) {
            const uint32_t a = rt->l1_ptr[k], b = rt->l1_ptr[k + 1];
            m1 = std::max<int64_t>(m1, (int64_t)(b - a));
            m2 = std::max<int64_t>(m2, (int64_t)rt->l1_l2[b] - (int64_t)rt->l1_l2[a]);
        }
        s->static_row_l1 = m1;
        s->static_row_l2 = m2;
    }
    rc = upload_tables(s);
    if (!rc) rc = reset_state(s);
    if (rc) {
        snn_sim_destroy(s);
        return rc;
    }
    *out = s;
    return SNN_OK;
}

static int launch_persist(snn_sim *s, int32_t T, const Dev &d)
{
    unsigned long long lim = s->barrier_limit_ns;
    const void *fn = s->owner ? (const void *)k_owner : persist_fn(s->pmode, s->defer, s->arrival, s->persist_bps);
    const size_t smem = s->owner ? s->owner_smem : s->persist_smem;
    // a launch's barrier arrivals (2 per step per block) stay below 2^32
    const int32_t cap = (int32_t)std::min<unsigned long long>(
        0x7FFFFFFFull, (0xFFFFFFFFull / (2ull * s->grid_persist)) - 1ull);
    while (T > 0) {
        int tt = std::min(T, cap);
        int skip = s->test_skip_arrival;
        s->test_skip_arrival = 0;  // once: the test checks the first launch's status
        void *args[] = {(void *)&d, (void *)&tt, (void *)&lim, (void *)&skip};
        // the grid barrier counts arrivals from zero in every launch
        CK(cudaMemsetAsync(s->ws + s->L.ctrl.off + offsetof(Ctrl, bar), 0, sizeof(Ctrl) - offsetof(Ctrl, bar),
                           s->stream));
        CK(cudaLaunchCooperativeKernel(fn, dim3(s->grid_persist), dim3(kThreads), args, smem, s->stream));
        T -= tt;
    }
    return SNN_OK;
}

extern "C" int snn_step(snn_sim *s, int32_t T)
{
    if (!s || T < 0) return SNN_E_ARG;
    if (s->persist) return launch_persist(s, T, s->dev);
    if (!s->g1) {
        int rc = capture(s, 1, &s->g1);
        if (!rc && s->U > 1) rc = capture(s, s->U, &s->gU);
        if (rc) return rc;
    }
    int32_t n = T;
    if (s->gU)
        for (; n >= s->U; n -= s->U) CK(cudaGraphLaunch(s->gU, s->stream));
    for (; n > 0; --n) CK(cudaGraphLaunch(s->g1, s->stream));
    return SNN_OK;
}

extern "C" int snn_profile_phases(snn_sim *s, int32_t T, double *phase_ms)
{
    if (!s || T < 0 || !phase_ms) return SNN_E_ARG;
    for (int k = 0; k < kPhases; ++k) phase_ms[k] = 0.0;
    if (s->persist) {
        // block 0 sums the parts of each step with the GPU's global timer
        Dev dp = s->dev;
        dp.phase_ns = (unsigned long long *)(s->ws + s->L.phase_ns.off);
        CK(cudaMemsetAsync(dp.phase_ns, 0, kPhases * sizeof(unsigned long long), s->stream));
        int rc = launch_persist(s, T, dp);
        if (rc) return rc;
        unsigned long long ns[kPhases];
        CK(cudaMemcpyAsync(ns, dp.phase_ns, sizeof(ns), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        for (int k = 0; k < kPhases; ++k) phase_ms[k] = ns[k] * 1e-6;
        return SNN_OK;
    }
    if (!s->gP) {
        // a graph of U steps with an event-record node before, between and
        // after the two step kernels of every step (cudaEventRecordExternal: a
        // plain record inside a capture only orders streams)
        const int U = 16;
        s->pev.resize((size_t)U * 3);
        for (auto &e : s->pev) CK(cudaEventCreate(&e));
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t le = cudaSuccess;
        const unsigned fl = cudaEventRecordExternal;
        for (int k = 0; k < U && le == cudaSuccess; ++k) {
            le = cudaEventRecordWithFlags(s->pev[3 * k], s->cap_stream, fl);
            if (le == cudaSuccess) le = launch_half(s, 0, k, s->cap_stream);
            if (le == cudaSuccess) le = cudaEventRecordWithFlags(s->pev[3 * k + 1], s->cap_stream, fl);
            if (le == cudaSuccess) le = launch_half(s, 1, k, s->cap_stream);
            if (le == cudaSuccess) le = cudaEventRecordWithFlags(s->pev[3 * k + 2], s->cap_stream, fl);
        }
        if (le == cudaSuccess) {
            k_advance<<<1, 1, 0, s->cap_stream>>>(s->dev, U);
            le = cudaGetLastError();
        }
        cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &g);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return SNN_E_CUDA;
        }
        cudaError_t ie = cudaGraphInstantiate(&s->gP, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return SNN_E_CUDA;
        s->UP = U;
    }
    int32_t left = T;
    while (left > 0) {
        // whole instrumented graphs, then plain single steps for the remainder
        if (left >= s->UP) {
            CK(cudaGraphLaunch(s->gP, s->stream));
            CK(cudaStreamSynchronize(s->stream));
            for (int k = 0; k < s->UP; ++k) {
                float a = 0.f, b = 0.f;
                CK(cudaEventElapsedTime(&a, s->pev[3 * k], s->pev[3 * k + 1]));
                CK(cudaEventElapsedTime(&b, s->pev[3 * k + 1], s->pev[3 * k + 2]));
                phase_ms[0] += a;
                phase_ms[4] += b;
            }
            left -= s->UP;
        } else {
            int rc = snn_step(s, left);
            if (rc) return rc;
            CK(cudaStreamSynchronize(s->stream));
            left = 0;
        }
    }
    return SNN_OK;
}

// ---------------------------------------------------------------- launch-shape autotuner
static int read_ctrl(snn_sim *s, Ctrl *c);

// A copy of a sim's dynamic state (snn_autotune): neuron state, delay ring,
// counters, tally rows, the hash slots from the current step on and the
// control word, taken after the queued runs of delivery by arrival step or
// by owner were moved into the ring (as a checkpoint does).  Restoring it
// puts the sim back at that step with its records intact.
struct Snapshot {
    std::vector<char> v, ref, ring, counters, tally, hash;
    Ctrl ctrl;
    long long t = 0;
};

static int materialize_queued(snn_sim *s, long long t);

static int snapshot_take(snn_sim *s, Snapshot &sn)
{
    const Layout &L = s->L;
    Ctrl c;
    int rc = read_ctrl(s, &c);
    if (rc) return rc;
    rc = materialize_queued(s, c.t);
    if (rc) return rc;
    rc = read_ctrl(s, &sn.ctrl);
    if (rc) return rc;
    sn.t = sn.ctrl.t;
    // the ring now holds every pending input of steps t .. t + D - 1, which
    // any delivery mode restored from the snapshot consumes
    sn.ctrl.inject_until = sn.t + L.D;
    auto take = [&](std::vector<char> &b, const Region &r, size_t off, size_t bytes) -> cudaError_t {
        b.resize(bytes);
        return bytes ? cudaMemcpy(b.data(), s->ws + r.off + off, bytes, cudaMemcpyDeviceToHost) : cudaSuccess;
    };
    CK(take(sn.v, L.V, 0, L.V.bytes));
    CK(take(sn.ref, L.ref, 0, L.ref.bytes));
    CK(take(sn.ring, L.ring, 0, L.ring.bytes));
    CK(take(sn.counters, L.counters, 0, L.counters.bytes));
    CK(take(sn.tally, L.tally, 0, L.tally.bytes));
    const long long h0 = std::min<long long>(sn.t, s->prm.hash_steps);
    CK(take(sn.hash, L.hash, (size_t)h0 * 16, (size_t)(s->prm.hash_steps - h0) * 16));
    return SNN_OK;
}

static int snapshot_restore(snn_sim *s, const Snapshot &sn)
{
    const Layout &L = s->L;
    char *w = s->ws;
    CK(cudaStreamSynchronize(s->stream));
    auto put = [&](const std::vector<char> &b, const Region &r, size_t off) -> cudaError_t {
        return b.empty() ? cudaSuccess : cudaMemcpy(w + r.off + off, b.data(), b.size(), cudaMemcpyHostToDevice);
    };
    CK(put(sn.v, L.V, 0));
    CK(put(sn.ref, L.ref, 0));
    CK(put(sn.ring, L.ring, 0));
    CK(put(sn.counters, L.counters, 0));
    CK(put(sn.tally, L.tally, 0));
    CK(put(sn.hash, L.hash, (size_t)std::min<long long>(sn.t, s->prm.hash_steps) * 16));
    CK(cudaMemcpy(w + L.ctrl.off, &sn.ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice));
    for (const Region *r : {&L.acc, &L.arr_cnt, &L.inb_cnt, &L.bucket_cnt, &L.inbox_cnt})
        if (r->bytes) CK(cudaMemset(w + r->off, 0, r->bytes));
    return SNN_OK;
}

// Turn delivery by arrival step on or off (the workspace holds its regions);
// captured graphs hold the old device view and are dropped.  The owner
// kernel is chosen by shape_owner; any other shape turns it off.
static void set_arrival(snn_sim *s, bool on)
{
    s->owner = false;
    on = on && s->L.n_arr > 0 && !s->defer;
    if (on == s->arrival) return;
    s->arrival = on;
    s->dev.n_arr = on ? s->L.n_arr : 0;
    for (cudaGraphExec_t *g : {&s->g1, &s->gU, &s->gP})
        if (*g) {
            cudaGraphExecDestroy(*g);
            *g = nullptr;
        }
}

extern "C" int snn_autotune(snn_sim *s, int32_t steps, int32_t *choice, double *best_ms)
{
    if (!s || steps < 1) return SNN_E_ARG;
    struct Shape {
        bool persist;
        int mode, b;
        bool arrival, owner;
    };
    std::vector<Shape> cand;
    if (s->L.n_own > 0 && !s->defer && s->allow_persist)
        for (int b = 2; b >= 1; --b) cand.push_back({true, 0, b, false, true});
    std::vector<bool> dels{false};
    if (s->L.n_arr > 0 && !s->defer) dels = {true, false};
    for (bool arr : dels) {
        if (s->allow_persist)
            for (int mode : {kModeSmem, kModeVec, kModeScalar})
                for (int b = 4; b >= 1; --b)
                    if (mode != kModeSmem || s->allow_smem) cand.push_back({true, mode, b, arr, false});
        cand.push_back({false, 0, 0, arr, false});
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = 1e300;
    // every shape starts from the sim's current state
    Snapshot snap;
    if (int r0 = snapshot_take(s, snap)) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return r0;
    }
    Shape pick = {s->persist, s->pmode, s->persist_bps, s->arrival, s->owner};
    int rc = SNN_OK;
    for (const Shape &c : cand) {
        set_arrival(s, c.arrival);
        if (c.owner) {
            s->persist = false;
            if (!shape_owner(s, c.b)) continue;
        } else if (c.persist) {
            s->persist = false;
            if (!shape_persist(s, c.mode, c.b)) continue;
        } else {
            s->persist = false;
        }
        // from the sim's state: a quarter of the steps to warm up, then the timed steps
        if ((rc = snapshot_restore(s, snap)) != SNN_OK) break;
        if ((rc = snn_step(s, std::max(1, steps / 4))) != SNN_OK) break;
        if (cudaEventRecord(e0, s->stream) != cudaSuccess) { rc = SNN_E_CUDA; break; }
        if ((rc = snn_step(s, steps)) != SNN_OK) break;
        if (cudaEventRecord(e1, s->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = SNN_E_CUDA;
            break;
        }
        Ctrl ctl;
        if ((rc = read_ctrl(s, &ctl)) != SNN_OK) break;
        if (ctl.status & kStTimeout) continue;  // a shape that cannot run here
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            pick = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->persist = false;
    set_arrival(s, pick.arrival);
    if (pick.owner) shape_owner(s, pick.b);
    else if (pick.persist) shape_persist(s, pick.mode, pick.b);
    const int rr = snapshot_restore(s, snap);
    if (rc == SNN_OK) rc = rr;
    if (choice)
        *choice = pick.owner ? 2000 + pick.b
                             : (pick.persist ? 100 * pick.mode + pick.b : 0) + (pick.arrival ? 1000 : 0);
    if (best_ms) *best_ms = best < 1e300 ? best / steps : -1.0;
    return rc;
}

// Fill the table pointers of a fan-out from the sim's device view.
static FoArgs fanout_tables(const snn_sim *s, const uint32_t *ids, int64_t n, int32_t *out)
{
    FoArgs a;
    std::memset(&a, 0, sizeof(a));
    const Dev &d = s->dev;
    a.ids = ids;
    a.n = n;
    a.fwd = s->rt->identity ? nullptr : (const uint32_t *)(s->ws + s->L.fwd.off);
    a.gid = d.gid;
    a.l1_ptr = d.l1_ptr;
    a.l1_l2 = d.l1_l2;
    a.l2 = d.l2;
    a.syn_td = d.syn_td;
    a.syn_w = d.syn_w;
    a.out = out;
    a.M = d.M;
    return a;
}

// Clear the scratch counters, run the three fan-out kernels on the sim's
// stream, wait, and map the scratch status to an error code.
static int run_fanout(snn_sim *s, const FoArgs &a, uint64_t *counts)
{
    cudaStream_t st = s->stream;
    CK(cudaMemsetAsync(a.cnt, 0, 4 * sizeof(unsigned int), st));
    CK(cudaMemsetAsync(a.ev, 0, sizeof(unsigned long long), st));
    if (a.n > 0) {
        const unsigned g = s->grid_route;
        k_fo_level1<<<g, kThreads, 0, st>>>(a);
        k_fo_level2<<<g, kThreads, 0, st>>>(a);
        k_fo_deliver<<<g, kThreads, 0, st>>>(a);
        CK(cudaGetLastError());
    }
    unsigned int c[4];
    unsigned long long ev = 0;
    CK(cudaMemcpyAsync(c, a.cnt, sizeof(c), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&ev, a.ev, sizeof(ev), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (counts) {
        counts[0] = c[0];
        counts[1] = c[1];
        counts[2] = ev;
    }
    if (c[2] & kFoStId) return SNN_E_ARG;
    if (c[2] & (kFoStBucket | kFoStInbox)) return SNN_E_CAPACITY;
    return SNN_OK;
}

// run_fanout with the sim's device current (the caller's current device is
// restored afterwards).
static int run_fanout_on_device(snn_sim *s, const FoArgs &a, uint64_t *counts)
{
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return SNN_E_CUDA;
    if (prev != s->device && cudaSetDevice(s->device) != cudaSuccess) return SNN_E_CUDA;
    const int rc = run_fanout(s, a, counts);
    if (prev != s->device && cudaSetDevice(prev) != cudaSuccess) return SNN_E_CUDA;
    return rc;
}

extern "C" int snn_deliver_spikes(snn_sim *s, const uint32_t *ids, int64_t n, int32_t *out,
                                  uint64_t *counts)
{
    if (!s || n < 0 || (n > 0 && (!ids || !out))) return SNN_E_ARG;
    FoArgs a = fanout_tables(s, ids, n, out);
    a.bucket = s->dev.bucket;
    a.cap1 = s->L.bucket.bytes / sizeof(uint32_t);
    a.inbox = s->dev.inbox;
    a.cap2 = s->L.inbox.bytes / sizeof(unsigned long long);
    a.cnt = (unsigned int *)(s->ws + s->L.fo_cnt.off);
    a.ev = (unsigned long long *)(s->ws + s->L.fo_cnt.off + 16);
    return run_fanout_on_device(s, a, counts);
}

// ---------------------------------------------------------------- fan-out without allocation
// snn_deliver_spikes_static: the same fan-out as snn_deliver_spikes, but its
// scratch (counters, level-1 list, level-2 list) lives in this fixed device
// array instead of the sim's workspace.  Every GPU that loads the library
// holds the array until the process exits; all calls share it.
constexpr size_t kStaticScratchBytes = (size_t)8 << 20;  // 8 MiB
static __device__ __align__(256) unsigned char g_fanout_scratch[kStaticScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};
}  // namespace

// Device address of g_fanout_scratch on `dev`, looked up once per device with
// that device current (host code only sees a host-side stand-in for the array).
static int static_scratch_address(int dev, void **out)
{
    if (dev < 0 || dev >= kMaxDevices) return SNN_E_RANGE;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        int prev = -1;
        if (cudaGetDevice(&prev) != cudaSuccess) return SNN_E_CUDA;
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return SNN_E_CUDA;
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_fanout_scratch);
        if (prev != dev) cudaSetDevice(prev);
        if (e != cudaSuccess || !p) return SNN_E_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SNN_OK;
}

extern "C" size_t snn_static_scratch_bytes(void)
{
    return kStaticScratchBytes;
}

extern "C" int snn_deliver_spikes_static(snn_sim *s, const uint32_t *ids, int64_t n, int32_t *out,
                                         uint64_t *counts)
{
    if (!s || n < 0 || (n > 0 && (!ids || !out))) return SNN_E_ARG;
    // worst case per spike (s->static_row_l1 / _l2, found when the sim was
    // created): its longest level-1 row and its most level-2 entries
    if (n > (int64_t)kStaticScratchBytes) return SNN_E_RANGE;
    const size_t head = 256;
    const size_t need1 = (((size_t)n * (size_t)s->static_row_l1 * sizeof(uint32_t)) + 255) & ~(size_t)255;
    const size_t need2 = (size_t)n * (size_t)s->static_row_l2 * sizeof(unsigned long long);
    if (head + need1 + need2 > kStaticScratchBytes) return SNN_E_RANGE;
    void *base = nullptr;
    int rc = static_scratch_address(s->device, &base);
    if (rc) return rc;
    char *b = (char *)base;
    FoArgs a = fanout_tables(s, ids, n, out);
    a.cnt = (unsigned int *)b;
    a.ev = (unsigned long long *)(b + 16);
    a.bucket = (uint32_t *)(b + head);
    a.cap1 = need1 / sizeof(uint32_t);
    a.inbox = (unsigned long long *)(b + head + need1);
    a.cap2 = need2 / sizeof(unsigned long long);
    return run_fanout_on_device(s, a, counts);
}

extern "C" int64_t snn_launches(const snn_sim *s, int32_t T)
{
    if (!s || T <= 0) return 0;
    if (s->persist) return 1;
    const int64_t graphs = (s->U > 1 ? T / s->U : 0) + (s->U > 1 ? T % s->U : T);
    return 2 * (int64_t)T + graphs;  // two step kernels + one k_advance per graph
}

extern "C" int64_t snn_launches_per_step(const snn_sim *s)
{
    return s ? 2 : 0;
}

static int read_ctrl(snn_sim *s, Ctrl *c)
{
    CK(cudaMemcpyAsync(c, s->dev.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return SNN_OK;
}

extern "C" int snn_sync_status(snn_sim *s)
{
    if (!s) return SNN_E_ARG;
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    Ctrl c;
    int rc = read_ctrl(s, &c);
    if (rc) return rc;
    if (c.status & kStTimeout) return SNN_E_TIMEOUT;
    if (c.status & (kStBucket | kStInbox | kStArrival)) return SNN_E_CAPACITY;
    return SNN_OK;
}

// Raster read-back: the spikes of step t0 + b (spk[off[b] .. off[b+1]),
// internal ids in the order the blocks reserved them) sorted in place by
// global id (gid; nullptr: the same), one block per step, a bitonic sort in
// shared memory of (global id << 32 | internal id).  Steps with more than
// cap spikes are left to the host.  Sorting again gives the same order.
__global__ void __launch_bounds__(1024) k_raster_sort(uint32_t *spk, const long long *off, const uint32_t *gid,
                                                      int cap)
{
    extern __shared__ unsigned long long keys[];
    const long long a = off[blockIdx.x], b = off[blockIdx.x + 1];
    const int n = (int)(b - a);
    if (n <= 1 || n > cap) return;
    int m = 1;
    while (m < n) m <<= 1;
    for (int x = threadIdx.x; x < m; x += blockDim.x) {
        if (x < n) {
            const uint32_t i = spk[a + x];
            keys[x] = ((unsigned long long)(gid ? gid[i] : i) << 32) | i;
        } else {
            keys[x] = ~0ull;
        }
    }
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int x = threadIdx.x; x < m; x += blockDim.x) {
                const int y = x ^ j;
                if (y > x) {
                    const unsigned long long u = keys[x], v = keys[y];
                    const bool up = (x & k) == 0;
                    if ((u > v) == up) {
                        keys[x] = v;
                        keys[y] = u;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int x = threadIdx.x; x < n; x += blockDim.x) spk[a + x] = (uint32_t)keys[x];
}

extern "C" int snn_read_raster(snn_sim *s, int64_t t0, int64_t t1, uint32_t *ids, int64_t cap,
                               int64_t *step_off, int64_t *n)
{
    if (!s || t0 < 0 || t1 < t0 || !step_off || !n) return SNN_E_ARG;
    *n = -1;
    Ctrl c;
    int rc = read_ctrl(s, &c);
    if (rc) return rc;
    if (t1 > c.rec_steps) return SNN_E_CAPACITY;
    const int64_t nst = t1 - t0;
    std::vector<long long> off((size_t)nst + 1);
    CK(cudaMemcpy(off.data(), s->dev.raster_off + t0, sizeof(long long) * (size_t)(nst + 1),
                  cudaMemcpyDeviceToHost));
    const int64_t tot = off[nst] - off[0];
    *n = tot;
    for (int64_t k = 0; k <= nst; ++k) step_off[k] = off[k] - off[0];
    if (tot > cap || (tot > 0 && !ids)) return tot > cap ? SNN_E_CAPACITY : SNN_E_ARG;
    if (tot > 0) {
        // every step's ids sorted by global id on the device (steps of up to
        // kSortCap spikes), then copied back and mapped to global ids
        constexpr int kSortCap = 8192;
        int64_t widest = 0;
        for (int64_t k = 0; k < nst; ++k) widest = std::max<int64_t>(widest, step_off[k + 1] - step_off[k]);
        const int cap_dev = (int)std::min<int64_t>(kSortCap, widest);
        if (cap_dev > 1) {
            int m = 1;
            while (m < cap_dev) m <<= 1;
            const size_t smem = sizeof(unsigned long long) * (size_t)m;
            CK(cudaFuncSetAttribute(k_raster_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            for (int64_t k0 = 0; k0 < nst; k0 += 65535) {
                const int64_t nb = std::min<int64_t>(65535, nst - k0);
                k_raster_sort<<<(unsigned)nb, 1024, smem, s->stream>>>(
                    s->dev.spk, s->dev.raster_off + t0 + k0, s->rt->identity ? nullptr : s->dev.gid, cap_dev);
                CK(cudaGetLastError());
            }
        }
        CK(cudaMemcpyAsync(ids, s->dev.spk + off[0], sizeof(uint32_t) * (size_t)tot, cudaMemcpyDeviceToHost,
                           s->stream));
        CK(cudaStreamSynchronize(s->stream));
        const uint32_t *inv = s->rt->perm_inv.data();
        for (int64_t k = 0; k < nst; ++k) {
            uint32_t *b = ids + step_off[k], *e = ids + step_off[k + 1];
            if (!s->rt->identity)
                for (uint32_t *x = b; x < e; ++x) *x = inv[*x];
            if (e - b > cap_dev) std::sort(b, e);
        }
    }
    return SNN_OK;
}

extern "C" int snn_read_currents(snn_sim *s, int64_t t, int32_t *out)
{
    if (!s || !out || t < 0) return SNN_E_ARG;
    const snn_sim_params &p = s->prm;
    if (p.cur_every <= 0 || t % p.cur_every || t / p.cur_every >= p.cur_slots) return SNN_E_ARG;
    Ctrl c;
    int rc = read_ctrl(s, &c);
    if (rc) return rc;
    if (t >= c.t) return SNN_E_STATE;
    const int64_t M = s->rt->M;
    std::vector<int32_t> buf((size_t)M);
    CK(cudaMemcpy(buf.data(), s->dev.cur_rec + (t / p.cur_every) * M, sizeof(int32_t) * (size_t)M,
                  cudaMemcpyDeviceToHost));
    const uint32_t *inv = s->rt->perm_inv.data();
    for (int64_t k = 0; k < M; ++k) out[inv[k]] = buf[k];
    return SNN_OK;
}

extern "C" int snn_read_hashes(snn_sim *s, int64_t t0, int64_t t1, uint64_t *cur, uint64_t *v)
{
    if (!s || t0 < 0 || t1 < t0) return SNN_E_ARG;
    if (t1 > s->prm.hash_steps) return SNN_E_CAPACITY;
    std::vector<unsigned long long> h((size_t)(2 * (t1 - t0)));
    if (t1 > t0) {
        CK(cudaStreamSynchronize(s->stream));
        CK(cudaMemcpy(h.data(), s->dev.hash + 2 * t0, sizeof(unsigned long long) * h.size(),
                      cudaMemcpyDeviceToHost));
    }
    for (int64_t k = 0; k < t1 - t0; ++k) {
        if (cur) cur[k] = h[2 * k];
        if (v) v[k] = h[2 * k + 1];
    }
    return SNN_OK;
}

// Totals of the counters: the closing thread's slots plus every block's
// tally row.
static int read_counters(snn_sim *s, unsigned long long *c)
{
    const Layout &L = s->L;
    std::vector<unsigned long long> rows((size_t)L.tally_rows * C_N);
    CK(cudaMemcpyAsync(c, s->dev.counters, sizeof(unsigned long long) * C_N, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(rows.data(), s->dev.tally, sizeof(unsigned long long) * rows.size(), cudaMemcpyDeviceToHost,
                       s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (int64_t r = 0; r < L.tally_rows; ++r)
        for (int k = 0; k < C_N; ++k) c[k] += rows[(size_t)r * C_N + k];
    return SNN_OK;
}

extern "C" int snn_read_counts(snn_sim *s, snn_counts *o)
{
    if (!s || !o) return SNN_E_ARG;
    unsigned long long c[C_N];
    int rc = read_counters(s, c);
    if (rc) return rc;
    o->steps = c[C_STEPS];
    o->spikes = c[C_SPIKES];
    o->events = c[C_EVENTS];
    o->l1_local = c[C_L1_LOCAL];
    o->l1_xvn = c[C_L1_XVN];
    o->l2_local = c[C_L2_BASE + kClsLocal];
    o->l2_peer = c[C_L2_BASE + kClsPeer];
    o->l2_relay_local = c[C_L2_BASE + kClsRelayLocal];
    o->l2_relay_remote = c[C_L2_BASE + kClsRelayRemote];
    o->direct = o->l2_peer + o->l2_relay_local + o->l2_relay_remote;
    o->direct_xvn = o->l2_relay_local + o->l2_relay_remote;
    return SNN_OK;
}

extern "C" int snn_read_state(snn_sim *s, float *V, uint8_t *ref, int64_t *t)
{
    if (!s) return SNN_E_ARG;
    const int64_t M = s->rt->M;
    const uint32_t *inv = s->rt->perm_inv.data();
    CK(cudaStreamSynchronize(s->stream));
    if (V) {
        std::vector<float> b((size_t)M);
        CK(cudaMemcpy(b.data(), s->dev.V, sizeof(float) * (size_t)M, cudaMemcpyDeviceToHost));
        for (int64_t k = 0; k < M; ++k) V[inv[k]] = b[k];
    }
    if (ref) {
        std::vector<uint8_t> b((size_t)M);
        CK(cudaMemcpy(b.data(), s->dev.ref, (size_t)M, cudaMemcpyDeviceToHost));
        for (int64_t k = 0; k < M; ++k) ref[inv[k]] = b[k];
    }
    if (t) {
        Ctrl c;
        int rc = read_ctrl(s, &c);
        if (rc) return rc;
        *t = c.t;
    }
    return SNN_OK;
}

extern "C" int snn_read_inbox_pairs(snn_sim *s, uint64_t *pairs, int64_t cap, int64_t *n)
{
    if (!s || !n) return SNN_E_ARG;
    const snn_routing *rt = s->rt;
    const Layout &L = s->L;
    CK(cudaStreamSynchronize(s->stream));
    // the last step's inbox fill counts (its step parity), one per exchange pair
    Ctrl c;
    int rc = read_ctrl(s, &c);
    if (rc) return rc;
    const int pl = (int)((c.t + 1) & 1);  // parity of step t - 1
    const size_t n_ip = rt->ipair_cap.size();
    std::vector<uint32_t> cnt(n_ip * kPairStride);
    if (n_ip)
        CK(cudaMemcpy(cnt.data(), s->dev.inbox_cnt + (size_t)pl * n_ip * kPairStride, sizeof(uint32_t) * cnt.size(),
                      cudaMemcpyDeviceToHost));
    int64_t tot = 0;
    for (int32_t ip = 0; ip < rt->P; ++ip) {
        for (uint32_t k = rt->ipair_ptr[ip]; k < rt->ipair_ptr[ip + 1]; ++k) {
            const uint32_t m = std::min(cnt[(size_t)k * kPairStride], L.inbox_cap_h[k]);
            if (m == 0) continue;
            const int32_t q = rt->ipair_dst[k];
            std::vector<unsigned long long> ent(m);
            CK(cudaMemcpy(ent.data(), s->dev.inbox + L.inbox_base_h[k], sizeof(unsigned long long) * m,
                          cudaMemcpyDeviceToHost));
            for (uint32_t x = 0; x < m; ++x) {
                const int64_t off = (int64_t)(ent[x] >> kLenBits);
                const int64_t i = std::upper_bound(rt->csr.begin(), rt->csr.end(), off) - rt->csr.begin() - 1;
                if (pairs && tot < cap)
                    pairs[tot] = ((uint64_t)rt->perm_inv[i] << 32) | (uint32_t)rt->part_of_ip[q];
                ++tot;
            }
        }
    }
    *n = tot;
    return SNN_OK;
}

// checkpoint image: header, V, ref, ring, counters
namespace {
struct CkptHeader {
    uint64_t magic;
    int64_t M;
    int32_t D, pad;
    long long t;
};
constexpr uint64_t kCkptMagic = 0x534E4E434B505431ULL;
}  // namespace

// Move the runs queued by delivery by arrival step or by owner, and the
// input slot, into the delay ring (next step t), so that the ring and the
// neuron state are the whole dynamic state; steps < t + D then consume the
// ring slots (Ctrl::inject_until).  Nothing to do with ring delivery.
static int materialize_queued(snn_sim *s, long long t)
{
    const Layout &L = s->L;
    if (!s->arrival && !s->owner) return SNN_OK;
    if (s->arrival) {
        const unsigned g = (unsigned)std::max(1, s->sms * 4);
        k_materialize<<<g, kThreads, 0, s->stream>>>(s->dev, t);
        CK(cudaGetLastError());
        CK(cudaMemsetAsync(s->ws + L.arr_cnt.off, 0, L.arr_cnt.bytes, s->stream));
    } else {
        const unsigned g = (unsigned)std::max(1, std::min(s->rt->P, s->sms * 4));
        k_materialize_owner<<<g, kThreads, 0, s->stream>>>(s->dev, t);
        CK(cudaGetLastError());
        CK(cudaMemsetAsync(s->ws + L.inb_cnt.off, 0, L.inb_cnt.bytes, s->stream));
    }
    const long long until = t + L.D;
    CK(cudaMemcpyAsync(s->ws + L.ctrl.off + offsetof(Ctrl, inject_until), &until, sizeof(until),
                       cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return SNN_OK;
}

extern "C" int snn_state_bytes(snn_sim *s, size_t *bytes)
{
    if (!s || !bytes) return SNN_E_ARG;
    const Layout &L = s->L;
    *bytes = sizeof(CkptHeader) + L.V.bytes + L.ref.bytes + L.ring.bytes + L.counters.bytes;
    return SNN_OK;
}

extern "C" int snn_save_state(snn_sim *s, void *buf, size_t capb)
{
    size_t need = 0;
    if (snn_state_bytes(s, &need) || !buf || capb < need) return SNN_E_ARG;
    Ctrl c;
    int rc = read_ctrl(s, &c);
    if (rc) return rc;
    const Layout &L = s->L;
    rc = materialize_queued(s, (long long)c.t);
    if (rc) return rc;
    char *b = (char *)buf;
    CkptHeader h{kCkptMagic, s->rt->M, L.D, 0, c.t};
    std::memcpy(b, &h, sizeof(h));
    b += sizeof(h);
    for (const Region *r : {&L.V, &L.ref, &L.ring}) {
        CK(cudaMemcpy(b, s->ws + r->off, r->bytes, cudaMemcpyDeviceToHost));
        b += r->bytes;
    }
    unsigned long long tot[C_N];
    rc = read_counters(s, tot);
    if (rc) return rc;
    std::memcpy(b, tot, sizeof(tot));
    return SNN_OK;
}

extern "C" int snn_load_state(snn_sim *s, const void *buf, size_t bytes)
{
    size_t need = 0;
    if (snn_state_bytes(s, &need) || !buf || bytes < need) return SNN_E_ARG;
    const Layout &L = s->L;
    const char *b = (const char *)buf;
    CkptHeader h;
    std::memcpy(&h, b, sizeof(h));
    if (h.magic != kCkptMagic || h.M != s->rt->M || h.D != L.D) return SNN_E_ARG;
    b += sizeof(h);
    CK(cudaStreamSynchronize(s->stream));
    for (const Region *r : {&L.V, &L.ref, &L.ring, &L.counters}) {
        CK(cudaMemcpy(s->ws + r->off, b, r->bytes, cudaMemcpyHostToDevice));
        b += r->bytes;
    }
    CK(cudaMemset(s->dev.tally, 0, L.tally.bytes));
    Ctrl c;
    std::memset(&c, 0, sizeof(c));
    c.t = h.t;
    // delivery by arrival step: the ring holds the restored partial sums of
    // steps h.t .. h.t + D - 1, which those steps consume
    c.inject_until = (s->arrival || s->owner) ? h.t + L.D : 0;
    for (int k = 0; k < 3; ++k) c.head[k] = -1;  // records restart empty and stay off after a restore
    CK(cudaMemcpy(s->dev.ctrl, &c, sizeof(c), cudaMemcpyHostToDevice));
    if (h.t < s->prm.hash_steps)
        CK(cudaMemset(s->dev.hash + 2 * h.t, 0, sizeof(unsigned long long) * 2 * (size_t)(s->prm.hash_steps - h.t)));
    CK(cudaMemset(s->dev.bucket_cnt, 0, L.bucket_cnt.bytes));
    CK(cudaMemset(s->dev.inbox_cnt, 0, L.inbox_cnt.bytes));
    if (L.acc.bytes) CK(cudaMemset(s->ws + L.acc.off, 0, L.acc.bytes));
    if (L.arr_cnt.bytes) CK(cudaMemset(s->ws + L.arr_cnt.off, 0, L.arr_cnt.bytes));
    if (L.inb_cnt.bytes) CK(cudaMemset(s->ws + L.inb_cnt.off, 0, L.inb_cnt.bytes));
    return SNN_OK;
}

extern "C" int snn_sim_reset(snn_sim *s, int32_t reupload)
{
    if (!s) return SNN_E_ARG;
    if (reupload) {
        int rc = upload_tables(s);
        if (rc) return rc;
    }
    return reset_state(s);
}
