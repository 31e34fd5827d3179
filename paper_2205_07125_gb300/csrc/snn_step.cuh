// Step kernels of one simulation step t (sm_103a), included by snn_sim.cu.
//
// The routing is the paper's two-level route (arXiv 2205.07125, Sec. IV.B);
// the neuron model is LIF (Table I); the arithmetic follows the library's
// documented readings (include/snn.h).  A step has two halves, each block
// taking an equal share of the work in both:
//   a1 consume ring slot t mod D, Poisson drive (Philox4x32-10, inverse CDF);
//   a2 FP32 LIF update + threshold (no FMA, fixed order);
//   a3 warp-scan / block-scan compaction of the spikes into the step's spike
//      list (one reservation per block);
//   -- grid-wide synchronisation: the list is complete --
//   a4 level-1 bucketing of an equal share of the list per block, the
//      level-1 and level-2 entries of a round of spikes spread over the
//      block's threads: each spike's entry is appended to the bucket of every
//      destination VN in its level-1 row (one entry per VN: deduplicated);
//   a5 level-2 relay expansion: every (spike, VN) entry becomes an inbox
//      entry of each partition of that VN holding targets;
//   a6 delivery of the round: the level-2 segments are staged in shared
//      memory (long segments cut into 128-synapse pieces, one warp each;
//      short ones walked by one lane) and every synapse adds its int16
//      weight with a 32-bit reduction into ring[(t + d) mod D][target];
//   -- grid-wide synchronisation: step t + 1 may read its ring slot --
// Splitting the list evenly keeps a block that found many spikes from
// holding up the step.  Delivery of step t writes only slots t+1 .. t+D-1
// (D = max delay + 1), never the slot step t reads.  Exchange fill counters
// are kept twice, by step parity: step t fills parity t & 1 and clears the
// other one, which only step t - 1 used.  The spike counts and raster heads
// of steps rotate through three slots (a step's slot is read during the
// next step, cleared during the one after).
//
// Two ways to run: k_persist, one cooperative launch for T steps with
// bounded grid barriers (each split into arrival and wait, with work that
// needs no other block in between), and the CUDA-graph path, k_update and
// k_route per step with programmatic dependent launch.  k_persist<kModeSmem,
// true> adds minimum-delay batching: the delay >= 2 synapses of a step are
// delivered during the next step's table walk.
#pragma once

#include <cuda_runtime.h>

#include "snn_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kPTab = 32;
constexpr int kLongCap = 512;   // staged pieces of one routing round
constexpr int kShortCap = 1024; // staged short segments of one routing round
constexpr int kRound = 16;      // spikes routed per round (<= 32)
constexpr int kOwn = 64;        // own spikes of a step whose tables a block prefetches
// Exchange fill counters are keyed by (source partition, destination) pair,
// so each sees only the spikes of one source partition, and each owns a
// 128-byte line: the counters of one partition then spread over many L2
// slices instead of queueing in a few.
constexpr int kPairStride = 32;

// status bits
constexpr uint32_t kStBucket = 1u, kStInbox = 2u, kStRaster = 4u, kStTimeout = 8u, kStArrival = 16u;

// Delivery by arrival step (Dev::n_arr > 0): a step delivers only into the
// input slot of the next step.  The delay-1 runs of its segments go there at
// once; the run of delay d >= 2 is queued on the list of step t + d - 1 and
// delivered by that step.  Runs staged in shared memory per routing round
// before one reservation per list and round: kArrPool runs, kMaxArr lists.
constexpr int kArrPool = 2048;
constexpr int kMaxArr = 8;

// Routing variants of a step: every delay into the delay ring (or the
// deferred lists), delivery by arrival step, delivery into the destination
// partition's own input (k_owner: every run queued on its partition's list
// of its arrival step, nothing delivered during the routing).
enum { kRtRing = 0, kRtArrival = 1, kRtOwner = 2 };

// Parts of a step timed by block 0 of k_persist (snn_profile_phases): the
// update of the neurons (a1-a2) and their spike compaction (a3), the
// prefetch of the block's own spikes' tables and its queued deliveries, the
// rest of the first barrier's wait, the routing walk (a4-a5) and the
// routing rounds' deliveries and copies (a6), the next step's input-free
// update with the second barrier's wait.
constexpr int kPhases = 7;

// counter slots: steps and spikes in Dev::counters (closing thread), the
// others in each block's tally row
enum { C_STEPS = 0, C_SPIKES, C_EVENTS, C_L1_LOCAL, C_L1_XVN, C_L2_BASE /* + cls (4) */, C_N = 16 };
constexpr int kTally = 7;  // slots C_EVENTS .. C_L2_BASE + 3, consecutive

constexpr int kBarGroups = 16;  // groups of the two-level grid-barrier arrival

struct Ctrl {
    long long t;              // next step to run
    long long head[3];        // raster write head of step t at slot t mod 3 (-1: recording stopped)
    long long rec_steps;      // steps whose raster offsets are valid
    long long inject_until;   // delivery by arrival step: steps < inject_until also consume their
                              // delay-ring slot (partial sums restored from a checkpoint)
    unsigned int status;
    int pad;
    alignas(128) unsigned int S_acc[3];   // spikes of step t at slot t mod 3
    alignas(128) unsigned long long bar;  // grid-barrier arrivals of the running k_persist launch
    // two-level arrival (Dev::bar_groups > 1): the blocks b = g mod G arrive
    // on grp[g].arr; the last of them forwards one arrival to bar (fwd: the
    // group's spike count forwarded so far).  Zeroed with bar.
    struct alignas(128) BarGroup {
        unsigned long long arr, fwd;
    } grp[kBarGroups];
};

// Drive of one network of a batch (independent networks stepped together);
// 16-byte aligned: the first four thresholds are read as one uint4.
struct __align__(16) NetDrive {
    uint32_t th[kPTab];  // finite Poisson thresholds, th[k] for k < fin
    int fin;
    uint32_t key0, key1;  // Philox key (the network's drive seed)
    int pad;
    long long off;        // first id of the network (a multiple of 4)
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
    const uint2 *row;         // [M+1] first level-1 and level-2 entry of each internal neuron
    const unsigned long long *csr;  // [M+1] first synapse of each internal neuron
    const uint32_t *l1_pair;  // exchange pair (source partition, VN) of each level-1 entry
    const uint32_t *l2_pair;  // exchange pair (source partition, partition) of each level-2 entry
    // exchange buffers, one region per pair (source partition p, destination)
    uint32_t *bucket;                        // level-1 entry ids, region (p, VN g)
    const ulonglong2 *bucket_slot;           // [n_bpair] region {first entry, capacity}
    uint32_t *bucket_cnt;                    // [2][n_bpair * kPairStride], by step parity
    unsigned long long *inbox;               // segments offset << 24 | length, region (p, q)
    const ulonglong2 *inbox_slot;            // [n_ipair] region {first entry, capacity}
    uint32_t *inbox_cnt;                     // [2][n_ipair * kPairStride], by step parity
    uint32_t *spk_step;  // [M] spikes of the running step (internal ids), in list order
    // records
    uint32_t *spk;
    long long *raster_off;
    unsigned long long *hash;
    int32_t *cur_rec;
    unsigned long long *counters;  // [C_N] steps and spikes
    unsigned long long *tally;     // [tally_rows][C_N] per-block event and message tallies
    unsigned long long *phase_ns;  // [kPhases] k_persist: block 0's time per part of a step (profiling)
    Ctrl *ctrl;
    // delivery by arrival step (n_arr > 0; 0: every delay at the spike step
    // into the delay ring)
    int32_t *acc;                  // [2][M] input of step t in slot t & 1
    unsigned long long *arr;       // [n_arr][arr_cap] queued runs: offset << 24 | length
    unsigned int *arr_cnt;         // [n_arr * kPairStride] fill of each list
    const uint4 *dcnt;             // [n_l2] u16 x 8: synapses of delay <= k + 1 in the segment
    unsigned long long arr_cap;
    int n_arr;                     // lists: the largest delay (list of step s: s mod n_arr)
    // delivery into each partition's own input (k_owner): per internal
    // partition q and arrival step s, the runs that arrive at q at step s
    // (list s mod n_own of q)
    unsigned long long *inb;       // records: offset << 24 | length
    const ulonglong2 *inb_slot;    // [P] {first record of q's list 0, capacity of each of q's lists}
    unsigned int *inb_cnt;         // [P * n_own * kPairStride] fill of each list
    const long long *pbase;        // [P + 1] first internal neuron of each internal partition
    int n_own;                     // lists per partition (the largest delay); 0: not available
    int vec_pieces;                // deliver staged pieces with 16-byte / 8-byte loads
    int bar_groups;                // > 1: two-level grid-barrier arrival over this many groups
    int prefetch_state;            // global neuron state: prefetch the next step's lines into L2
    int async_rec;                 // queued runs delivered with asynchronous copies (deliver_records_async)
    // scalars
    long long M;
    int P, n_vn, vn_size, D;
    int n_bpair, n_ipair;
    long long chunk_q;  // kModeSmem: quads owned by each block of k_persist
    float alpha, e_l, v_th, v_reset;
    int t_ref, w_ext, i_bias, th_fin;
    uint32_t key0, key1;
    long long raster_cap, raster_steps, hash_steps;
    int cur_every, cur_slots;
    uint32_t th32[kPTab];   // finite Poisson thresholds (the closing 2^32 is implied)
    // batches: the network of each quad of ids and every network's drive
    // (nullptr for a single network, which takes th32 / th_fin / key0 / key1)
    const uint16_t *net_of;
    const NetDrive *net_drive;
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

// Start moving the line holding p into L2 (no register result).
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Row bounds of spiking neuron i are the first thing its routing reads:
// start fetching them when the spike is found.
__device__ __forceinline__ void prefetch_rows(const Dev &d, long long j0, unsigned int m)
{
    for (; m; m &= m - 1u) {
        const long long i = j0 + __ffs(m) - 1;
        prefetch_l2(d.row + i);
        prefetch_l2(d.row + i + 1);
        prefetch_l2(d.csr + i);
        prefetch_l2(d.csr + i + 1);
    }
}

// Every 128-byte line of [a, b), one line per lane in turn (whole warp).
__device__ __forceinline__ void prefetch_span(const void *a, const void *b, int lane)
{
    const uintptr_t e = (uintptr_t)b;
    for (uintptr_t x = ((uintptr_t)a & ~(uintptr_t)127) + (uintptr_t)lane * 128u; x < e; x += 32u * 128u)
        prefetch_l2((const void *)x);
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

__device__ __forceinline__ unsigned long long atom_add_acq_rel(unsigned long long *p, unsigned long long x)
{
    unsigned long long old;
    asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(x) : "memory");
    return old;
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
// cooperative launch).  Each block adds one arrival to the low 32 bits of
// Ctrl::bar, which the host zeroes before the launch (and keeps the
// arrivals of a launch below 2^32); barrier k is complete when they reach
// (k + 1) * gridDim.x.  The high 32 bits carry what the arrivals add there:
// each block's spike count of the step at the step's first barrier.  A block-wide barrier, then a release add and acquire
// loads at GPU scope make every write of every block before the barrier
// visible to every block after it.  The wait is bounded: past limit_ns the
// block records kStTimeout and gives up, and a block that sees another one's
// timeout gives up too.  Returns false when the block gave up.
// The barrier in two halves: grid_arrive (block-wide barrier, then the
// release add) and grid_wait (the bounded acquire wait, then a block-wide
// barrier); work between them must not depend on other blocks.
// Two-level arrival (groups G > 1, G <= gridDim.x): block b arrives on
// the word of group g = b mod G with an acquire-release add; the block that
// completes its group's barrier k (its group's arrivals reach (k + 1) n_g)
// forwards one arrival and the group's spike count since its last forward
// to Ctrl::bar with a release add.  Barrier k is then complete when bar's
// arrivals reach (k + 1) G.  The acquire-release chain makes every write of
// the group's blocks visible to whoever acquires bar.
__device__ __forceinline__ void grid_arrive(Ctrl *c, unsigned long long k, int groups, bool arrive = true,
                                            unsigned long long add = 1ull)
{
    __syncthreads();
    groups = min(groups, (int)gridDim.x);
    if (threadIdx.x == 0 && arrive) {
        if (groups <= 1) {
            red_release(&c->bar, add);
        } else {
            const unsigned int g = blockIdx.x % (unsigned int)groups;
            const unsigned int n_g = (gridDim.x - g + (unsigned int)groups - 1u) / (unsigned int)groups;
            Ctrl::BarGroup *gr = &c->grp[g];
            const unsigned long long old = atom_add_acq_rel(&gr->arr, add);
            if ((unsigned int)old + 1u == (unsigned int)((k + 1ull) * n_g)) {
                const unsigned long long cum = (old >> 32) + (add >> 32);
                const unsigned long long fw = *(volatile unsigned long long *)&gr->fwd;
                *(volatile unsigned long long *)&gr->fwd = cum;
                red_release(&c->bar, 1ull + ((cum - fw) << 32));
            }
        }
    }
}

__device__ __forceinline__ bool grid_wait(Ctrl *c, unsigned long long k, int groups, unsigned long long limit_ns,
                                          unsigned long long *word = nullptr)
{
    __shared__ int s_ok;
    groups = min(groups, (int)gridDim.x);
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long target = (k + 1ull) * (groups > 1 ? (unsigned long long)groups : gridDim.x);
        const unsigned long long deadline = global_ns() + limit_ns;
        unsigned int spins = 0;
        unsigned long long v;
        while (((v = ld_acquire(&c->bar)) & 0xFFFFFFFFull) < target) {
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
        if (word) *word = v;  // (shared memory: read after the barrier below)
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}


// Drive of a neuron: the Poisson thresholds (the first four as values, the
// rest behind a pointer: shared memory for a single network, the batch table
// otherwise) and the Philox key and id offset of its network.
struct Drive {
    uint32_t t0, t1, t2, t3;
    int fin;
    const uint32_t *th;
    uint32_t key0, key1;
    long long off;
};

// Drive of global id g; th_smem: the single network's thresholds staged in
// shared memory (lanes index them divergently, which the kernel-parameter
// bank would serialise).
__device__ __forceinline__ Drive drive_of(const Dev &d, const uint32_t *th_smem, uint32_t g)
{
    Drive r;
    if (!d.net_of) {
        r.t0 = d.th32[0];
        r.t1 = d.th32[1];
        r.t2 = d.th32[2];
        r.t3 = d.th32[3];
        r.fin = d.th_fin;
        r.th = th_smem;
        r.key0 = d.key0;
        r.key1 = d.key1;
        r.off = 0;
    } else {
        const NetDrive *nd = d.net_drive + __ldg(d.net_of + (g >> 2));
        const uint4 t = __ldg(reinterpret_cast<const uint4 *>(nd->th));
        r.t0 = t.x;
        r.t1 = t.y;
        r.t2 = t.z;
        r.t3 = t.w;
        r.fin = __ldg(&nd->fin);
        r.th = nd->th;
        r.key0 = __ldg(&nd->key0);
        r.key1 = __ldg(&nd->key1);
        r.off = __ldg(&nd->off);
    }
    return r;
}

// Drive of one neuron in weight units: k * w_ext + i_bias (uint32
// arithmetic), k = number of finite thresholds <= u (they ascend): the first
// four compared at once, the rest (rare: k >= 4 has probability ~1.4 % at
// 0.8 arrivals per step) one by one.  u: the neuron's drive word; dr: its
// network's drive.
__device__ __forceinline__ uint32_t drive_units(const Dev &d, const Drive &dr, uint32_t u)
{
    int k = (0 < dr.fin && u >= dr.t0) + (1 < dr.fin && u >= dr.t1) + (2 < dr.fin && u >= dr.t2) +
            (3 < dr.fin && u >= dr.t3);
    if (k == 4)
        while (k < dr.fin && u >= dr.th[k]) ++k;
    return (uint32_t)k * (uint32_t)d.w_ext + (uint32_t)d.i_bias;
}

// The leak of a non-refractory neuron: e_l + alpha * (V - e_l).
__device__ __forceinline__ float lif_leak(const Dev &d, float v)
{
    const float uu = __fsub_rn(v, d.e_l);
    const float au = __fmul_rn(d.alpha, uu);
    return __fadd_rn(d.e_l, au);
}

// The rest of a2 once the recurrent input is known: I = irec + ext (the
// same uint32 sum as irec + k * w_ext + i_bias); v holds the leaked
// potential on entry and the new one on return.  Returns true on a spike.
__device__ __forceinline__ bool lif_finish(const Dev &d, uint32_t ext, int32_t irec, float &v, uint32_t &r)
{
    const int32_t I = (int32_t)((uint32_t)irec + ext);
    if (r > 0) {
        r -= 1;
        v = d.v_reset;
        return false;
    }
    const float x = __fmul_rn(__int2float_rn(I), 0.0009765625f);
    v = __fadd_rn(v, x);
    if (v >= d.v_th) {
        v = d.v_reset;
        r = (uint32_t)d.t_ref;
        return true;
    }
    return false;
}

// a1 + a2 for one neuron: returns true on a spike.  u: the neuron's drive
// word; dr: its network's drive.
__device__ __forceinline__ bool lif_neuron(const Dev &d, const Drive &dr, uint32_t u, int32_t irec, float &v,
                                           uint32_t &r)
{
    const uint32_t ext = drive_units(d, dr, u);
    v = lif_leak(d, v);
    return lif_finish(d, ext, irec, v, r);
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

// Shared-memory state of one routing round (from the block's StepShared).
struct Stage {
    unsigned long long *lng;   // [kLongCap] pieces: offset << 8 | length (<= kPiece)
    unsigned long long *sht;   // [kShortCap] short segments: offset << 8 | length (<= kShortSeg)
    unsigned int *nl, *ns;
    unsigned int (*ty)[kTally];  // [kWarps][kTally] tallies: events, l1 local, l1 cross-VN, l2 by class
    uint32_t *e0, *f0;           // [kRound] first level-1 / level-2 entry of each spike of a round
    uint32_t *pre1, *pre2;       // [kRound + 1] prefix of the level-1 / level-2 entry counts
    int *part;                   // [kRound] source partition of each spike
    // delivery by arrival step: the round's queued runs (pool) with their
    // list and rank in it, the runs per list and each list's reservation
    unsigned long long *arec;    // [kArrPool]
    unsigned short *atag;        // [kArrPool] rank << 4 | list
    unsigned int *an;            // runs in the pool
    unsigned int *ak;            // [kMaxArr] runs per list
    unsigned long long *abase;   // [kMaxArr] first slot reserved in each list
};

// Add a warp's per-lane tally v into slot k of its shared tally row (whole
// warp calls).
__device__ __forceinline__ void tally_add(const Stage &sg, int k, unsigned int v)
{
    v = __reduce_add_sync(0xFFFFFFFFu, v);  // one warp reduction instruction
    if ((threadIdx.x & 31) == 0) sg.ty[threadIdx.x >> 5][k] += v;
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

// Accumulator of a synapse of packed target word td: with fix (delivery by
// arrival step) fix[target], the next step's input slot, whatever the delay;
// else the delay-ring slot of step tm + delay.
__device__ __forceinline__ int32_t *syn_dst(const Dev &d, int tm, int32_t *fix, uint32_t td)
{
    if (fix) return fix + (td & kTgtMask);
    int sl = tm + (int)(td >> kTgtBits) + 1;
    if (sl >= d.D) sl -= d.D;
    return d.ring + (long long)sl * d.M + (td & kTgtMask);
}

// a6 for n consecutive synapses from offset o by one thread (the rare
// overflow of a staging list).
__device__ __forceinline__ unsigned int deliver_run(const Dev &d, int tm, int32_t *fix, unsigned long long o,
                                                    unsigned int n)
{
    for (unsigned int k = 0; k < n; ++k) {
        const uint32_t td = __ldcs(d.syn_td + o + k);
        const int32_t w = __ldcs(d.syn_w + o + k);
        atomicAdd(syn_dst(d, tm, fix, td), w);
    }
    return n;
}

// a6 for staged lists (pieces lng[0, nl), short segments sht[0, ns)) by
// the warps [w0, w0 + nwarp) of the block: a piece per warp (4 synapses per
// lane, every load in flight before the reductions), then short segments a
// lane each.  Delays count from slot tm (the spikes' step), or every synapse
// goes to fix (syn_dst).  Returns the synapses this thread delivered.
__device__ __forceinline__ unsigned int deliver_lists(const Dev &d, int tm, int32_t *fix, const unsigned long long *lng,
                                                      unsigned int nl, const unsigned long long *sht,
                                                      unsigned int ns, int w0, int nwarp)
{
    const int lane = threadIdx.x & 31, wid = (int)(threadIdx.x >> 5) - w0;
    unsigned int ev = 0;
    const unsigned int units = nl + (ns + 31u) / 32u;
    for (unsigned int u = (unsigned int)wid; u < units; u += (unsigned int)nwarp) {
        if (u < nl && d.vec_pieces) {
            // the piece as 16-byte target words and 8-byte weight words: lane
            // l takes synapses a + 4l .. a + 4l + 3 of the 4-aligned window
            // a = o & ~3 (and lane 0 the window's last four when the piece
            // runs past it), synapses outside [o, o + n) masked
            const unsigned long long e = lng[u];
            const unsigned long long o = e >> 8;
            const unsigned int n = (unsigned int)(e & 0xFFu);
            const unsigned long long a = o & ~3ull, end = o + n;
            const unsigned long long x0 = a + 4ull * (unsigned long long)lane;
            uint4 tv = make_uint4(0u, 0u, 0u, 0u), tx = tv;
            uint2 wv = make_uint2(0u, 0u), wx = wv;
            if (x0 < end) {
                tv = __ldcs(reinterpret_cast<const uint4 *>(d.syn_td + x0));
                wv = __ldcs(reinterpret_cast<const uint2 *>(d.syn_w + x0));
            }
            const bool extra = lane == 0 && a + 128ull < end;
            if (extra) {
                tx = __ldcs(reinterpret_cast<const uint4 *>(d.syn_td + a + 128ull));
                wx = __ldcs(reinterpret_cast<const uint2 *>(d.syn_w + a + 128ull));
            }
            const uint32_t tds[8] = {tv.x, tv.y, tv.z, tv.w, tx.x, tx.y, tx.z, tx.w};
            const uint32_t wws[4] = {wv.x, wv.y, wx.x, wx.y};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const unsigned long long x = (k < 4 ? x0 : a + 128ull) + (unsigned long long)(k & 3);
                if ((k < 4 || extra) && x >= o && x < end) {
                    const uint32_t ww = wws[k >> 1];
                    const int32_t w = (int32_t)(int16_t)(uint16_t)((k & 1) ? (ww >> 16) : (ww & 0xFFFFu));
                    atomicAdd(syn_dst(d, tm, fix, tds[k]), w);
                }
            }
            if (lane == 0) ev += n;
        } else if (u < nl) {
            const unsigned long long e = lng[u];
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
                if (x < n) atomicAdd(syn_dst(d, tm, fix, td[k]), w[k]);
            }
            if (lane == 0) ev += n;
        } else {
            const unsigned int x = (u - nl) * 32u + (unsigned int)lane;
            if (x < ns) {
                const unsigned long long e = sht[x];
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
                        if (k0 + k < n) atomicAdd(syn_dst(d, tm, fix, td[k]), w[k]);
                }
                ev += n;
            }
        }
    }
    return ev;
}

// a6 for the staged work of one routing round, all warps of the block.
// With delivery by arrival step the events were counted when routed.
__device__ __forceinline__ void deliver_staged(const Dev &d, int tm, int32_t *fix, const Stage &sg, unsigned int nl,
                                               unsigned int ns)
{
    const unsigned int ev = deliver_lists(d, tm, fix, sg.lng, nl, sg.sht, ns, 0, kWarps);
    tally_add(sg, 0, fix ? 0u : ev);
}

// Minimum-delay batching (k_persist): the synapses of delay >= 2 of a
// step's segments are not needed before step t + 2, so a block keeps their
// staged lists from one step's routing to the next and delivers them while
// its other warps walk the next step's routing tables (a latency chain that
// leaves the reduction units idle).  Lists by step parity.
constexpr int kDefLong = 256, kDefShort = 512;
constexpr int kTravWarps = 4;  // warps that walk the tables while the others deliver
struct Deferred {
    unsigned long long lng[2][kDefLong];
    unsigned long long sht[2][kDefShort];
    unsigned int nl[2], ns[2];
};

// The lists in a deferring k_persist, nothing in the others.
template <bool ON>
struct DeferSlot {
    Deferred df;
    __device__ Deferred *get() { return &df; }
};
template <>
struct DeferSlot<false> {
    __device__ Deferred *get() { return nullptr; }
};

// Staging of a run of n synapses at o (stage_run_warp below): a short run
// on the short list, a long one cut into pieces.  What does not fit is
// delivered by the thread at once (slot base tm: delivering early is exact,
// the run's slots are read later).

// Rank of this lane among the lanes of mask m below it.
__device__ __forceinline__ unsigned int lane_rank(unsigned int m)
{
    return __popc(m & ((1u << (threadIdx.x & 31)) - 1u));
}

// stage_run for a whole warp (every lane calls; n = 0: nothing to stage):
// one shared-memory reservation per list and warp, not one per lane, so the
// lanes do not queue on the same shared-memory word.
__device__ __forceinline__ unsigned int stage_run_warp(const Dev &d, int tm, int32_t *fix, unsigned long long o,
                                                       unsigned int n, unsigned long long *lng, unsigned int *nl,
                                                       unsigned int capl, unsigned long long *sht, unsigned int *ns,
                                                       unsigned int caps)
{
    const int lane = threadIdx.x & 31;
    unsigned int ev = 0;
    const bool is_short = n > 0 && n <= kShortSeg;
    const unsigned int ms = __ballot_sync(0xFFFFFFFFu, is_short);
    if (ms) {
        const int lead = __ffs(ms) - 1;
        unsigned int sb = 0;
        if (lane == lead) sb = atomicAdd(ns, (unsigned int)__popc(ms));
        sb = __shfl_sync(0xFFFFFFFFu, sb, lead) + lane_rank(ms);
        if (is_short) {
            if (sb < caps) sht[sb] = (o << 8) | n;
            else ev += deliver_run(d, tm, fix, o, n);
        }
    }
    const unsigned int np = n > kShortSeg ? (n + kPiece - 1u) / kPiece : 0u;
    unsigned int inc = np;
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, inc, k);
        if (lane >= k) inc += y;
    }
    const unsigned int tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
    if (tot) {
        unsigned int pb = 0;
        if (lane == 0) pb = atomicAdd(nl, tot);
        pb = __shfl_sync(0xFFFFFFFFu, pb, 0) + inc - np;
        for (unsigned int j = 0; j < np; ++j, ++pb) {
            const unsigned long long oo = o + (unsigned long long)j * kPiece;
            const unsigned int m = min(kPiece, n - j * kPiece);
            if (pb < capl) lng[pb] = (oo << 8) | m;
            else ev += deliver_run(d, tm, fix, oo, m);
        }
    }
    return ev;
}

// What a thread owes after walking its entries: the exchange write of its
// last entry (kind 1 bucket, 2 inbox; the fill-counter reservation stays in
// flight meanwhile), synapses it delivered itself, overflow bits.
struct Pending {
    int pk;
    unsigned int ppos;
    ulonglong2 pslot;
    unsigned long long pval;
    unsigned int ev, ovf;
};

// Barrier of the block, or of its threads [0, nthr) (named barrier 1).
__device__ __forceinline__ void sync_part(int nthr)
{
    if (nthr == kThreads) __syncthreads();
    else asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
}

// Queue runs on arrival list `list` (delivery by arrival step) for a whole
// warp (every lane calls; n = 0: no run): this lane's run of n synapses at
// o goes to the round's pool, or straight on the list when the pool is full.
// One pool and one rank reservation per warp.
__device__ __forceinline__ void arrival_queue_warp(const Dev &d, const Stage &sg, int list, unsigned long long o,
                                                   unsigned int n, unsigned int &ovf)
{
    const unsigned int m = __ballot_sync(0xFFFFFFFFu, n > 0);
    if (!m) return;
    const int lane = threadIdx.x & 31, lead = __ffs(m) - 1;
    unsigned int ps = 0;
    if (lane == lead) ps = atomicAdd(sg.an, (unsigned int)__popc(m));
    ps = __shfl_sync(0xFFFFFFFFu, ps, lead) + lane_rank(m);
    // ranks in the list only for the runs that found room in the pool
    const bool pooled = n > 0 && ps < (unsigned int)kArrPool;
    const unsigned int mp = __ballot_sync(0xFFFFFFFFu, pooled);
    unsigned int r = 0;
    if (mp) {
        const int lp = __ffs(mp) - 1;
        if (lane == lp) r = atomicAdd(&sg.ak[list], (unsigned int)__popc(mp));
        r = __shfl_sync(0xFFFFFFFFu, r, lp) + lane_rank(mp);
    }
    // the runs the pool has no room for go straight on the list: one
    // reservation for the warp's
    const bool direct = n > 0 && !pooled;
    const unsigned int mg = __ballot_sync(0xFFFFFFFFu, direct);
    unsigned int pos = 0;
    if (mg) {
        const int lg = __ffs(mg) - 1;
        if (lane == lg) pos = atomicAdd(&d.arr_cnt[(size_t)list * kPairStride], (unsigned int)__popc(mg));
        pos = __shfl_sync(0xFFFFFFFFu, pos, lg) + lane_rank(mg);
    }
    if (n == 0) return;
    const unsigned long long rec = (o << kLenBits) | (unsigned long long)n;
    if (pooled) {
        sg.arec[ps] = rec;
        sg.atag[ps] = (unsigned short)((r << 4) | (unsigned int)list);
    } else if (pos < d.arr_cap) {
        d.arr[(size_t)list * d.arr_cap + pos] = rec;
    } else {
        ovf |= kStArrival;
    }
}

// Delivery into the partitions' own input: queue the runs of the segment of
// synapses at o (delay counts dc) into destination partition q on q's
// lists of their arrival steps (the run of delay d on list (t + d) mod
// n_own; tmod = t mod n_own).
__device__ __forceinline__ void owner_queue(const Dev &d, unsigned int q, unsigned long long o, uint4 dc, int tmod,
                                            unsigned int &ovf)
{
    const ulonglong2 sl = d.inb_slot[q];
    const uint32_t c[kMaxArr] = {dc.x & 0xFFFFu, dc.x >> 16, dc.y & 0xFFFFu, dc.y >> 16,
                                 dc.z & 0xFFFFu, dc.z >> 16, dc.w & 0xFFFFu, dc.w >> 16};
    unsigned int pos[kMaxArr];
    // the reservations first, all in flight together, then the records
#pragma unroll
    for (int k = 0; k < kMaxArr; ++k) {
        const uint32_t lo = k ? c[k - 1] : 0u;
        pos[k] = 0xFFFFFFFFu;
        if (k < d.n_own && c[k] > lo) {
            int li = tmod + k + 1;
            while (li >= d.n_own) li -= d.n_own;
            pos[k] = atomicAdd(&d.inb_cnt[((size_t)q * d.n_own + li) * kPairStride], 1u);
        }
    }
#pragma unroll
    for (int k = 0; k < kMaxArr; ++k) {
        if (pos[k] == 0xFFFFFFFFu) continue;
        const uint32_t lo = k ? c[k - 1] : 0u;
        int li = tmod + k + 1;
        while (li >= d.n_own) li -= d.n_own;
        if (pos[k] < sl.y)
            d.inb[sl.x + (unsigned long long)li * sl.y + pos[k]] = ((o + lo) << kLenBits) | (unsigned long long)(c[k] - lo);
        else
            ovf |= kStArrival;
    }
}

// a4 + a5 for the nr <= kRound spikes at positions b0 .. b0+nr of the step's
// list, by the threads [0, nthr) (whole warps): the level-1 and level-2
// entries of all of them are numbered through and taken a thread each, so
// one spike's entries go out together.  Each level-2 entry's delivery is
// staged in shared memory as soon as the entry is read: all of the segment
// on the round's lists, or with df its delay-1 head (the synapses the next
// step reads; segments are sorted by delay) there and the rest on df's lists
// of parity cur.  With delivery by arrival step (fix: the next step's input
// slot) the delay-1 head is staged for fix and the run of each delay
// d >= 2 is queued for step t + d - 1 (t = the step, tmod = t mod n_arr).
// Counters of step parity par.
template <int RT>
__device__ __forceinline__ Pending route_traverse(const Dev &d, int par, int tm, unsigned int b0, unsigned int nr,
                                                  const Stage &sg, int nthr, Deferred *df, int cur,
                                                  int32_t *fix = nullptr, int tmod = 0)
{
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < nr) {
        const uint32_t i = d.spk_step[b0 + threadIdx.x];
        const uint2 a = d.row[i], b = d.row[i + 1];
        sg.e0[threadIdx.x] = a.x;
        sg.f0[threadIdx.x] = a.y;
        sg.pre1[threadIdx.x + 1] = b.x - a.x;
        sg.pre2[threadIdx.x + 1] = b.y - a.y;
        sg.part[threadIdx.x] = d.src_part[i];
    }
    if (threadIdx.x == 0) {
        *sg.nl = 0;
        *sg.ns = 0;
        if (RT == kRtArrival) *sg.an = 0;
    }
    if (RT == kRtArrival && threadIdx.x < kMaxArr) sg.ak[threadIdx.x] = 0;
    sync_part(nthr);
    if (threadIdx.x < 32) {
        // inclusive scans of the counts (kRound <= 32: one warp)
        uint32_t v1 = (unsigned int)lane < nr ? sg.pre1[lane + 1] : 0u;
        uint32_t v2 = (unsigned int)lane < nr ? sg.pre2[lane + 1] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y1 = __shfl_up_sync(0xFFFFFFFFu, v1, o), y2 = __shfl_up_sync(0xFFFFFFFFu, v2, o);
            if (lane >= o) {
                v1 += y1;
                v2 += y2;
            }
        }
        if ((unsigned int)lane < nr) {
            sg.pre1[lane + 1] = v1;
            sg.pre2[lane + 1] = v2;
        }
        if (lane == 0) {
            sg.pre1[0] = 0;
            sg.pre2[0] = 0;
        }
    }
    sync_part(nthr);
    uint32_t *bcnt = bucket_cnt_of(d, par);
    uint32_t *icnt = inbox_cnt_of(d, par);
    const uint32_t N1 = sg.pre1[nr], N = N1 + sg.pre2[nr];
    unsigned int l1_loc = 0, l1_xvn = 0;
    unsigned int cls[4] = {0, 0, 0, 0};
    Pending pn{0, 0u, make_ulonglong2(0ull, 0ull), 0ull, 0u, 0u};
    // the lanes of a warp take entries together (the staging below is
    // warp-collective); a lane past the end only stages nothing
    for (uint32_t x0 = threadIdx.x & ~31u; x0 < N; x0 += (uint32_t)nthr) {
        const uint32_t x = x0 + (uint32_t)lane;
        if (pn.pk == 1) {
            if (pn.ppos < pn.pslot.y) d.bucket[pn.pslot.x + pn.ppos] = (uint32_t)pn.pval;
            else pn.ovf |= kStBucket;
        } else if (pn.pk == 2) {
            if (pn.ppos < pn.pslot.y) d.inbox[pn.pslot.x + pn.ppos] = pn.pval;
            else pn.ovf |= kStInbox;
        }
        pn.pk = 0;
        // the segment this lane stages: the whole one, or its delay-1 head
        // with the rest on the deferred lists (df) or the arrival lists (ARR)
        unsigned long long so = 0;
        unsigned int sn = 0, rest = 0, oq = 0xFFFFFFFFu;
        uint4 dc = make_uint4(0u, 0u, 0u, 0u);
        if (x < N1) {
            // a4: one level-1 entry per destination VN, appended to bucket (p, g)
            const int k = prefix_find(sg.pre1, (int)nr, x);
            const uint32_t e = sg.e0[k] + (x - sg.pre1[k]);
            const int g = d.l1_vn[e];
            const uint32_t kp = d.l1_pair[e];
            pn.pslot = d.bucket_slot[kp];
            pn.ppos = atomicAdd(&bcnt[(size_t)kp * kPairStride], 1u);
            pn.pval = e;
            pn.pk = 1;
            if (g == sg.part[k] / d.vn_size) ++l1_loc;
            else ++l1_xvn;
        } else if (x < N) {
            // a5: the relay of the entry's VN expands it into inbox (p, q) of
            // partition q; the segment's delivery is staged
            const uint32_t y = x - N1;
            const int k = prefix_find(sg.pre2, (int)nr, y);
            const uint32_t f = sg.f0[k] + (y - sg.pre2[k]);
            const DevL2 l = d.l2[f];
            const uint32_t kq = d.l2_pair[f];
            pn.pslot = d.inbox_slot[kq];
            pn.ppos = atomicAdd(&icnt[(size_t)kq * kPairStride], 1u);
            const unsigned long long off = l.off & kOffMask;
            pn.pval = (off << kLenBits) | (unsigned long long)l.len;
            pn.pk = 2;
            so = off;
            if constexpr (RT == kRtArrival) {
                dc = d.dcnt[f];         // runs by delay: synapses of delay <= k + 1
                sn = dc.x & 0xFFFFu;    // the delay-1 head
                pn.ev += l.len;         // events counted when routed
            } else if constexpr (RT == kRtOwner) {
                dc = d.dcnt[f];
                oq = l.q;
                pn.ev += l.len;
            } else if (!df) {
                sn = l.len;
            } else {
                sn = (unsigned int)(l.off >> kOffBits);  // delay-1 head of the segment
                rest = l.len - sn;
            }
            // per-class tallies without a dynamically indexed (local-memory) array
            cls[0] += l.cls == 0;
            cls[1] += l.cls == 1;
            cls[2] += l.cls == 2;
            cls[3] += l.cls == 3;
        }
        if constexpr (RT == kRtOwner) {
            if (oq != 0xFFFFFFFFu) owner_queue(d, oq, so, dc, tmod, pn.ovf);
        } else if constexpr (RT == kRtArrival) {
            stage_run_warp(d, tm, fix, so, sn, sg.lng, sg.nl, kLongCap, sg.sht, sg.ns, kShortCap);
            const uint32_t c[kMaxArr] = {dc.x & 0xFFFFu, dc.x >> 16, dc.y & 0xFFFFu, dc.y >> 16,
                                         dc.z & 0xFFFFu, dc.z >> 16, dc.w & 0xFFFFu, dc.w >> 16};
#pragma unroll
            for (int k = 1; k < kMaxArr; ++k) {
                if (k < d.n_arr) {  // (block-uniform)
                    int li = tmod + k;
                    if (li >= d.n_arr) li -= d.n_arr;
                    arrival_queue_warp(d, sg, li, so + c[k - 1], c[k] > c[k - 1] ? c[k] - c[k - 1] : 0u, pn.ovf);
                }
            }
        } else if (!df) {
            pn.ev += stage_run_warp(d, tm, nullptr, so, sn, sg.lng, sg.nl, kLongCap, sg.sht, sg.ns, kShortCap);
        } else {
            pn.ev += stage_run_warp(d, tm, nullptr, so, sn, sg.lng, sg.nl, kLongCap, sg.sht, sg.ns, kShortCap);
            pn.ev += stage_run_warp(d, tm, nullptr, so + sn, rest, df->lng[cur], &df->nl[cur], kDefLong,
                                    df->sht[cur], &df->ns[cur], kDefShort);
        }
    }
    tally_add(sg, 1, l1_loc);
    tally_add(sg, 2, l1_xvn);
#pragma unroll
    for (int k = 0; k < 4; ++k) tally_add(sg, 3 + k, cls[k]);
    return pn;
}

// a6 of a round (whole block, after a block barrier) and the exchange write
// each thread still owes (pn from route_traverse; zero for the threads that
// did not walk).  With delivery by arrival step (fix) the round's queued
// runs go to their lists: one reservation per list, issued before the
// delivery, the copy after it.
template <int RT>
__device__ __forceinline__ void route_finish(const Dev &d, int tm, int32_t *fix, const Stage &sg, Pending pn)
{
    if (RT == kRtArrival && threadIdx.x < (unsigned int)d.n_arr) {
        const unsigned int n = sg.ak[threadIdx.x];
        if (n) sg.abase[threadIdx.x] = atomicAdd(&d.arr_cnt[(size_t)threadIdx.x * kPairStride], n);
    }
    if constexpr (RT != kRtOwner)
        deliver_staged(d, tm, fix, sg, min(*sg.nl, (unsigned int)kLongCap), min(*sg.ns, (unsigned int)kShortCap));
    if constexpr (RT == kRtArrival) {
        __syncthreads();
        const unsigned int na = min(*sg.an, (unsigned int)kArrPool);
        for (unsigned int x = threadIdx.x; x < na; x += kThreads) {
            const unsigned int tag = sg.atag[x];
            const unsigned int li = tag & 15u;
            const unsigned long long pos = sg.abase[li] + (tag >> 4);
            if (pos < d.arr_cap) d.arr[(size_t)li * d.arr_cap + pos] = sg.arec[x];
            else pn.ovf |= kStArrival;
        }
    }
    if (pn.pk == 1) {
        if (pn.ppos < pn.pslot.y) d.bucket[pn.pslot.x + pn.ppos] = (uint32_t)pn.pval;
        else pn.ovf |= kStBucket;
    } else if (pn.pk == 2) {
        if (pn.ppos < pn.pslot.y) d.inbox[pn.pslot.x + pn.ppos] = pn.pval;
        else pn.ovf |= kStInbox;
    }
    if (pn.ovf) atomicOr(&d.ctrl->status, pn.ovf);
    tally_add(sg, 0, pn.ev);
}


// a6 for runs queued on an arrival list (delivery by arrival step): records
// recs[lo, hi) (offset << 24 | length) into fix by the block's warps, 32
// records per warp at a time.  The warp numbers the synapses of its 32 runs
// through (a warp scan of the lengths) and takes them 32 U at a time, U per
// lane with every load in flight before the reductions; a lane finds the
// run of its synapse by a binary search over the lanes' prefix sums.  The
// next 32 records are loaded while the current ones are delivered.
template <int U>
__device__ __forceinline__ void deliver_records(const Dev &d, int32_t *fix, const unsigned long long *recs,
                                                unsigned long long lo, unsigned long long hi)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long step = (unsigned long long)kWarps * 32u;
    unsigned long long b = lo + (unsigned long long)wid * 32u;
    unsigned long long rec = (b + lane < hi) ? __ldcs(recs + b + lane) : 0ull;
    for (; b < hi; b += step) {
        const unsigned long long nx = b + step + (unsigned long long)lane;
        const unsigned long long rec_next = nx < hi ? __ldcs(recs + nx) : 0ull;
        const unsigned long long o = rec >> kLenBits;
        const unsigned int n = (unsigned int)(rec & kLenMask);
        // exclusive prefix of the run lengths over the warp
        unsigned int inc = n;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, inc, k);
            if (lane >= k) inc += y;
        }
        const unsigned int ex = inc - n;
        const unsigned int tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
        for (unsigned int base = 0; base < tot; base += 32u * U) {
            uint32_t td[U];
            int32_t w[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const unsigned int y = base + (unsigned int)k * 32u + (unsigned int)lane;
                // the last lane whose run starts at or before y
                int r = 0;
#pragma unroll
                for (int h = 16; h > 0; h >>= 1) {
                    const unsigned int v = __shfl_sync(0xFFFFFFFFu, ex, r + h);
                    if (v <= y) r += h;
                }
                const unsigned long long orr = __shfl_sync(0xFFFFFFFFu, o, r);
                const unsigned int er = __shfl_sync(0xFFFFFFFFu, ex, r);
                if (y < tot) {
                    td[k] = __ldcs(d.syn_td + orr + (y - er));
                    w[k] = __ldcs(d.syn_w + orr + (y - er));
                }
            }
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const unsigned int y = base + (unsigned int)k * 32u + (unsigned int)lane;
                if (y < tot) atomicAdd(fix + (td[k] & kTgtMask), w[k]);
            }
        }
        rec = rec_next;
    }
}

// deliver_records with the synapse loads as asynchronous 4-byte copies into
// a per-warp shared-memory stage (two stages): while one batch's copies are
// in flight, the previous batch's reductions run, so the loads in flight do
// not cost registers.  Each lane reads back only the slots it copied itself
// (cp.async.wait_group is per thread), so no warp barrier is needed.  The
// weight comes as the aligned 4-byte word holding it.
template <int U>
__device__ __forceinline__ void deliver_records_async(const Dev &d, int32_t *fix, const unsigned long long *recs,
                                                      unsigned long long lo, unsigned long long hi)
{
    __shared__ uint32_t s_td[kWarps][2][U * 32];
    __shared__ uint32_t s_w[kWarps][2][U * 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long step = (unsigned long long)kWarps * 32u;
    const uint32_t *w32 = reinterpret_cast<const uint32_t *>(d.syn_w);
    unsigned long long b = lo + (unsigned long long)wid * 32u;
    unsigned long long rec = (b + lane < hi) ? __ldcs(recs + b + lane) : 0ull;
    unsigned long long rec_next = 0ull;
    unsigned long long o = 0ull;
    unsigned int ex = 0, tot = 0, base = 0;
    // the group of 32 records starting at b: run offsets and the exclusive
    // prefix of their lengths over the warp
    auto group = [&]() {
        const unsigned long long nx = b + step + (unsigned long long)lane;
        rec_next = nx < hi ? __ldcs(recs + nx) : 0ull;
        o = rec >> kLenBits;
        const unsigned int n = (unsigned int)(rec & kLenMask);
        unsigned int inc = n;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, inc, k);
            if (lane >= k) inc += y;
        }
        ex = inc - n;
        tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
        base = 0;
    };
    if (b < hi) group();
    int st = 0;
    bool pend = false;
    unsigned int pmask = 0, psel = 0;
    auto reduce = [&](int s2, unsigned int mask, unsigned int sel) {
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (mask & (1u << k)) {
                const uint32_t td = s_td[wid][s2][k * 32 + lane];
                const uint32_t ww = s_w[wid][s2][k * 32 + lane];
                const int32_t w = (sel & (1u << k)) ? (int32_t)(int16_t)(ww >> 16) : (int32_t)(int16_t)(ww & 0xFFFFu);
                atomicAdd(fix + (td & kTgtMask), w);
            }
    };
    while (b < hi) {
        // issue the batch (b, base) into stage st
        unsigned int mask = 0, sel = 0;
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const unsigned int y = base + (unsigned int)k * 32u + (unsigned int)lane;
            int r = 0;
#pragma unroll
            for (int h = 16; h > 0; h >>= 1) {
                const unsigned int v = __shfl_sync(0xFFFFFFFFu, ex, r + h);
                if (v <= y) r += h;
            }
            const unsigned long long orr = __shfl_sync(0xFFFFFFFFu, o, r);
            const unsigned int er = __shfl_sync(0xFFFFFFFFu, ex, r);
            if (y < tot) {
                const unsigned long long idx = orr + (y - er);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(&s_td[wid][st][k * 32 + lane])),
                             "l"(d.syn_td + idx)
                             : "memory");
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(&s_w[wid][st][k * 32 + lane])),
                             "l"(w32 + (idx >> 1))
                             : "memory");
                mask |= 1u << k;
                sel |= (unsigned int)(idx & 1ull) << k;
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        // the previous batch's reductions while this one is in flight
        if (pend) {
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            reduce(st ^ 1, pmask, psel);
        }
        pend = true;
        pmask = mask;
        psel = sel;
        st ^= 1;
        base += 32u * U;
        if (base >= tot) {
            b += step;
            rec = rec_next;
            if (b < hi) group();
        }
    }
    if (pend) {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        reduce(st ^ 1, pmask, psel);
    }
}

// ---------------------------------------------------------------- a1-a6
// How a step reaches its neurons' state:
//   kModeScalar  one neuron per thread, grid-stride over global memory;
//   kModeVec     four neurons per thread with 16-byte global loads (M % 4 == 0);
//   kModeSmem    k_persist only: each block owns a contiguous run of quads
//                whose V and ref stay in shared memory for the whole launch;
//                the block's part of ring slot t comes in with one bulk copy
//                (cp.async.bulk, mbarrier completion) per step.
enum { kModeScalar = 0, kModeVec = 1, kModeSmem = 2 };

// Shared-memory state of a block in kModeSmem.
struct Resident {
    float4 *V;                 // [cq] membrane potentials of the block's quads
    int4 *ring;                // [cq] this step's ring slot, staged by the bulk copy
    int4 *ext;                 // [cq] this step's drive in weight units (pre_update)
    uint32_t *ref;             // [cq] refractory counters, one byte per neuron
    unsigned long long *bar;   // mbarrier of the bulk copy
    long long q0;              // first quad of the block
    int nq;                    // quads of the block
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global memory into this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Wait until phase `parity` of `bar` completes, for at most limit_ns.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, unsigned long long limit_ns)
{
    const unsigned long long deadline = global_ns() + limit_ns;
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (global_ns() > deadline) return false;
    }
}

// a1 + a2 for the quad of neurons j0 .. j0+3 (internal ids): membrane
// potentials vv, recurrent inputs ii, refractory counters r4 (a byte each).
// Returns the spike bits.
__device__ __forceinline__ unsigned int update_quad(const Dev &d, const uint32_t *th, long long t, long long j0,
                                                    float (&vv)[4], const int32_t (&ii)[4], uint32_t &r4,
                                                    bool do_hash, unsigned long long &hc, unsigned long long &hv)
{
    // one Philox block serves the four neurons of a quad (networks of a batch
    // start at multiples of 4); a reordering map needs a block per neuron
    Drive dq = drive_of(d, th, d.gid ? d.gid[j0] : (uint32_t)j0);
    uint4 wq = make_uint4(0u, 0u, 0u, 0u);
    if (!d.gid) wq = philox4(dq.key0, dq.key1, (uint32_t)((j0 - dq.off) >> 2), (uint32_t)t);
    unsigned int m = 0;
    uint32_t r_out = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t g = d.gid ? d.gid[j0 + k] : (uint32_t)(j0 + k);
        uint32_t u;
        if (d.gid) {
            if (k > 0) dq = drive_of(d, th, g);
            u = uint4_word(philox4(dq.key0, dq.key1, (uint32_t)((g - dq.off) >> 2), (uint32_t)t), g & 3u);
        } else {
            u = uint4_word(wq, (uint32_t)k);
        }
        uint32_t r = (r4 >> (8 * k)) & 0xFFu;
        if (lif_neuron(d, dq, u, ii[k], vv[k], r)) m |= 1u << k;
        r_out |= r << (8 * k);
        if (do_hash) {
            hc += mix64(((unsigned long long)g << 32) | (uint32_t)ii[k]);
            hv += mix64(((unsigned long long)g << 32) | __float_as_uint(vv[k]));
        }
    }
    r4 = r_out;
    return m;
}

// The input-free half of a1 + a2 of step t for the block's resident quads
// (kModeSmem), run while the block waits at the grid barrier that ends step
// t - 1: the drive of each neuron in weight units into rs.ext and the leak
// e_l + alpha * (V - e_l) in place of V.  update_step<kModeSmem> adds the
// recurrent input in the order lif_neuron uses.  th: the thresholds staged in
// shared memory.
__device__ __forceinline__ void pre_update(const Dev &d, long long t, const uint32_t *th, const Resident &rs)
{
    for (int lq = threadIdx.x; lq < rs.nq; lq += kThreads) {
        const long long j0 = (rs.q0 + lq) * 4;
        Drive dq = drive_of(d, th, d.gid ? d.gid[j0] : (uint32_t)j0);
        uint4 wq = make_uint4(0u, 0u, 0u, 0u);
        if (!d.gid) wq = philox4(dq.key0, dq.key1, (uint32_t)((j0 - dq.off) >> 2), (uint32_t)t);
        const float4 v4 = rs.V[lq];
        const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
        uint32_t ex[4];
        float lv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t u;
            if (d.gid) {
                const uint32_t g = d.gid[j0 + k];
                if (k > 0) dq = drive_of(d, th, g);
                u = uint4_word(philox4(dq.key0, dq.key1, (uint32_t)((g - dq.off) >> 2), (uint32_t)t), g & 3u);
            } else {
                u = uint4_word(wq, (uint32_t)k);
            }
            ex[k] = drive_units(d, dq, u);
            lv[k] = lif_leak(d, vv[k]);
        }
        rs.V[lq] = make_float4(lv[0], lv[1], lv[2], lv[3]);
        rs.ext[lq] = make_int4((int)ex[0], (int)ex[1], (int)ex[2], (int)ex[3]);
    }
}

// The routing round's pool of queued runs (delivery by arrival step), in
// the kernels that route with it; nothing in the others.
template <bool ON>
struct ArrivalPool {
    unsigned long long rec[kArrPool];
    unsigned short tag[kArrPool];
    __device__ unsigned long long *r() { return rec; }
    __device__ unsigned short *g() { return tag; }
};
template <>
struct ArrivalPool<false> {
    __device__ unsigned long long *r() { return nullptr; }
    __device__ unsigned short *g() { return nullptr; }
};

// Shared-memory scratch of a block's step.
struct StepShared {
    unsigned long long lng[kLongCap];
    unsigned long long sht[kShortCap];
    unsigned int wsum[kWarps];
    unsigned int tot, gbase, nl, ns;
    long long head;
    long long t0;
    unsigned long long h[2][kWarps];
    unsigned int tally[kWarps][kTally];
    uint32_t th[kPTab];
    uint32_t e0[kRound], f0[kRound], pre1[kRound + 1], pre2[kRound + 1];
    int part[kRound];
    uint32_t own[kOwn];       // the block's own spikes of the step (the first kOwn)
    unsigned int n_own, obase;
    // k_persist: the first barrier's word, the spike sum it carried at the
    // last step, and the raster head of the next step
    unsigned long long word;
    uint32_t prevS;
    long long headv;
    // delivery by arrival step: the routing round's queued runs (Stage), the
    // step's arrival list share of this block, restored ring slots
    unsigned long long *arec;   // -> the kernel's ArrivalPool (delivery by arrival step)
    unsigned short *atag;
    unsigned int an, ak[kMaxArr];
    unsigned long long abase[kMaxArr];
    unsigned int arr_n;
    long long inj_until;
    // profiling (block 0 of k_persist): time per part, last stamp
    unsigned long long prof[kPhases + 1];
    int prof_on;
};

// Add the time since the last stamp to part k (k < 0: only restart).
__device__ __forceinline__ void prof_stamp(StepShared &sh, int k)
{
    if (sh.prof_on && threadIdx.x == 0) {
        const unsigned long long now = global_ns();
        if (k >= 0) sh.prof[k] += now - sh.prof[kPhases];
        sh.prof[kPhases] = now;
    }
}

// Delivery by arrival step: this block's equal share of the runs queued for
// step t (list t mod n_arr, complete since the last step's routing) into
// the next step's input slot (all threads call); U loads per lane in flight.
template <int U>
__device__ __forceinline__ void arrival_share(const Dev &d, long long t, StepShared &sh)
{
    const int li = (int)(t % d.n_arr);
    if (threadIdx.x == 0)
        sh.arr_n = min(*(volatile unsigned int *)&d.arr_cnt[(size_t)li * kPairStride],
                       (unsigned int)min(d.arr_cap, 0xFFFFFFFFull));
    __syncthreads();
    const unsigned long long n = sh.arr_n;
    const unsigned long long lo = n * blockIdx.x / gridDim.x, hi = n * (blockIdx.x + 1) / gridDim.x;
    if (d.async_rec)
        deliver_records_async<U>(d, d.acc + (size_t)((t + 1) & 1) * (size_t)d.M, d.arr + (size_t)li * d.arr_cap, lo,
                                 hi);
    else
        deliver_records<U>(d, d.acc + (size_t)((t + 1) & 1) * (size_t)d.M, d.arr + (size_t)li * d.arr_cap, lo, hi);
}

// a3: compaction of the spikes each thread collected in bits[0, NC) (bit b
// of word c is neuron id_of(c, b)) into step t's spike list: a block-wide
// scan numbers them and one reservation per block places them (all threads
// call; without spikes this costs one barrier).
template <int NC, class IdOf>
__device__ __forceinline__ void compact_spikes_multi(const Dev &d, long long t, StepShared &sh,
                                                     const uint32_t (&bits)[NC], IdOf id_of)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned int cnt = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) cnt += __popc(bits[c]);
    if (!__syncthreads_or(cnt)) return;
    unsigned int x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh.wsum[wid] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int tot = 0;
        for (int w = 0; w < kWarps; ++w) {
            const unsigned int cw = sh.wsum[w];
            sh.wsum[w] = tot;
            tot += cw;
        }
        sh.gbase = atomicAdd(&d.ctrl->S_acc[slot3(t)], tot);
        sh.obase = sh.n_own;
        sh.n_own += tot;
    }
    __syncthreads();
    unsigned int pos = sh.gbase + sh.wsum[wid] + x - cnt;
    unsigned int lp = sh.obase + sh.wsum[wid] + x - cnt;
#pragma unroll
    for (int c = 0; c < NC; ++c)
        for (uint32_t bb = bits[c]; bb; bb &= bb - 1u, ++lp) {
            const uint32_t id = id_of(c, __ffs(bb) - 1);
            d.spk_step[pos++] = id;
            if (lp < (unsigned int)kOwn) sh.own[lp] = id;
        }
}

// The same for one word of bits (bit b is neuron id_of(b)).
template <class IdOf>
__device__ __forceinline__ void compact_spikes(const Dev &d, long long t, StepShared &sh, uint32_t bits,
                                               IdOf id_of)
{
    const uint32_t b1[1] = {bits};
    compact_spikes_multi<1>(d, t, sh, b1, [&](int, int b) { return id_of(b); });
}

// While the block waits at the grid barrier after a3: pull the routing
// tables and synapses of its own spikes (whichever block routes them) from
// HBM into L2 — level-1 and level-2 entries, their pair ids and the synapse
// run — one spike per warp.  With delivery by arrival step the synapse run
// is left out: this step delivers only the delay-1 head of each segment,
// and the rest is read up to seven steps later, after L2 has turned over.
__device__ __forceinline__ void prefetch_own(const Dev &d, const StepShared &sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned int n = min(sh.n_own, (unsigned int)kOwn);
    for (unsigned int x = wid; x < n; x += kWarps) {
        const uint32_t i = sh.own[x];
        const uint2 r0 = d.row[i], r1 = d.row[i + 1];
        prefetch_span(d.l1_vn + r0.x, d.l1_vn + r1.x, lane);
        prefetch_span(d.l1_l2 + r0.x, d.l1_l2 + r1.x, lane);
        prefetch_span(d.l1_pair + r0.x, d.l1_pair + r1.x, lane);
        prefetch_span(d.l2 + r0.y, d.l2 + r1.y, lane);
        prefetch_span(d.l2_pair + r0.y, d.l2_pair + r1.y, lane);
        if (d.n_arr == 0) {
            const unsigned long long s0 = d.csr[i], s1 = d.csr[i + 1];
            prefetch_span(d.syn_td + s0, d.syn_td + s1, lane);
            prefetch_span(d.syn_w + s0, d.syn_w + s1, lane);
        }
    }
}

// Input of a quad plus the restored partial sums at p (delivery by arrival
// step, first steps after a restore), which are consumed (zeroed).
__device__ __forceinline__ int4 take_restored(int32_t *p, int4 i4)
{
    const int4 x = *reinterpret_cast<const int4 *>(p);
    *reinterpret_cast<int4 *>(p) = make_int4(0, 0, 0, 0);
    return make_int4((int)((uint32_t)i4.x + (uint32_t)x.x), (int)((uint32_t)i4.y + (uint32_t)x.y),
                     (int)((uint32_t)i4.z + (uint32_t)x.z), (int)((uint32_t)i4.w + (uint32_t)x.w));
}

// Global neuron state (kModeVec): while the step's last grid barrier
// completes, pull into L2 the lines the next step's update of this block
// reads (potentials, refractory counters, input slot), so that the update's
// loads do not wait on DRAM.  Prefetches only: nothing is read or written.
template <bool ARR>
__device__ __forceinline__ void prefetch_state_vec(const Dev &d, long long t)
{
    const long long nq = d.M / 4, stride = (long long)gridDim.x * kThreads;
    const int32_t *in = ARR ? d.acc + (size_t)(t & 1) * (size_t)d.M : d.ring + (long long)(t % d.D) * d.M;
    // a 128-byte line holds 8 quads of V and of the input, 32 of ref: one
    // lane in 8 (in 32 for ref lines) issues the prefetch
    for (long long q = (long long)blockIdx.x * kThreads + threadIdx.x; q < nq; q += stride) {
        if ((threadIdx.x & 7) == 0) {
            prefetch_l2(d.V + q * 4);
            prefetch_l2(in + q * 4);
        }
        if ((threadIdx.x & 31) == 0) prefetch_l2(d.ref + q * 4);
    }
}

// First half of step t on this block's share of the neurons (all threads
// call): a1-a3, the spikes into the step's list.  In kModeSmem, rs is the
// block's resident state and `phase` the parity of the bulk copy's
// mbarrier; a copy that does not complete within limit_ns records
// kStTimeout.
template <int MODE, bool ARR, int QB = 4>
__device__ __forceinline__ void update_step(const Dev &d, long long t, StepShared &sh, const Resident &rs,
                                            uint32_t phase, unsigned long long limit_ns)
{
    Ctrl *c = d.ctrl;
    const int par = (int)(t & 1);
    const int slot = (int)(t % d.D);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool do_hash = t < d.hash_steps;
    const bool do_cur = d.cur_every > 0 && (t % d.cur_every) == 0 && (t / d.cur_every) < d.cur_slots;
    // the step's input: its delay-ring slot, or with delivery by arrival
    // step its input slot t & 1 plus, for the first steps after a restore,
    // the ring slot holding the restored partial sums (inj)
    int32_t *ring = ARR ? d.acc + (size_t)(t & 1) * (size_t)d.M : d.ring + (long long)slot * d.M;
    int32_t *inj = (ARR && t < sh.inj_until) ? d.ring + (long long)slot * d.M : nullptr;
    int32_t *cur = do_cur ? d.cur_rec + (t / d.cur_every) * d.M : nullptr;
    if constexpr (MODE == kModeSmem) {
        // a1: the block's part of ring slot t, in flight while the counters
        // are cleared.  The slot was written through the generic proxy
        // (other blocks' reductions, ordered by the grid barrier) and the
        // staging buffer was last read by this block's threads: both are
        // ordered before the async-proxy copy by the proxy fences.
        __syncthreads();
        if (threadIdx.x == 0 && rs.nq > 0) {
            asm volatile("fence.proxy.async.global;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bulk_load(rs.ring, ring + rs.q0 * 4, (uint32_t)rs.nq * 16u, rs.bar);
        }
    }
    {
        // clear the other parity (used by step t - 1 only; step t + 1 fills
        // it) and the spike count of step t + 1
        uint32_t *b1 = bucket_cnt_of(d, par ^ 1), *i1 = inbox_cnt_of(d, par ^ 1);
        const int nb = d.n_bpair, ni = nb + d.n_ipair;
        for (int x = blockIdx.x * kThreads + threadIdx.x; x < ni; x += gridDim.x * kThreads) {
            if (x < nb) b1[(size_t)x * kPairStride] = 0;
            else i1[(size_t)(x - nb) * kPairStride] = 0;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            c->S_acc[slot3(t + 1)] = 0;
            // the arrival list step t - 1 delivered (step t's routing refills it)
            if (ARR) d.arr_cnt[(size_t)((t + d.n_arr - 1) % d.n_arr) * kPairStride] = 0;
        }
    }
    if (threadIdx.x < kPTab) sh.th[threadIdx.x] = d.th32[threadIdx.x];
    if (threadIdx.x == 0) sh.n_own = 0u;
    __syncthreads();

    unsigned long long hc = 0, hv = 0;
    // a1 + a2 over this block's neurons; each thread collects its spikes as
    // bits (4 per quad, 1 per neuron in kModeScalar) and a3 runs once the
    // word is full or the neurons are done
    if constexpr (MODE == kModeSmem) {
        if (rs.nq > 0 && !mbar_wait(rs.bar, phase, limit_ns)) atomicOr(&c->status, kStTimeout);
        const long long qb = rs.q0 + threadIdx.x;
        for (int l0 = 0; l0 < rs.nq; l0 += 8 * kThreads) {
            uint32_t bits = 0;
#pragma unroll 2
            for (int k = 0; k < 8; ++k) {
                const int lq = l0 + k * kThreads + (int)threadIdx.x;
                if (lq < rs.nq) {
                    const long long j0 = (rs.q0 + lq) * 4;
                    const float4 v4 = rs.V[lq];
                    int4 i4 = rs.ring[lq];
                    uint32_t r4 = rs.ref[lq];
                    *reinterpret_cast<int4 *>(ring + j0) = make_int4(0, 0, 0, 0);
                    if (inj) i4 = take_restored(inj + j0, i4);
                    if (cur) *reinterpret_cast<int4 *>(cur + j0) = i4;
                    // rs.V holds the leaked potentials and rs.ext the drive
                    // (pre_update, during the last grid barrier)
                    const int4 e4 = rs.ext[lq];
                    float vv[4] = {v4.x, v4.y, v4.z, v4.w};
                    const int32_t ii[4] = {i4.x, i4.y, i4.z, i4.w};
                    const uint32_t ex[4] = {(uint32_t)e4.x, (uint32_t)e4.y, (uint32_t)e4.z, (uint32_t)e4.w};
                    unsigned int m = 0;
                    uint32_t r_out = 0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint32_t r = (r4 >> (8 * q)) & 0xFFu;
                        if (lif_finish(d, ex[q], ii[q], vv[q], r)) m |= 1u << q;
                        r_out |= r << (8 * q);
                        if (do_hash) {
                            const uint32_t g = d.gid ? d.gid[j0 + q] : (uint32_t)(j0 + q);
                            hc += mix64(((unsigned long long)g << 32) | (uint32_t)ii[q]);
                            hv += mix64(((unsigned long long)g << 32) | __float_as_uint(vv[q]));
                        }
                    }
                    prefetch_rows(d, j0, m);
                    bits |= m << (4 * k);
                    rs.V[lq] = make_float4(vv[0], vv[1], vv[2], vv[3]);
                    rs.ref[lq] = r_out;
                }
            }
            prof_stamp(sh, 0);
            compact_spikes(d, t, sh, bits,
                          [&](int b) { return (uint32_t)((qb + l0 + (b >> 2) * kThreads) * 4 + (b & 3)); });
            prof_stamp(sh, 1);
        }
    } else if constexpr (MODE == kModeVec) {
        const long long nq = d.M / 4, stride = (long long)gridDim.x * kThreads;
        const long long qb = (long long)blockIdx.x * kThreads + threadIdx.x;
        // NCH chunks of 8 quads per thread, their spikes compacted together
        constexpr int NCH = QB > 1 ? 4 : 1;
        for (long long B = (long long)blockIdx.x * kThreads; B < nq; B += NCH * 8 * stride) {
        uint32_t bw[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) bw[c] = 0u;
        for (int c = 0; c < NCH; ++c) {
            const long long b0 = B + c * 8 * stride;
            if (b0 >= nq) break;  // (block-uniform)
            uint32_t bits = 0;
            // QB quads' state loaded before any of them is written back, so
            // that their loads are in flight together
            for (int k0 = 0; k0 < 8; k0 += QB) {
                float4 v4[QB];
                int4 i4[QB];
                uint32_t r4[QB];
#pragma unroll
                for (int k = 0; k < QB; ++k) {
                    const long long q = b0 + (k0 + k) * stride + threadIdx.x;
                    if (q < nq) {
                        v4[k] = *reinterpret_cast<const float4 *>(d.V + q * 4);
                        i4[k] = *reinterpret_cast<const int4 *>(ring + q * 4);
                        r4[k] = *reinterpret_cast<const uint32_t *>(d.ref + q * 4);
                    }
                }
#pragma unroll
                for (int k = 0; k < QB; ++k) {
                    const long long q = b0 + (k0 + k) * stride + threadIdx.x;
                    if (q < nq) {
                        const long long j0 = q * 4;
                        *reinterpret_cast<int4 *>(ring + j0) = make_int4(0, 0, 0, 0);
                        if (inj) i4[k] = take_restored(inj + j0, i4[k]);
                        if (cur) *reinterpret_cast<int4 *>(cur + j0) = i4[k];
                        float vv[4] = {v4[k].x, v4[k].y, v4[k].z, v4[k].w};
                        const int32_t ii[4] = {i4[k].x, i4[k].y, i4[k].z, i4[k].w};
                        const unsigned int m = update_quad(d, sh.th, t, j0, vv, ii, r4[k], do_hash, hc, hv);
                        prefetch_rows(d, j0, m);
                        bits |= m << (4 * (k0 + k));
                        *reinterpret_cast<float4 *>(d.V + j0) = make_float4(vv[0], vv[1], vv[2], vv[3]);
                        *reinterpret_cast<uint32_t *>(d.ref + j0) = r4[k];
                    }
                }
            }
            bw[c] = bits;
        }
        const long long base = B - (long long)blockIdx.x * kThreads;
        prof_stamp(sh, 0);
        compact_spikes_multi<NCH>(d, t, sh, bw, [&](int c, int b) {
            return (uint32_t)((qb + base + (long long)c * 8 * stride + (b >> 2) * stride) * 4 + (b & 3));
        });
        prof_stamp(sh, 1);
        }
    } else {
        const long long stride = (long long)gridDim.x * kThreads;
        const long long jb = (long long)blockIdx.x * kThreads + threadIdx.x;
        for (long long b0 = (long long)blockIdx.x * kThreads; b0 < d.M; b0 += 32 * stride) {
            uint32_t bits = 0;
            for (int k = 0; k < 32; ++k) {
                const long long j = b0 + k * stride + threadIdx.x;
                if (j < d.M) {
                    float v = d.V[j];
                    int32_t irec = ring[j];
                    uint32_t r = d.ref[j];
                    ring[j] = 0;
                    if (inj) {
                        irec = (int32_t)((uint32_t)irec + (uint32_t)inj[j]);
                        inj[j] = 0;
                    }
                    if (cur) cur[j] = irec;
                    const uint32_t g = d.gid ? d.gid[j] : (uint32_t)j;
                    const Drive dr = drive_of(d, sh.th, g);
                    const uint32_t u =
                        uint4_word(philox4(dr.key0, dr.key1, (uint32_t)((g - dr.off) >> 2), (uint32_t)t), g & 3u);
                    if (lif_neuron(d, dr, u, irec, v, r)) {
                        bits |= 1u << k;
                        prefetch_rows(d, j, 1u);
                    }
                    if (do_hash) {
                        hc += mix64(((unsigned long long)g << 32) | (uint32_t)irec);
                        hv += mix64(((unsigned long long)g << 32) | __float_as_uint(v));
                    }
                    d.V[j] = v;
                    d.ref[j] = (uint8_t)r;
                }
            }
            const long long base = b0 - (long long)blockIdx.x * kThreads;
            compact_spikes(d, t, sh, bits, [&](int b) { return (uint32_t)(jb + base + b * stride); });
        }
    }
    if (do_hash) {
        hc = warp_sum(hc);
        hv = warp_sum(hv);
        if (lane == 0) {
            sh.h[0][wid] = hc;
            sh.h[1][wid] = hv;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long a = 0, b = 0;
            for (int w = 0; w < kWarps; ++w) {
                a += sh.h[0][w];
                b += sh.h[1][w];
            }
            atomicAdd(&d.hash[2 * t], a);
            atomicAdd(&d.hash[2 * t + 1], b);
        }
    }
}

// Second half of step t (all threads call): a4-a6 for this block's share of
// the step's spikes, an equal share of the list for every block, and their
// raster copy.
template <int RT>
__device__ __forceinline__ void route_step(const Dev &d, long long t, StepShared &sh, bool carried = false,
                                           Deferred *df = nullptr, int cur = 0)
{
    const Stage sg{sh.lng, sh.sht, &sh.nl, &sh.ns, sh.tally, sh.e0, sh.f0, sh.pre1, sh.pre2, sh.part,
                   sh.arec, sh.atag, &sh.an, sh.ak, sh.abase};
    Ctrl *c = d.ctrl;
    // delivery by arrival step: everything this step delivers goes to the
    // next step's input slot
    int32_t *fix = RT == kRtArrival ? d.acc + (size_t)((t + 1) & 1) * (size_t)d.M : nullptr;
    const int tmod = RT == kRtArrival ? (int)(t % d.n_arr) : RT == kRtOwner ? (int)(t % d.n_own) : 0;
    if (threadIdx.x == 0) {
        if (carried) {
            // k_persist: the step's spike count from the barrier word (the sum
            // of the blocks' counts less the last one) and the raster head
            // this block carries from step to step as close_step does
            const uint32_t hiw = (uint32_t)(sh.word >> 32);
            sh.tot = hiw - sh.prevS;
            sh.prevS = hiw;
            sh.head = sh.headv;
            sh.headv = next_head(d, sh.headv, sh.tot, t);
        } else {
            // one thread reads the step words: every warp loading them would
            // queue thousands of requests on one L2 line
            sh.tot = *(volatile unsigned int *)&c->S_acc[slot3(t)];
            sh.head = *(volatile long long *)&c->head[slot3(t)];
        }
    }
    if (threadIdx.x < kWarps * kTally) (&sh.tally[0][0])[threadIdx.x] = 0u;
    if (df && threadIdx.x == 0) {
        df->nl[cur] = 0u;
        df->ns[cur] = 0u;
    }
    __syncthreads();
    const unsigned long long S = sh.tot;
    const unsigned int lo = (unsigned int)(S * blockIdx.x / gridDim.x);
    const unsigned int hi = (unsigned int)(S * (blockIdx.x + 1) / gridDim.x);
    const int par = (int)(t & 1);
    const int tm = (int)(t % d.D);
    // with df: the delay >= 2 lists of step t - 1 (slot base of that step),
    // delivered by some warps while the others walk the first round's tables
    const int prev = cur ^ 1;
    const int tmp = (int)((t - 1 + d.D) % d.D);
    const unsigned int pl = df ? min(df->nl[prev], (unsigned int)kDefLong) : 0u;
    const unsigned int ps = df ? min(df->ns[prev], (unsigned int)kDefShort) : 0u;
    if (df && lo >= hi)
        tally_add(sg, 0, deliver_lists(d, tmp, nullptr, df->lng[prev], pl, df->sht[prev], ps, 0, kWarps));
    for (unsigned int b = lo; b < hi; b += kRound) {
        const unsigned int nr = min(hi - b, (unsigned int)kRound);
        const bool split = df && b == lo;
        Pending pn{0, 0u, make_ulonglong2(0ull, 0ull), 0ull, 0u, 0u};
        prof_stamp(sh, 5);
        if (!split || threadIdx.x < kTravWarps * 32)
            pn = route_traverse<RT>(d, par, tm, b, nr, sg, split ? kTravWarps * 32 : kThreads, df, cur, fix, tmod);
        else
            tally_add(sg, 0,
                      deliver_lists(d, tmp, nullptr, df->lng[prev], pl, df->sht[prev], ps, kTravWarps,
                                    kWarps - kTravWarps));
        __syncthreads();
        prof_stamp(sh, 4);
        route_finish<RT>(d, tm, fix, sg, pn);
        __syncthreads();
    }
    if (sh.head >= 0)
        for (unsigned int k = lo + threadIdx.x; k < hi; k += kThreads) d.spk[sh.head + k] = d.spk_step[k];
    // tallies of the routed spikes into this block's row (no other block
    // touches it: the reductions never wait on another block)
    __syncthreads();
    if (threadIdx.x < kTally) {
        unsigned long long a = 0;
        for (int w = 0; w < kWarps; ++w) a += sh.tally[w][threadIdx.x];
        if (a) atomicAdd(&d.tally[(size_t)blockIdx.x * C_N + C_EVENTS + threadIdx.x], a);
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
// Step t = ctrl->t + k of a captured graph: k_update (a1-a3) then k_route
// (a4-a6).  Block 0 of k_update closes step t - 1 (the graph's first step was
// closed by the graph before); k_advance closes the graph's last step and
// moves ctrl->t past its steps.
template <int MODE, bool ARR>
__global__ void __launch_bounds__(kThreads) k_update(const Dev d, int k)
{
    __shared__ StepShared sh;
    pdl_enter();
    if (threadIdx.x == 0) {
        sh.t0 = *(volatile long long *)&d.ctrl->t;
        sh.inj_until = *(volatile long long *)&d.ctrl->inject_until;
        sh.prof_on = 0;
        sh.arec = nullptr;
        sh.atag = nullptr;
    }
    __syncthreads();
    const long long t = sh.t0 + k;
    if (k > 0 && blockIdx.x == 0 && threadIdx.x == 0) close_step(d, t - 1);
    // one quad per thread on this grid: no batching of the loads
    update_step<MODE, ARR, 1>(d, t, sh, Resident{}, 0u, 0ull);
    // delivery by arrival step: the runs queued for this step (they go to
    // the next step's input slot, which no block reads in this kernel)
    if constexpr (ARR) arrival_share<8>(d, t, sh);
}

template <bool ARR>
__global__ void __launch_bounds__(kThreads) k_route(const Dev d, int k)
{
    __shared__ StepShared sh;
    __shared__ ArrivalPool<ARR> pool;
    pdl_enter();
    if (threadIdx.x == 0) {
        sh.t0 = *(volatile long long *)&d.ctrl->t;
        sh.prof_on = 0;
        sh.arec = pool.r();
        sh.atag = pool.g();
    }
    __syncthreads();
    route_step<ARR ? kRtArrival : kRtRing>(d, sh.t0 + k, sh);
}

__global__ void k_advance(const Dev d, int steps)
{
    pdl_enter();
    const long long t = d.ctrl->t;
    if (steps > 0) close_step(d, t + steps - 1);
    d.ctrl->t = t + steps;
}

// ---------------------------------------------------------------- persistent
// T steps in one cooperative launch: update_step, grid barrier, route_step,
// grid barrier.  Block 0 closes step t - 1 while step t updates and the last
// step after the final barrier.  Every wait is bounded (limit_ns per barrier
// and per bulk copy); a timeout ends the run with kStTimeout in the status
// word.  With phase_ns set, block 0 sums its own work of both halves and its
// waits at the two barriers.  skip_arrival
// (tests of the bounded wait only): block 0 waits at the first barrier
// without arriving, so every block's wait runs out.  In kModeSmem block b
// owns quads [b cq, (b + 1) cq) (cq = Dev::chunk_q) and keeps their V and
// ref in dynamic shared memory from the launch's start to its end, and the
// second barrier of a step is split: between its arrival and its wait the
// block computes the next step's drive and leak (pre_update), which need no
// other block's data.  DEFER: minimum-delay batching (Deferred); the last
// step's delay >= 2 lists are delivered before the launch ends.
// Blocks per SM the persistent kernel is built for (MINB): 3 with the neuron
// state in shared memory (80 registers); on global state 2 (128 registers,
// four quads' loads batched) or 3 (80 registers, two quads batched: more
// warps per SM for the latency-bound halves).
template <int MINB>
__host__ __device__ constexpr int persist_quad_batch()
{
    return MINB >= 3 ? 2 : 4;
}

template <int MODE, bool DEFER, bool ARR, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_persist(const Dev d, int T,
                                                                                   unsigned long long limit_ns,
                                                         int skip_arrival)
{
    __shared__ StepShared sh;
    __shared__ ArrivalPool<ARR> pool;
    __shared__ DeferSlot<DEFER> dslot;
    Deferred *df = dslot.get();
    __shared__ __align__(8) unsigned long long s_bar;
    extern __shared__ __align__(128) unsigned char s_dyn[];
    Ctrl *c = d.ctrl;
    Resident rs{};
    if constexpr (MODE == kModeSmem) {
        const long long cq = d.chunk_q;
        rs.V = reinterpret_cast<float4 *>(s_dyn);
        rs.ring = reinterpret_cast<int4 *>(s_dyn + cq * 16);
        rs.ext = reinterpret_cast<int4 *>(s_dyn + cq * 32);
        rs.ref = reinterpret_cast<uint32_t *>(s_dyn + cq * 48);
        rs.bar = &s_bar;
        rs.q0 = (long long)blockIdx.x * cq;
        rs.nq = (int)max(0ll, min(cq, d.M / 4 - rs.q0));
        for (int lq = threadIdx.x; lq < rs.nq; lq += kThreads) {
            rs.V[lq] = reinterpret_cast<const float4 *>(d.V)[rs.q0 + lq];
            rs.ref[lq] = reinterpret_cast<const uint32_t *>(d.ref)[rs.q0 + lq];
        }
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sh.t0 = *(volatile long long *)&c->t;
        sh.inj_until = *(volatile long long *)&c->inject_until;
        sh.headv = *(volatile long long *)&c->head[slot3(sh.t0)];
        sh.prevS = 0u;
        sh.arec = pool.r();
        sh.atag = pool.g();
        if constexpr (DEFER) {
            df->nl[0] = df->nl[1] = 0u;
            df->ns[0] = df->ns[1] = 0u;
        }
    }
    if (threadIdx.x < kPTab) sh.th[threadIdx.x] = d.th32[threadIdx.x];
    __syncthreads();
    const long long t0 = sh.t0;
    if constexpr (MODE == kModeSmem) {
        if (T > 0) pre_update(d, t0, sh.th, rs);
    }
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    // profiling: each part's time is added to sh.prof as soon as it ends
    const bool prof = d.phase_ns != nullptr && lead;
    if (threadIdx.x == 0) {
        sh.prof_on = prof ? 1 : 0;
        for (int k = 0; k <= kPhases; ++k) sh.prof[k] = 0;
    }
    __syncthreads();
    auto stamp = [&](int k) { prof_stamp(sh, k); };
    int done = 0, issued = 0;
    long long closed = t0 - 1;
    for (int s = 0; s < T; ++s) {
        const long long t = t0 + s;
        stamp(-1);
        if (s > 0 && lead) {
            close_step(d, t - 1);
            closed = t - 1;
        }
        update_step<MODE, ARR, persist_quad_batch<MINB>()>(d, t, sh, rs, (uint32_t)(s & 1), limit_ns);
        ++issued;
        stamp(1);
        // the first barrier carries the block's spike count in the word's high half
        grid_arrive(c, 2ull * s, d.bar_groups, !(skip_arrival && s == 0 && blockIdx.x == 0),
                    1ull + ((unsigned long long)sh.n_own << 32));
        prefetch_own(d, sh);
        // delivery by arrival step: the runs queued for this step, while the
        // barrier completes (they need no spike of this step)
        if constexpr (ARR) arrival_share<(MODE == kModeSmem || MINB >= 3) ? 4 : 8>(d, t, sh);
        stamp(2);
        if (!grid_wait(c, 2ull * s, d.bar_groups, limit_ns, &sh.word)) break;
        stamp(3);
        route_step<ARR ? kRtArrival : kRtRing>(d, t, sh, true, df, s & 1);
        stamp(5);
        // the next step's input-free update runs while the barrier completes
        grid_arrive(c, 2ull * s + 1ull, d.bar_groups);
        if constexpr (MODE == kModeSmem) {
            if (s + 1 < T) pre_update(d, t + 1, sh.th, rs);
        } else if constexpr (MODE == kModeVec) {
            if (s + 1 < T && d.prefetch_state) prefetch_state_vec<ARR>(d, t + 1);
        }
        if (!grid_wait(c, 2ull * s + 1ull, d.bar_groups, limit_ns)) break;
        stamp(6);
        ++done;
    }
    if constexpr (DEFER) {
        if (T > 0 && done == T) {
            // the last step's delay >= 2 lists: their slots are read by the
            // next launch's steps, after this one ends
            const Stage sg{sh.lng, sh.sht, &sh.nl, &sh.ns, sh.tally, sh.e0, sh.f0, sh.pre1, sh.pre2, sh.part,
                           sh.arec, sh.atag, &sh.an, sh.ak, sh.abase};
            const int last = (T - 1) & 1;
            if (threadIdx.x < kWarps * kTally) (&sh.tally[0][0])[threadIdx.x] = 0u;
            __syncthreads();
            tally_add(sg, 0,
                      deliver_lists(d, (int)((t0 + T - 1) % d.D), nullptr, df->lng[last],
                                    min(df->nl[last], (unsigned int)kDefLong), df->sht[last],
                                    min(df->ns[last], (unsigned int)kDefShort), 0, kWarps));
            __syncthreads();
            if (threadIdx.x < kTally) {
                unsigned long long a = 0;
                for (int w = 0; w < kWarps; ++w) a += sh.tally[w][threadIdx.x];
                if (a) atomicAdd(&d.tally[(size_t)blockIdx.x * C_N + C_EVENTS + threadIdx.x], a);
            }
        }
    }
    if constexpr (MODE == kModeSmem) {
        // after a timeout, give this block's last bulk copy a bounded wait
        // before its shared memory is released
        __syncthreads();
        if (rs.nq > 0 && issued > 0 && (*(volatile unsigned int *)&c->status & kStTimeout))
            mbar_wait(rs.bar, (uint32_t)((issued - 1) & 1), limit_ns);
        // the resident state goes back to global memory
        for (int lq = threadIdx.x; lq < rs.nq; lq += kThreads) {
            reinterpret_cast<float4 *>(d.V)[rs.q0 + lq] = rs.V[lq];
            reinterpret_cast<uint32_t *>(d.ref)[rs.q0 + lq] = rs.ref[lq];
        }
    }
    if (lead) {
        if (t0 + done - 1 > closed) close_step(d, t0 + done - 1);
        c->t = t0 + done;
        if (prof)
            for (int k = 0; k < kPhases; ++k) d.phase_ns[k] += sh.prof[k];
    }
}


// ---------------------------------------------------------------- partition-owned delivery
// Delivery into each partition's own input: at step t the block that owns
// partition q adds the runs on q's list of step t (the runs of every delay
// whose arrival step is t, queued by the routing of steps t - 8 .. t - 1)
// into a shared-memory accumulator with shared-memory reductions, then runs
// a1-a3 on q's neurons from it.  No global input slot, no global reductions:
// each partition receives its messages and delivers them into its own
// neurons, as each GPU of the paper's system does (Sec. I, Sec. IV.B).

// Shared-memory reduction at p (a shared-memory address).
__device__ __forceinline__ void red_shared_add(const int32_t *p, int32_t v)
{
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}

// The records recs[0, n) (offset << 24 | length) into acc[target - b0], all
// warps of the block: a warp numbers the synapses of 32 runs through and
// takes them U per lane with every load in flight (as deliver_records).
template <int U>
__device__ __forceinline__ void owner_deliver(const Dev &d, int32_t *acc, long long b0,
                                              const unsigned long long *recs, unsigned long long n)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long step = (unsigned long long)kWarps * 32u;
    unsigned long long b = (unsigned long long)wid * 32u;
    unsigned long long rec = (b + lane < n) ? __ldcs(recs + b + lane) : 0ull;
    for (; b < n; b += step) {
        const unsigned long long nx = b + step + (unsigned long long)lane;
        const unsigned long long rec_next = nx < n ? __ldcs(recs + nx) : 0ull;
        const unsigned long long o = rec >> kLenBits;
        const unsigned int len = (unsigned int)(rec & kLenMask);
        unsigned int inc = len;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, inc, k);
            if (lane >= k) inc += y;
        }
        const unsigned int ex = inc - len;
        const unsigned int tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
        for (unsigned int base = 0; base < tot; base += 32u * U) {
            uint32_t td[U];
            int32_t w[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const unsigned int y = base + (unsigned int)k * 32u + (unsigned int)lane;
                int r = 0;
#pragma unroll
                for (int h = 16; h > 0; h >>= 1) {
                    const unsigned int v = __shfl_sync(0xFFFFFFFFu, ex, r + h);
                    if (v <= y) r += h;
                }
                const unsigned long long orr = __shfl_sync(0xFFFFFFFFu, o, r);
                const unsigned int er = __shfl_sync(0xFFFFFFFFu, ex, r);
                if (y < tot) {
                    td[k] = __ldcs(d.syn_td + orr + (y - er));
                    w[k] = __ldcs(d.syn_w + orr + (y - er));
                }
            }
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const unsigned int y = base + (unsigned int)k * 32u + (unsigned int)lane;
                if (y < tot) red_shared_add(acc + ((long long)(td[k] & kTgtMask) - b0), w[k]);
            }
        }
        rec = rec_next;
    }
}

// a1 + a2 of neuron j with recurrent input irec (scalar path of the owner's
// partition ends); returns true on a spike.
__device__ __forceinline__ bool owner_neuron(const Dev &d, const uint32_t *th, long long t, long long j, int32_t irec,
                                             bool do_hash, unsigned long long &hc, unsigned long long &hv)
{
    float v = d.V[j];
    uint32_t r = d.ref[j];
    const uint32_t g = d.gid ? d.gid[j] : (uint32_t)j;
    const Drive dr = drive_of(d, th, g);
    const uint32_t u = uint4_word(philox4(dr.key0, dr.key1, (uint32_t)((g - dr.off) >> 2), (uint32_t)t), g & 3u);
    const bool spk = lif_neuron(d, dr, u, irec, v, r);
    if (do_hash) {
        hc += mix64(((unsigned long long)g << 32) | (uint32_t)irec);
        hv += mix64(((unsigned long long)g << 32) | __float_as_uint(v));
    }
    d.V[j] = v;
    d.ref[j] = (uint8_t)r;
    return spk;
}

// Phase A of step t for the partitions this block owns (q = blockIdx.x,
// + gridDim.x, ...): the partition's queued runs of step t into the
// shared accumulator acc, then a1-a3 on its neurons (all threads call).
__device__ __forceinline__ void owner_update(const Dev &d, long long t, StepShared &sh, int32_t *acc)
{
    Ctrl *c = d.ctrl;
    const int par = (int)(t & 1);
    const int slot = (int)(t % d.D);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool do_hash = t < d.hash_steps;
    const bool do_cur = d.cur_every > 0 && (t % d.cur_every) == 0 && (t / d.cur_every) < d.cur_slots;
    int32_t *inj = t < sh.inj_until ? d.ring + (long long)slot * d.M : nullptr;
    int32_t *cur = do_cur ? d.cur_rec + (t / d.cur_every) * d.M : nullptr;
    const int li = (int)(t % d.n_own);
    {
        // clear the other parity of the exchange counters (used by step t - 1
        // only) and the spike count of step t + 1
        uint32_t *b1 = bucket_cnt_of(d, par ^ 1), *i1 = inbox_cnt_of(d, par ^ 1);
        const int nb = d.n_bpair, ni = nb + d.n_ipair;
        for (int x = blockIdx.x * kThreads + threadIdx.x; x < ni; x += gridDim.x * kThreads) {
            if (x < nb) b1[(size_t)x * kPairStride] = 0;
            else i1[(size_t)(x - nb) * kPairStride] = 0;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) c->S_acc[slot3(t + 1)] = 0;
    }
    if (threadIdx.x < kPTab) sh.th[threadIdx.x] = d.th32[threadIdx.x];
    if (threadIdx.x == 0) sh.n_own = 0u;
    unsigned long long hc = 0, hv = 0;
    for (int q = blockIdx.x; q < d.P; q += gridDim.x) {
        const long long b0 = d.pbase[q], b1 = d.pbase[q + 1];
        const int n = (int)(b1 - b0);
        for (int x = threadIdx.x; x < n; x += kThreads) acc[x] = 0;
        __syncthreads();
        // the runs arriving at q at step t
        const ulonglong2 sl = d.inb_slot[q];
        unsigned int *cnt = &d.inb_cnt[((size_t)q * d.n_own + li) * kPairStride];
        if (threadIdx.x == 0) sh.arr_n = min(*(volatile unsigned int *)cnt, (unsigned int)sl.y);
        __syncthreads();
        owner_deliver<8>(d, acc, b0, d.inb + sl.x + (unsigned long long)li * sl.y, sh.arr_n);
        __syncthreads();
        // the list is consumed: step t's routing refills it for step t + n_own
        if (threadIdx.x == 0) *cnt = 0u;
        prof_stamp(sh, 0);
        // a1 + a2: quads of 4 aligned ids [qa, qb), the ends one by one
        const long long qa = (b0 + 3) / 4, qb = b1 / 4;
        const int nh = qa * 4 > b1 ? n : (int)(qa * 4 - b0);           // head neurons
        const int nt = qb >= qa ? (int)(b1 - qb * 4) : 0;              // tail neurons
        constexpr int NCH = 4, QB = 4;
        const long long stride = kThreads;
        uint32_t bx = 0;  // head / tail spikes of this thread (bit 0)
        long long jx = -1;
        if (threadIdx.x < nh + nt) {
            jx = threadIdx.x < nh ? b0 + threadIdx.x : qb * 4 + (threadIdx.x - nh);
            int32_t irec = acc[jx - b0];
            if (inj) {
                irec = (int32_t)((uint32_t)irec + (uint32_t)inj[jx]);
                inj[jx] = 0;
            }
            if (cur) cur[jx] = irec;
            if (owner_neuron(d, sh.th, t, jx, irec, do_hash, hc, hv)) {
                bx = 1u;
                prefetch_rows(d, jx, 1u);
            }
        }
        bool first = true;
        for (long long B = qa + threadIdx.x; first || B - threadIdx.x < qb; B += NCH * 8 * stride) {
            // (block-uniform trip count; the head/tail word joins the first compaction)
            uint32_t bw[NCH + 1];
#pragma unroll
            for (int k = 0; k <= NCH; ++k) bw[k] = 0u;
            for (int cc = 0; cc < NCH; ++cc) {
                for (int k0 = 0; k0 < 8; k0 += QB) {
                    float4 v4[QB];
                    uint32_t r4[QB];
#pragma unroll
                    for (int k = 0; k < QB; ++k) {
                        const long long Q = B + (cc * 8 + k0 + k) * stride;
                        if (Q < qb) {
                            v4[k] = *reinterpret_cast<const float4 *>(d.V + Q * 4);
                            r4[k] = *reinterpret_cast<const uint32_t *>(d.ref + Q * 4);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < QB; ++k) {
                        const long long Q = B + (cc * 8 + k0 + k) * stride;
                        if (Q < qb) {
                            const long long j0 = Q * 4;
                            const int a = (int)(j0 - b0);
                            int4 i4 = make_int4(acc[a], acc[a + 1], acc[a + 2], acc[a + 3]);
                            if (inj) i4 = take_restored(inj + j0, i4);
                            if (cur) *reinterpret_cast<int4 *>(cur + j0) = i4;
                            float vv[4] = {v4[k].x, v4[k].y, v4[k].z, v4[k].w};
                            const int32_t ii[4] = {i4.x, i4.y, i4.z, i4.w};
                            const unsigned int m = update_quad(d, sh.th, t, j0, vv, ii, r4[k], do_hash, hc, hv);
                            prefetch_rows(d, j0, m);
                            bw[cc] |= m << (4 * (k0 + k));
                            *reinterpret_cast<float4 *>(d.V + j0) = make_float4(vv[0], vv[1], vv[2], vv[3]);
                            *reinterpret_cast<uint32_t *>(d.ref + j0) = r4[k];
                        }
                    }
                }
            }
            if (first) bw[NCH] = bx;
            const long long Bb = B - threadIdx.x;
            const long long jxx = jx;
            prof_stamp(sh, 0);
            compact_spikes_multi<NCH + 1>(d, t, sh, bw, [&](int cc, int b) {
                if (cc == NCH) return (uint32_t)jxx;
                return (uint32_t)((Bb + threadIdx.x + (long long)cc * 8 * stride + (b >> 2) * stride) * 4 + (b & 3));
            });
            prof_stamp(sh, 1);
            first = false;
        }
        __syncthreads();  // the accumulator is reused by the next partition
    }
    if (do_hash) {
        hc = warp_sum(hc);
        hv = warp_sum(hv);
        if (lane == 0) {
            sh.h[0][wid] = hc;
            sh.h[1][wid] = hv;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long a = 0, b = 0;
            for (int w = 0; w < kWarps; ++w) {
                a += sh.h[0][w];
                b += sh.h[1][w];
            }
            atomicAdd(&d.hash[2 * t], a);
            atomicAdd(&d.hash[2 * t + 1], b);
        }
    }
}

// T steps in one cooperative launch with partition-owned delivery: phase A
// (owner_update), grid barrier, the routing half (route_step<kRtOwner>),
// grid barrier.  Bounded waits, closing of steps and the skip_arrival test
// switch as in k_persist.  Dynamic shared memory: the accumulator of the
// largest partition.
__global__ void __launch_bounds__(kThreads, 2) k_owner(const Dev d, int T, unsigned long long limit_ns,
                                                       int skip_arrival)
{
    __shared__ StepShared sh;
    extern __shared__ __align__(16) int32_t s_acc[];
    Ctrl *c = d.ctrl;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    if (threadIdx.x == 0) {
        sh.t0 = *(volatile long long *)&c->t;
        sh.inj_until = *(volatile long long *)&c->inject_until;
        sh.headv = *(volatile long long *)&c->head[slot3(sh.t0)];
        sh.prevS = 0u;
        sh.arec = nullptr;
        sh.atag = nullptr;
        sh.prof_on = (d.phase_ns != nullptr && lead) ? 1 : 0;
        for (int k = 0; k <= kPhases; ++k) sh.prof[k] = 0;
    }
    __syncthreads();
    const long long t0 = sh.t0;
    int done = 0;
    long long closed = t0 - 1;
    for (int s = 0; s < T; ++s) {
        const long long t = t0 + s;
        prof_stamp(sh, -1);
        if (s > 0 && lead) {
            close_step(d, t - 1);
            closed = t - 1;
        }
        owner_update(d, t, sh, s_acc);
        prof_stamp(sh, 1);
        grid_arrive(c, 2ull * s, d.bar_groups, !(skip_arrival && s == 0 && blockIdx.x == 0),
                    1ull + ((unsigned long long)sh.n_own << 32));
        prefetch_own(d, sh);
        prof_stamp(sh, 2);
        if (!grid_wait(c, 2ull * s, d.bar_groups, limit_ns, &sh.word)) break;
        prof_stamp(sh, 3);
        route_step<kRtOwner>(d, t, sh, true, nullptr, 0);
        prof_stamp(sh, 5);
        grid_arrive(c, 2ull * s + 1ull, d.bar_groups);
        if (!grid_wait(c, 2ull * s + 1ull, d.bar_groups, limit_ns)) break;
        prof_stamp(sh, 6);
        ++done;
    }
    if (lead) {
        if (t0 + done - 1 > closed) close_step(d, t0 + done - 1);
        c->t = t0 + done;
        if (sh.prof_on)
            for (int k = 0; k < kPhases; ++k) d.phase_ns[k] += sh.prof[k];
    }
}

}  // namespace
