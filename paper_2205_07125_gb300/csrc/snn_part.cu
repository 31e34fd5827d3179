// Device partitioner (sm_103a): Algorithm 1 (Sec. IV.A) with batched
// growth, the parallel form of the greedy that the paper leaves as future
// work (Sec. VII, parallelization of algorithms).
//
// One cooperative launch per iteration t grows parts 0..P-2 one after the
// other; the last part takes the rest; the host keeps the iteration with the
// smallest objective.  A part grows in rounds:
//   scatter  the members that joined in the last round add their weight W_a
//            to acc[j] of every neuron j they share a synapse with (either
//            direction, with multiplicity): gain(j) = W_j * acc[j] is
//            sum_{i in part} (c_ij + c_ji) W_i W_j;
//   select   the `need` unassigned neurons with the largest gains (ties:
//            lowest id) by a radix select over unique 64-bit keys
//            (gain << idbits | (2^idbits - 1 - j)), 11 bits per pass, one
//            shared-memory histogram per block merged into a global one;
//   join     block 0 sorts the round's members by key and lets them join in
//            that order until the part's weight reaches sum(W)/P.
// need = min(B, unassigned, max(1, n_k / g)) (g = 0 drops the last term),
// n_k = the part's size so far.  Every step is integer arithmetic, so the
// result does not depend on the order of the atomic additions: it equals the
// sequential reading with the same rounds bit for bit, and with B = 1 the
// one-neuron-at-a-time greedy.  Grid barriers are bounded (a block that
// waits past the limit records a timeout and the launch ends).
#include <cuda_runtime.h>

#include "snn_internal.h"

namespace {

constexpr int kPT = 256;                 // threads per block
constexpr int kPW = kPT / 32;
constexpr int kDigit = 11;               // radix digit bits
constexpr int kBins = 1 << kDigit;
constexpr int kMaxPass = (64 + kDigit - 1) / kDigit;
constexpr int kMaxBatch = 2048;          // largest round
constexpr int kChunk = 256;              // synapses per scatter task

constexpr uint32_t kPStTimeout = 1u, kPStRange = 2u, kPStFault = 4u;

struct PCtl {
    alignas(128) unsigned long long bar;  // grid-barrier arrivals of the running launch
    alignas(128) unsigned int nsel;       // members found by the selection
    alignas(128) unsigned int status;
    unsigned int seed_id;                 // seed of part k: lowest unassigned id (t == 1, atomicMin) or the
                                          // drawn one (t > 1); all ones between parts
    int stop;                             // part k is full
    int na;                               // members that joined in the last round
    long long wk, nk, n_un;               // weight and size of part k, unassigned neurons
    unsigned long long obj;               // objective of the iteration
    // setup results
    unsigned long long gain_max;          // largest possible gain
    unsigned long long deg_max;           // largest out- or in-degree
};

struct PDev {
    const long long *ptr;       // [M+1] out-synapses of each neuron
    const uint32_t *tgt;        // [E]
    long long *in_ptr;          // [M+1] in-synapses of each neuron
    uint32_t *in_src;           // [E]
    uint32_t *W;                // [M] out-degree
    unsigned long long *acc;    // [M] weight shared with the growing part
    unsigned long long *key;    // [M] selection key of the round (0: assigned)
    int32_t *lab;               // [M] part of each neuron (-1: unassigned)
    uint32_t *fill;             // [M] in-degree counters of the in-list build
    uint32_t *hist;             // [2][kMaxPass][kBins] by round parity
    unsigned long long *sel;    // [kMaxBatch] keys of the round's members
    uint32_t *added;            // [kMaxBatch] members that joined in the last round
    uint32_t *cnt;              // [grid] unassigned neurons per block
    const uint32_t *rword;      // [P] Philox words of the seeds (t > 1)
    unsigned long long *wpart;  // [P] part weights of the iteration
    PCtl *c;
    long long M, E, Wtot;
    int P, B, grow, t, idbits, nbits, npass, chunks;
    unsigned long long limit_ns;
};

__device__ __forceinline__ unsigned long long p_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded grid barrier number k of the launch (cooperative: every block is
// resident).  A block-wide barrier, a release add and acquire loads at GPU
// scope make the writes of every block before it visible after it.  Returns
// false (after recording kPStTimeout) when the wait runs out or another
// block's did.
__device__ __forceinline__ bool p_sync(PCtl *c, unsigned long long k, unsigned long long limit_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long target = (k + 1ull) * gridDim.x;
        asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(&c->bar) : "memory");
        const unsigned long long deadline = p_ns() + limit_ns;
        unsigned int spins = 0;
        for (;;) {
            unsigned long long v;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(&c->bar) : "memory");
            if (v >= target) break;
            if ((++spins & 15u) == 0u) {
                if (*(volatile unsigned int *)&c->status & kPStTimeout) {
                    ok = 0;
                    break;
                }
                if (p_ns() > deadline) {
                    atomicOr(&c->status, kPStTimeout);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(32);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class T>
__device__ __forceinline__ T p_block_sum(T v, T *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    T s = 0;
#pragma unroll
    for (int w = 0; w < kPW; ++w) s += sh[w];
    return s;
}

// Exclusive block scan of one value per thread (thread order).
template <class T>
__device__ __forceinline__ T p_block_excl(T v, T *sh, T &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    T base = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kPW; ++w) {
        if (w < wid) base += sh[w];
        tot += sh[w];
    }
    total = tot;
    return base + x - v;
}

// ------------------------------------------------------------------ setup
// Out-degrees, in-degree counts and the target range check.
__global__ void k_part_degrees(PDev d)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < d.M; i += stride)
        d.W[i] = (uint32_t)(d.ptr[i + 1] - d.ptr[i]);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < d.E; e += stride) {
        const uint32_t j = d.tgt[e];
        if (j < (unsigned long long)d.M) atomicAdd(&d.fill[j], 1u);
        else atomicOr(&d.c->status, kPStRange);
    }
}

// in_ptr = exclusive scan of the in-degrees (one block); fill goes back to
// zero for the per-target cursors of k_part_in_lists.
__global__ void __launch_bounds__(1024) k_part_scan(PDev d)
{
    __shared__ long long sh[32];
    const long long n = d.M;
    const long long per = (n + blockDim.x - 1) / blockDim.x;
    const long long a = min(n, (long long)threadIdx.x * per), b = min(n, a + per);
    long long s = 0;
    for (long long i = a; i < b; ++i) s += d.fill[i];
    // block-wide exclusive scan of the thread sums
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = s;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    long long base = 0;
    for (int w = 0; w < wid; ++w) base += sh[w];
    long long run = base + x - s;
    for (long long i = a; i < b; ++i) {
        d.in_ptr[i] = run;
        run += d.fill[i];
        d.fill[i] = 0;
    }
    if (threadIdx.x == blockDim.x - 1) d.in_ptr[n] = run;
}

// in_src: the sources of every neuron's in-synapses (list order is the
// atomics' order, which no later step depends on).  One warp per source.
__global__ void k_part_in_lists(PDev d)
{
    const int lane = threadIdx.x & 31;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = w0; i < d.M; i += nw)
        for (long long e = d.ptr[i] + lane; e < d.ptr[i + 1]; e += 32) {
            const uint32_t j = d.tgt[e];
            if (j >= (unsigned long long)d.M) continue;
            const uint32_t pos = atomicAdd(&d.fill[j], 1u);
            d.in_src[d.in_ptr[j] + pos] = (uint32_t)i;
        }
}

// Largest possible gain W_j * sum of W over j's synapses in both directions
// and the largest degree (for the selection key width and the scatter's
// chunking).  A gain that would not fit 64 bits records kPStRange.
__global__ void k_part_bounds(PDev d)
{
    const int lane = threadIdx.x & 31;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long j = w0; j < d.M; j += nw) {
        unsigned long long s = 0;
        for (long long e = d.ptr[j] + lane; e < d.ptr[j + 1]; e += 32) {
            const uint32_t x = d.tgt[e];
            if (x < (unsigned long long)d.M) s += d.W[x];
        }
        for (long long e = d.in_ptr[j] + lane; e < d.in_ptr[j + 1]; e += 32) s += d.W[d.in_src[e]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        if (lane == 0) {
            const unsigned long long wj = d.W[j];
            if (__umul64hi(wj, s) != 0ull) atomicOr(&d.c->status, kPStRange);
            atomicMax(&d.c->gain_max, wj * s);
            const unsigned long long dg = max(d.ptr[j + 1] - d.ptr[j], d.in_ptr[j + 1] - d.in_ptr[j]);
            atomicMax(&d.c->deg_max, dg);
        }
    }
}

// ------------------------------------------------------------------ growth
struct PShared {
    union {
        uint32_t hist[kBins];
        struct {
            unsigned long long key[kMaxBatch];
            long long pre[kMaxBatch];
        } s;
    } u;
    long long red64[kPW];
    unsigned long long redu[kPW];
    uint32_t red32[kPW];
    long long n_un, nk, wk;
    int stop, na, digit;
    unsigned long long above;
    unsigned int seed;
};

// Neuron slice [lo, hi) of this block.
__device__ __forceinline__ void p_slice(const PDev &d, long long &lo, long long &hi)
{
    lo = d.M * blockIdx.x / gridDim.x;
    hi = d.M * (blockIdx.x + 1) / gridDim.x;
}

// Thread 0 reads the control words written before the last barrier.
__device__ __forceinline__ void p_read_ctl(const PDev &d, PShared &sh)
{
    if (threadIdx.x == 0) {
        volatile PCtl *c = d.c;
        sh.n_un = c->n_un;
        sh.nk = c->nk;
        sh.wk = c->wk;
        sh.stop = c->stop;
        sh.na = c->na;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kPT) k_part_grow(PDev d)
{
    __shared__ PShared sh;
    PCtl *c = d.c;
    long long lo, hi;
    p_slice(d, lo, hi);
    unsigned long long bk = 0;  // barriers passed
    unsigned int round = 0;
    const unsigned long long idmask = (1ull << d.idbits) - 1ull;
    const int lane = threadIdx.x & 31;
    const long long gwarp = ((long long)blockIdx.x * kPT + threadIdx.x) >> 5;
    const long long nwarp = ((long long)gridDim.x * kPT) >> 5;
    bool ok = true;

    for (int k = 0; k < d.P - 1 && ok; ++k) {
        p_read_ctl(d, sh);
        if (sh.n_un == 0) break;
        // a new part: clear the shared weights; find the seed
        for (long long j = lo + threadIdx.x; j < hi; j += kPT) d.acc[j] = 0ull;
        if (d.t == 1) {
            unsigned int m = 0xFFFFFFFFu;
            for (long long j = lo + threadIdx.x; j < hi; j += kPT)
                if (__ldcg(d.lab + j) < 0) {
                    m = (unsigned int)j;
                    break;
                }
            m = __reduce_min_sync(0xFFFFFFFFu, m);
            if (lane == 0) sh.red32[threadIdx.x >> 5] = m;
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned int b = 0xFFFFFFFFu;
                for (int w = 0; w < kPW; ++w) b = min(b, sh.red32[w]);
                if (b != 0xFFFFFFFFu) atomicMin(&c->seed_id, b);
            }
        } else {
            unsigned int n = 0;
            for (long long j = lo + threadIdx.x; j < hi; j += kPT) n += __ldcg(d.lab + j) < 0;
            n = p_block_sum(n, sh.red32);
            if (threadIdx.x == 0) d.cnt[blockIdx.x] = n;
        }
        if (!(ok = p_sync(c, bk++, d.limit_ns))) break;
        if (d.t != 1) {
            // the r-th unassigned neuron in id order, r = word mod unassigned
            const unsigned long long r = (unsigned long long)d.rword[k] % (unsigned long long)sh.n_un;
            unsigned long long pre = 0;
            for (int x = threadIdx.x; x < (int)blockIdx.x; x += kPT) pre += __ldcg(d.cnt + x);
            pre = p_block_sum(pre, sh.redu);
            const unsigned long long mine = __ldcg(d.cnt + blockIdx.x);
            if (r >= pre && r < pre + mine) {
                // walk the slice in blocks of kPT ids, scanning the flags
                unsigned long long need = r - pre;
                for (long long j0 = lo; j0 < hi; j0 += kPT) {
                    const long long j = j0 + threadIdx.x;
                    const unsigned int f = (j < hi && __ldcg(d.lab + j) < 0) ? 1u : 0u;
                    unsigned int tot;
                    const unsigned int ex = p_block_excl(f, sh.red32, tot);
                    if (f && ex == need) c->seed_id = (unsigned int)j;
                    if (need < tot) break;
                    need -= tot;
                }
            }
            if (!(ok = p_sync(c, bk++, d.limit_ns))) break;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const unsigned int s = *(volatile unsigned int *)&c->seed_id;
            c->seed_id = 0xFFFFFFFFu;
            if (s >= (unsigned long long)d.M) {
                // no seed found: record it and end the growth
                atomicOr(&c->status, kPStFault);
                c->stop = 1;
                c->n_un = 0;
            } else {
            d.lab[s] = k;
            d.added[0] = s;
            const long long wk = d.W[s];
            const long long n_un = sh.n_un - 1;
            c->wk = wk;
            c->nk = 1;
            c->n_un = n_un;
            c->na = 1;
            c->stop = !(wk * (long long)d.P < d.Wtot) || n_un == 0;
            }
        }
        if (!(ok = p_sync(c, bk++, d.limit_ns))) break;

        for (;;) {
            p_read_ctl(d, sh);
            if (sh.stop) break;
            const int par = (int)(round & 1u);
            ++round;
            // scatter: (member, direction, chunk of kChunk synapses) per warp
            const long long tasks = (long long)sh.na * 2 * d.chunks;
            for (long long x = gwarp; x < tasks; x += nwarp) {
                const uint32_t a = __ldcg(d.added + x / (2 * d.chunks));
                const int rem = (int)(x % (2 * d.chunks));
                const bool in = rem >= d.chunks;
                const long long ch = rem - (in ? d.chunks : 0);
                const long long b0 = in ? d.in_ptr[a] : d.ptr[a];
                const long long b1 = in ? d.in_ptr[a + 1] : d.ptr[a + 1];
                const long long s0 = b0 + ch * kChunk;
                const long long s1 = min(b1, s0 + kChunk);
                const unsigned long long wa = d.W[a];
                for (long long e = s0 + lane; e < s1; e += 32) {
                    const uint32_t j = in ? d.in_src[e] : d.tgt[e];
                    atomicAdd(d.acc + j, wa);
                }
            }
            long long need = min((long long)d.B, sh.n_un);
            if (d.grow > 0) need = min(need, max(1ll, sh.nk / d.grow));
            if (!(ok = p_sync(c, bk++, d.limit_ns))) break;

            // select: the need-th largest key by radix passes over the digits
            uint32_t *gh = d.hist + (size_t)par * kMaxPass * kBins;
            unsigned long long prefix = 0, mask = 0;
            unsigned long long remk = (unsigned long long)need;
            for (int p = 0; p < d.npass && ok; ++p) {
                const int top = d.nbits - kDigit * p;
                const int shift = max(0, top - kDigit);
                const unsigned long long dmask = (1ull << (top - shift)) - 1ull;
                for (int x = threadIdx.x; x < kBins; x += kPT) sh.u.hist[x] = 0u;
                __syncthreads();
                for (long long j = lo + threadIdx.x; j < hi; j += kPT) {
                    unsigned long long kj;
                    if (p == 0) {
                        kj = 0ull;
                        if (__ldcg(d.lab + j) < 0)
                            kj = ((unsigned long long)d.W[j] * __ldcg(d.acc + j)) << d.idbits |
                                 (idmask - (unsigned long long)j);
                        d.key[j] = kj;
                    } else {
                        kj = d.key[j];
                    }
                    if (kj != 0ull && (kj & mask) == prefix) atomicAdd(&sh.u.hist[(kj >> shift) & dmask], 1u);
                }
                __syncthreads();
                for (int x = threadIdx.x; x < kBins; x += kPT)
                    if (sh.u.hist[x]) atomicAdd(gh + p * kBins + x, sh.u.hist[x]);
                if (!(ok = p_sync(c, bk++, d.limit_ns))) break;
                // the digit whose bin holds the remk-th largest key
                constexpr int kPer = kBins / kPT;
                uint32_t v[kPer];
                unsigned long long s = 0;
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    v[q] = __ldcg(gh + p * kBins + threadIdx.x * kPer + q);
                    s += v[q];
                }
                // suffix sums over threads: keys in bins above this thread's
                unsigned long long tot;
                const unsigned long long ex = p_block_excl(s, sh.redu, tot);
                unsigned long long above = tot - ex - s;
#pragma unroll
                for (int q = kPer - 1; q >= 0; --q) {
                    if (above < remk && above + v[q] >= remk) {
                        sh.digit = threadIdx.x * kPer + q;
                        sh.above = above;
                    }
                    above += v[q];
                }
                __syncthreads();
                remk -= sh.above;
                prefix |= (unsigned long long)sh.digit << shift;
                mask |= dmask << shift;
                __syncthreads();
            }
            if (!ok) break;
            // the keys are unique: the need members are the keys >= prefix
            {
                uint32_t *other = d.hist + (size_t)(par ^ 1) * kMaxPass * kBins;
                for (long long x = (long long)blockIdx.x * kPT + threadIdx.x; x < kMaxPass * kBins;
                     x += (long long)gridDim.x * kPT)
                    other[x] = 0u;
            }
            for (long long j = lo + threadIdx.x; j < hi; j += kPT) {
                const unsigned long long kj = d.key[j];
                if (kj != 0ull && kj >= prefix) {
                    const unsigned int pos = atomicAdd(&c->nsel, 1u);
                    if (pos < (unsigned int)kMaxBatch) d.sel[pos] = kj;  // (more is a fault, flagged below)
                }
            }
            if (!(ok = p_sync(c, bk++, d.limit_ns))) break;

            // join (block 0): sort the members by key, descending; they join
            // in that order while the part's weight is below sum(W)/P
            if (blockIdx.x == 0) {
                const unsigned int nsel = *(volatile unsigned int *)&c->nsel;
                if (nsel != (unsigned int)need) {
                    // not the round's size: record it and end the growth
                    if (threadIdx.x == 0) {
                        atomicOr(&c->status, kPStFault);
                        c->stop = 1;
                        c->n_un = 0;
                        c->nsel = 0u;
                    }
                    goto joined;
                }
                const int n = (int)nsel;
                int n2 = 1;
                while (n2 < n) n2 <<= 1;
                for (int x = threadIdx.x; x < n2; x += kPT) sh.u.s.key[x] = x < n ? __ldcg(d.sel + x) : 0ull;
                __syncthreads();
                for (int size = 2; size <= n2; size <<= 1)
                    for (int stride = size >> 1; stride > 0; stride >>= 1) {
                        for (int x = threadIdx.x; x < n2; x += kPT) {
                            const int y = x ^ stride;
                            if (y > x) {
                                const bool desc = (x & size) == 0;
                                const unsigned long long a = sh.u.s.key[x], b = sh.u.s.key[y];
                                if (desc ? a < b : a > b) {
                                    sh.u.s.key[x] = b;
                                    sh.u.s.key[y] = a;
                                }
                            }
                        }
                        __syncthreads();
                    }
                // inclusive prefix sums of the members' weights, kPer per thread
                constexpr int kPer = kMaxBatch / kPT;
                long long w[kPer];
                long long s = 0;
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    const int x = threadIdx.x * kPer + q;
                    w[q] = x < n ? (long long)d.W[idmask - (sh.u.s.key[x] & idmask)] : 0ll;
                    s += w[q];
                }
                long long tot;
                long long run = p_block_excl(s, sh.red64, tot);
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    run += w[q];
                    const int x = threadIdx.x * kPer + q;
                    if (x < n) sh.u.s.pre[x] = run;
                }
                __syncthreads();
                // members before the first one whose join fills the part
                unsigned int cont = 0;
                for (int x = threadIdx.x; x < n; x += kPT)
                    cont += ((sh.wk + sh.u.s.pre[x]) * (long long)d.P < d.Wtot) && (sh.n_un - x - 1 > 0);
                const int m = min(n, (int)p_block_sum(cont, sh.red32) + 1);
                for (int x = threadIdx.x; x < m; x += kPT) {
                    const uint32_t id = (uint32_t)(idmask - (sh.u.s.key[x] & idmask));
                    d.lab[id] = k;
                    d.added[x] = id;
                }
                if (threadIdx.x == 0) {
                    const long long wk = sh.wk + sh.u.s.pre[m - 1];
                    const long long n_un = sh.n_un - m;
                    c->wk = wk;
                    c->nk = sh.nk + m;
                    c->n_un = n_un;
                    c->na = m;
                    c->stop = !(wk * (long long)d.P < d.Wtot) || n_un == 0;
                    c->nsel = 0u;
                }
            }
        joined:
            if (!(ok = p_sync(c, bk++, d.limit_ns))) break;
        }
    }
    if (!ok) return;
    // the last part takes the rest
    for (long long j = lo + threadIdx.x; j < hi; j += kPT)
        if (__ldcg(d.lab + j) < 0) d.lab[j] = d.P - 1;
    if (!p_sync(c, bk++, d.limit_ns)) return;
    // objective (sum over cut synapses of W_i W_j) and part weights; one
    // warp per source neuron
    unsigned long long cut = 0;
    for (long long i = gwarp; i < d.M; i += nwarp) {
        const int li = __ldcg(d.lab + i);
        const unsigned long long wi = d.W[i];
        if (lane == 0) atomicAdd(d.wpart + li, wi);
        for (long long e = d.ptr[i] + lane; e < d.ptr[i + 1]; e += 32) {
            const uint32_t j = d.tgt[e];
            if (__ldcg(d.lab + j) != li) cut += wi * d.W[j];
        }
    }
    cut = p_block_sum(cut, sh.redu);
    if (threadIdx.x == 0 && cut) atomicAdd(&c->obj, cut);
}

// ------------------------------------------------------------------ host
struct PLayout {
    size_t ptr, in_ptr, tgt, in_src, W, acc, key, lab, best, fill, hist, sel, added, cnt, rword, wpart,
        ctl, total;
};

constexpr int kMaxGrid = 4096;

PLayout p_layout(long long M, long long E, int P)
{
    PLayout L;
    size_t o = 0;
    auto put = [&](size_t &f, size_t bytes) {
        f = o;
        o += (bytes + 255) & ~(size_t)255;
    };
    put(L.ctl, sizeof(PCtl));
    put(L.ptr, 8 * (size_t)(M + 1));
    put(L.in_ptr, 8 * (size_t)(M + 1));
    put(L.tgt, 4 * (size_t)(E > 0 ? E : 1));
    put(L.in_src, 4 * (size_t)(E > 0 ? E : 1));
    put(L.W, 4 * (size_t)M);
    put(L.acc, 8 * (size_t)M);
    put(L.key, 8 * (size_t)M);
    put(L.lab, 4 * (size_t)M);
    put(L.best, 4 * (size_t)M);
    put(L.fill, 4 * (size_t)M);
    put(L.hist, 4 * (size_t)2 * kMaxPass * kBins);
    put(L.sel, 8 * (size_t)kMaxBatch);
    put(L.added, 4 * (size_t)kMaxBatch);
    put(L.cnt, 4 * (size_t)kMaxGrid);
    put(L.rword, 4 * (size_t)P);
    put(L.wpart, 8 * (size_t)P * 2);
    L.total = o;
    return L;
}

int bit_length(unsigned long long x)
{
    int n = 0;
    while (x) {
        ++n;
        x >>= 1;
    }
    return n;
}

#define PCK(x)                                    \
    do {                                          \
        cudaError_t e_ = (x);                     \
        if (e_ != cudaSuccess) return SNN_E_CUDA; \
    } while (0)

}  // namespace

extern "C" void snn_partition_device_params_default(snn_partition_device_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->iters = 4;
    p->batch = 2048;
    p->grow = 2;
    p->seed = 7;
}

extern "C" int snn_partition_device_workspace_bytes(const snn_network *net, int32_t P, size_t *bytes)
{
    if (!net || !net->syn_ptr || net->n_neurons <= 0 || !bytes || P < 1 || P > net->n_neurons) return SNN_E_ARG;
    *bytes = p_layout(net->n_neurons, net->syn_ptr[net->n_neurons], P).total;
    return SNN_OK;
}

extern "C" int snn_partition_device(const snn_network *net, int32_t P, const snn_partition_device_params *prm,
                                    void *workspace, size_t workspace_bytes, void *stream, int32_t *part_of,
                                    snn_partition_stats *stats)
{
    if (!net || !net->syn_ptr || !prm || !part_of || !workspace) return SNN_E_ARG;
    const long long M = net->n_neurons;
    if (M <= 0 || P < 1 || P > M) return SNN_E_ARG;
    if (M >= (1ll << snn::kTgtBits)) return SNN_E_RANGE;
    if (prm->iters < 1 || prm->batch < 1 || prm->batch > kMaxBatch || prm->grow < 0) return SNN_E_ARG;
    const long long E = net->syn_ptr[M];
    if (net->syn_ptr[0] != 0 || E < 0 || (E > 0 && !net->syn_tgt)) return SNN_E_ARG;
    const PLayout L = p_layout(M, E, P);
    if (workspace_bytes < L.total || ((uintptr_t)workspace & 255)) return SNN_E_NOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)workspace;

    int dev = 0, sms = 0, coop = 0, occ = 0;
    PCK(cudaGetDevice(&dev));
    PCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PCK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return SNN_E_NODEV;
    PCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_part_grow, kPT, 0));
    if (occ < 1) return SNN_E_NODEV;
    // two blocks per SM: the rounds' barriers cost more with more blocks,
    // the scatter of a large round wants more than one per SM
    const int grid = std::min(kMaxGrid, sms * std::min(occ, 2));

    PDev d;
    std::memset(&d, 0, sizeof(d));
    d.ptr = (const long long *)(w + L.ptr);
    d.tgt = (const uint32_t *)(w + L.tgt);
    d.in_ptr = (long long *)(w + L.in_ptr);
    d.in_src = (uint32_t *)(w + L.in_src);
    d.W = (uint32_t *)(w + L.W);
    d.acc = (unsigned long long *)(w + L.acc);
    d.key = (unsigned long long *)(w + L.key);
    d.lab = (int32_t *)(w + L.lab);
    d.fill = (uint32_t *)(w + L.fill);
    d.hist = (uint32_t *)(w + L.hist);
    d.sel = (unsigned long long *)(w + L.sel);
    d.added = (uint32_t *)(w + L.added);
    d.cnt = (uint32_t *)(w + L.cnt);
    d.rword = (const uint32_t *)(w + L.rword);
    d.wpart = (unsigned long long *)(w + L.wpart);
    d.c = (PCtl *)(w + L.ctl);
    d.M = M;
    d.E = E;
    d.Wtot = E;
    d.P = P;
    d.B = prm->batch;
    d.grow = prm->grow;
    d.limit_ns = 2000000000ull;

    // tables to the device; in-lists and the key width on the device
    PCK(cudaMemcpyAsync((void *)d.ptr, net->syn_ptr, 8 * (size_t)(M + 1), cudaMemcpyHostToDevice, st));
    if (E > 0) PCK(cudaMemcpyAsync((void *)d.tgt, net->syn_tgt, 4 * (size_t)E, cudaMemcpyHostToDevice, st));
    PCK(cudaMemsetAsync(d.c, 0, sizeof(PCtl), st));
    PCK(cudaMemsetAsync(d.fill, 0, 4 * (size_t)M, st));
    const int g2 = sms * 8;
    k_part_degrees<<<g2, 256, 0, st>>>(d);
    k_part_scan<<<1, 1024, 0, st>>>(d);
    k_part_in_lists<<<g2, 256, 0, st>>>(d);
    k_part_bounds<<<g2, 256, 0, st>>>(d);
    PCK(cudaGetLastError());
    PCtl ctl;
    PCK(cudaMemcpyAsync(&ctl, d.c, sizeof(PCtl), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    if (ctl.status & kPStRange) return SNN_E_ARG;
    d.idbits = std::max(1, bit_length((unsigned long long)M));
    d.nbits = bit_length(ctl.gain_max) + d.idbits;
    if (d.nbits > 64) return SNN_E_RANGE;
    d.npass = (d.nbits + kDigit - 1) / kDigit;
    d.chunks = (int)std::max(1ull, (ctl.deg_max + kChunk - 1) / kChunk);

    std::vector<uint32_t> rw((size_t)P);
    unsigned long long best = 0;
    for (int t = 1; t <= prm->iters; ++t) {
        for (int k = 0; k < P; ++k) rw[k] = snn::philox_word0(prm->seed, (uint32_t)t, (uint32_t)k, 0xA1u);
        PCK(cudaMemcpyAsync((void *)d.rword, rw.data(), 4 * (size_t)P, cudaMemcpyHostToDevice, st));
        std::memset(&ctl, 0, sizeof(ctl));
        ctl.n_un = M;
        ctl.seed_id = 0xFFFFFFFFu;
        PCK(cudaMemcpyAsync(d.c, &ctl, sizeof(PCtl), cudaMemcpyHostToDevice, st));
        PCK(cudaMemsetAsync(d.lab, 0xFF, 4 * (size_t)M, st));
        PCK(cudaMemsetAsync(d.hist, 0, 4 * (size_t)2 * kMaxPass * kBins, st));
        PCK(cudaMemsetAsync(d.wpart, 0, 8 * (size_t)P, st));
        d.t = t;
        void *args[] = {&d};
        PCK(cudaLaunchCooperativeKernel((const void *)k_part_grow, dim3(grid), dim3(kPT), args, 0, st));
        PCK(cudaMemcpyAsync(&ctl, d.c, sizeof(PCtl), cudaMemcpyDeviceToHost, st));
        PCK(cudaStreamSynchronize(st));
        if (ctl.status & kPStTimeout) return SNN_E_TIMEOUT;
        if (ctl.status & kPStFault) return SNN_E_STATE;
        if (t == 1 || ctl.obj < best) {
            best = ctl.obj;
            PCK(cudaMemcpyAsync(w + L.best, d.lab, 4 * (size_t)M, cudaMemcpyDeviceToDevice, st));
            PCK(cudaMemcpyAsync(d.wpart + P, d.wpart, 8 * (size_t)P, cudaMemcpyDeviceToDevice, st));
        }
    }
    std::vector<unsigned long long> wp((size_t)P);
    PCK(cudaMemcpyAsync(part_of, w + L.best, 4 * (size_t)M, cudaMemcpyDeviceToHost, st));
    PCK(cudaMemcpyAsync(wp.data(), d.wpart + P, 8 * (size_t)P, cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    if (stats) {
        stats->objective = (int64_t)best;
        stats->min_weight = (int64_t)*std::min_element(wp.begin(), wp.end());
        stats->max_weight = (int64_t)*std::max_element(wp.begin(), wp.end());
    }
    return SNN_OK;
}
