// Routing tables built on the GPU (sm_103a): the O(E) scans and the
// per-neuron synapse sort of the two-level routing build (Sec. IV.B), the
// table-building half of the parallel design the paper leaves as future
// work (Sec. VII).  The host keeps what is O(M) or O(P^2): validation,
// Algorithm 2 grouping, the internal orders and the exchange-pair
// numbering (the helpers snn_routing_build uses), so both builders give the
// same tables byte for byte.
//   pass A  (warp per source neuron, label order): target and delay checks,
//           the largest delay, inter-partition synapse counts PG[p][q];
//   pass B  (warp per internal neuron): distinct destination partitions and
//           VNs per neuron (shared-memory bitmaps), exchange-pair worst cases;
//   pass C  (block per internal neuron, in chunks of neurons): the neuron's
//           synapses sorted by (destination partition, delay, target,
//           weight) in shared memory (bitonic), written to the internal CSR,
//           with one level-2 entry per destination-partition run (its
//           delay-1 count packed into the offset) and one level-1 entry per
//           destination-VN run; each chunk is copied back to the host tables.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <system_error>
#include <thread>
#include <vector>

#include "snn_internal.h"

using namespace snn;

namespace {

constexpr int kRT = 256;
constexpr int kRW = kRT / 32;
constexpr int kCapSmall = 1024;   // synapses per neuron of the shared-memory sort, small blocks
constexpr int kCapBig = 16384;    // largest out-degree of the device builder
constexpr int kSegCapBig = 4096;  // segments of one neuron (<= P <= 4096)

constexpr uint32_t kRBadId = 1u, kRBadDelay = 2u, kRCap = 4u, kRCount = 8u;

struct RDev {
    const long long *sp;
    const uint32_t *tgt;
    const int16_t *w;
    const uint8_t *d;
    const int32_t *part_of;   // [M] labels
    const uint32_t *perm_fwd; // [M] global -> internal
    const uint32_t *perm_inv; // [M] internal -> global
    const uint16_t *ipo;      // [P] internal partition of each label
    long long M, E;
    int P, n_vn, s;
    unsigned int *flags;      // [0] status bits, [1] largest delay
    unsigned long long *PG;   // [P*P] label order
    uint32_t *nseg, *nvn;     // [M] internal order
    uint32_t *bc, *ic;        // [P*n_vn], [P*P] internal order (worst cases, then pair ids)
    const long long *csr, *l2p;  // [M+1]
    const uint32_t *l1p;         // [M+1]
    long long k0, k1, syn0, l20, l10;
    uint32_t *o_td;
    int16_t *o_w;
    L2Entry *o_l2;
    uint32_t *o_l2pair;
    uint16_t *o_l1vn;
    uint32_t *o_l1l2, *o_l1pair;
};

// ------------------------------------------------------------------ pass A
__global__ void __launch_bounds__(kRT) k_route_scan(RDev d)
{
    const int lane = threadIdx.x & 31;
    const long long w0 = ((long long)blockIdx.x * kRT + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * kRT) >> 5;
    unsigned int dmax = 1, bad = 0;
    for (long long i = w0; i < d.M; i += nw) {
        const int p = d.part_of[i];
        const long long b = d.sp[i], e1 = d.sp[i + 1];
        for (long long base = b; base < e1; base += 32) {
            const long long e = base + lane;
            int key = -1;
            if (e < e1) {
                const uint32_t t = d.tgt[e];
                const unsigned int dl = d.d[e];
                if (t >= (unsigned long long)d.M) bad |= kRBadId;
                else if (dl < 1u || dl > (unsigned int)kMaxDelay) bad |= kRBadDelay;
                else {
                    dmax = max(dmax, dl);
                    const int q = d.part_of[t];
                    if (q != p) key = q;
                }
            }
            // one reduction per distinct destination partition of the 32 synapses
            const unsigned int same = __match_any_sync(0xFFFFFFFFu, key);
            if (key >= 0 && lane == __ffs(same) - 1)
                atomicAdd(d.PG + (size_t)p * d.P + key, (unsigned long long)__popc(same));
        }
    }
    dmax = __reduce_max_sync(0xFFFFFFFFu, dmax);
    bad = __reduce_or_sync(0xFFFFFFFFu, bad);
    if (lane == 0) {
        atomicMax(d.flags + 1, dmax);
        if (bad) atomicOr(d.flags, bad);
    }
}

// ------------------------------------------------------------------ pass B
__global__ void __launch_bounds__(kRT) k_route_count(RDev d)
{
    extern __shared__ uint32_t bm[];  // per warp: (P + 31) / 32 + (n_vn + 31) / 32 words
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int wq = (d.P + 31) >> 5, wg = (d.n_vn + 31) >> 5;
    uint32_t *bq = bm + (size_t)wid * (wq + wg), *bg = bq + wq;
    for (int x = lane; x < wq + wg; x += 32) bq[x] = 0u;
    __syncwarp();
    const long long w0 = ((long long)blockIdx.x * kRT + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * kRT) >> 5;
    for (long long kk = w0; kk < d.M; kk += nw) {
        const uint32_t i = d.perm_inv[kk];
        const int ps = d.ipo[d.part_of[i]];
        unsigned int ns = 0, nv = 0;
        for (long long e = d.sp[i] + lane; e < d.sp[i + 1]; e += 32) {
            const int q = d.ipo[d.part_of[d.tgt[e]]];
            const uint32_t bit = 1u << (q & 31);
            if (!(atomicOr(bq + (q >> 5), bit) & bit)) {
                ++ns;
                atomicAdd(d.ic + (size_t)ps * d.P + q, 1u);
                const int g = q / d.s;
                const uint32_t gb = 1u << (g & 31);
                if (!(atomicOr(bg + (g >> 5), gb) & gb)) {
                    ++nv;
                    atomicAdd(d.bc + (size_t)ps * d.n_vn + g, 1u);
                }
            }
        }
        ns = __reduce_add_sync(0xFFFFFFFFu, ns);
        nv = __reduce_add_sync(0xFFFFFFFFu, nv);
        if (lane == 0) {
            d.nseg[kk] = ns;
            d.nvn[kk] = nv;
        }
        __syncwarp();
        for (int x = lane; x < wq + wg; x += 32) bq[x] = 0u;
        __syncwarp();
    }
}

// ------------------------------------------------------------------ pass C
// Exclusive scan over the block of one count per thread; returns the
// thread's base, total in *tot.
__device__ __forceinline__ int r_scan(int v, int *sh, int &tot)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    int base = 0, t = 0;
#pragma unroll
    for (int w = 0; w < kRW; ++w) {
        if (w < wid) base += sh[w];
        t += sh[w];
    }
    tot = t;
    return base + x - v;
}

__device__ __forceinline__ int r_q(unsigned long long k) { return (int)(k >> 48); }
__device__ __forceinline__ unsigned int r_delay0(unsigned long long k) { return (unsigned int)(k >> (16 + kTgtBits)) & 15u; }

// One block per internal neuron of [k0, k1) whose out-degree is in (lo_deg,
// CAP] (neurons without synapses have no entries); keys in shared memory
// (CAP of them), segment arrays of SEGCAP.
template <int CAP, int SEGCAP>
__device__ __forceinline__ void route_emit(const RDev &d, int lo_deg, unsigned long long *key, int *seg_start,
                                           int *seg_d1)
{
    __shared__ int sh[kRW];
    const int tid = threadIdx.x;
    for (long long kk = d.k0 + blockIdx.x; kk < d.k1; kk += gridDim.x) {
        const uint32_t i = d.perm_inv[kk];
        const long long b = d.sp[i];
        const int n = (int)(d.sp[i + 1] - b);
        if (n <= lo_deg || n > CAP) continue;  // (the host rejects out-degrees above kCapBig)
        const int ps = d.ipo[d.part_of[i]], hs = ps / d.s;
        int n2 = 1;
        while (n2 < n) n2 <<= 1;
        for (int r = tid; r < n2; r += kRT) {
            unsigned long long k = ~0ull;
            if (r < n) {
                const uint32_t t = d.tgt[b + r];
                const unsigned long long q = d.ipo[d.part_of[t]];
                const unsigned long long td = d.perm_fwd[t] | ((uint32_t)(d.d[b + r] - 1) << kTgtBits);
                k = q << 48 | td << 16 | (uint16_t)d.w[b + r];
            }
            key[r] = k;
        }
        __syncthreads();
        for (int size = 2; size <= n2; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int x = tid; x < n2; x += kRT) {
                    const int y = x ^ stride;
                    if (y > x) {
                        const bool asc = (x & size) == 0;
                        const unsigned long long a = key[x], c = key[y];
                        if (asc ? a > c : a < c) {
                            key[x] = c;
                            key[y] = a;
                        }
                    }
                }
                __syncthreads();
            }
        // the internal CSR
        const long long ob = d.csr[kk] - d.syn0;
        for (int r = tid; r < n; r += kRT) {
            const unsigned long long k = key[r];
            d.o_td[ob + r] = (uint32_t)(k >> 16);
            d.o_w[ob + r] = (int16_t)(uint16_t)k;
        }
        // destination-partition runs: thread t takes the elements [t*per, ...)
        const int per = (n + kRT - 1) / kRT;
        const int r0 = min(n, tid * per), r1 = min(n, r0 + per);
        int cnt = 0;
        for (int r = r0; r < r1; ++r) cnt += (r == 0 || r_q(key[r]) != r_q(key[r - 1]));
        int nseg;
        int si = r_scan(cnt, sh, nseg) - 1;
        if (nseg > SEGCAP) {
            if (tid == 0) atomicOr(d.flags, kRCap);
            __syncthreads();
            continue;
        }
        for (int r = r0; r < r1; ++r)
            if (r == 0 || r_q(key[r]) != r_q(key[r - 1])) {
                ++si;
                seg_start[si] = r;
                seg_d1[si] = -1;
            }
        __syncthreads();
        // first synapse of delay > 1 in each run (runs are sorted by delay)
        si = r_scan(cnt, sh, nseg) - 1;
        for (int r = r0; r < r1; ++r) {
            const bool start = r == 0 || r_q(key[r]) != r_q(key[r - 1]);
            if (start) ++si;
            if (r_delay0(key[r]) != 0u && (start || r_delay0(key[r - 1]) == 0u)) seg_d1[si] = r;
        }
        __syncthreads();
        if (tid == 0 && (uint32_t)nseg != d.nseg[kk]) atomicOr(d.flags, kRCount);
        // level-2 entries
        const long long f0 = d.l2p[kk];
        for (int x = tid; x < nseg; x += kRT) {
            const int st = seg_start[x], en = x + 1 < nseg ? seg_start[x + 1] : n;
            const int q = r_q(key[st]);
            const unsigned long long n1 = seg_d1[x] >= 0 ? (unsigned long long)(seg_d1[x] - st)
                                                          : (unsigned long long)(en - st);
            const int g = q / d.s;
            uint8_t cls;
            if (g == hs) cls = q == ps ? kClsLocal : kClsPeer;
            else cls = q == g * d.s + vn_rank(hs, g, d.s) ? kClsRelayLocal : kClsRelayRemote;
            L2Entry e;
            e.off = (unsigned long long)(d.csr[kk] + st) | (n1 << kOffBits);
            e.len = (uint32_t)(en - st);
            e.q = (uint16_t)q;
            e.cls = cls;
            e.pad = 0;
            d.o_l2[f0 + x - d.l20] = e;
            d.o_l2pair[f0 + x - d.l20] = d.ic[(size_t)ps * d.P + q];
        }
        // destination-VN runs over the partition runs
        const int pv = (nseg + kRT - 1) / kRT;
        const int v0 = min(nseg, tid * pv), v1 = min(nseg, v0 + pv);
        int cv = 0;
        for (int x = v0; x < v1; ++x)
            cv += x == 0 || r_q(key[seg_start[x]]) / d.s != r_q(key[seg_start[x - 1]]) / d.s;
        int nv;
        int vi = r_scan(cv, sh, nv) - 1;
        const long long e0 = d.l1p[kk];
        for (int x = v0; x < v1; ++x) {
            const int g = r_q(key[seg_start[x]]) / d.s;
            if (x == 0 || g != r_q(key[seg_start[x - 1]]) / d.s) {
                ++vi;
                d.o_l1vn[e0 + vi - d.l10] = (uint16_t)g;
                d.o_l1l2[e0 + vi - d.l10] = (uint32_t)(f0 + x);
                d.o_l1pair[e0 + vi - d.l10] = d.bc[(size_t)ps * d.n_vn + g];
            }
        }
        if (tid == 0 && (uint32_t)nv != d.nvn[kk]) atomicOr(d.flags, kRCount);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kRT) k_route_emit_small(RDev d)
{
    __shared__ unsigned long long key[kCapSmall];
    __shared__ int seg_start[kCapSmall], seg_d1[kCapSmall];
    route_emit<kCapSmall, kCapSmall>(d, 0, key, seg_start, seg_d1);
}

__global__ void __launch_bounds__(kRT) k_route_emit_big(RDev d)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    unsigned long long *key = reinterpret_cast<unsigned long long *>(dyn);
    int *seg_start = reinterpret_cast<int *>(dyn + 8 * (size_t)kCapBig);
    int *seg_d1 = seg_start + kSegCapBig;
    route_emit<kCapBig, kSegCapBig>(d, kCapSmall, key, seg_start, seg_d1);
}

constexpr size_t kBigSmem = 8 * (size_t)kCapBig + 2 * 4 * (size_t)kSegCapBig;

// ------------------------------------------------------------------ host
struct RLayout {
    size_t sp, tgt, w, d, part_of, perm_fwd, perm_inv, ipo, flags, PG, nseg, nvn, bc, ic, csr, l2p, l1p, o_td,
        o_w, o_l2, o_l2pair, o_l1vn, o_l1l2, o_l1pair, total;
    long long cap_syn, cap_ent;
};

long long max_degree(const snn_network *net)
{
    long long m = 0;
    for (long long i = 0; i < net->n_neurons; ++i) m = std::max<long long>(m, net->syn_ptr[i + 1] - net->syn_ptr[i]);
    return m;
}

RLayout r_layout(long long M, long long E, int P, int n_vn, long long maxdeg)
{
    RLayout L;
    size_t o = 0;
    auto put = [&](size_t &f, size_t bytes) {
        f = o;
        o += (bytes + 255) & ~(size_t)255;
    };
    // a chunk holds at least the largest neuron
    L.cap_syn = std::max<long long>(std::min<long long>(E, 1ll << 26), std::max<long long>(maxdeg, 1));
    L.cap_ent = std::max<long long>(std::min<long long>(E, 1ll << 24), std::max<long long>(maxdeg, 1));
    const size_t e1 = (size_t)std::max<long long>(E, 1);
    put(L.flags, 64);
    put(L.sp, 8 * (size_t)(M + 1));
    put(L.tgt, 4 * e1);
    put(L.w, 2 * e1);
    put(L.d, e1);
    put(L.part_of, 4 * (size_t)M);
    put(L.perm_fwd, 4 * (size_t)M);
    put(L.perm_inv, 4 * (size_t)M);
    put(L.ipo, 2 * (size_t)P);
    put(L.PG, 8 * (size_t)P * P);
    put(L.nseg, 4 * (size_t)M);
    put(L.nvn, 4 * (size_t)M);
    put(L.bc, 4 * (size_t)P * n_vn);
    put(L.ic, 4 * (size_t)P * P);
    put(L.csr, 8 * (size_t)(M + 1));
    put(L.l2p, 8 * (size_t)(M + 1));
    put(L.l1p, 4 * (size_t)(M + 1));
    put(L.o_td, 4 * (size_t)L.cap_syn);
    put(L.o_w, 2 * (size_t)L.cap_syn);
    put(L.o_l2, sizeof(L2Entry) * (size_t)L.cap_ent);
    put(L.o_l2pair, 4 * (size_t)L.cap_ent);
    put(L.o_l1vn, 2 * (size_t)L.cap_ent);
    put(L.o_l1l2, 4 * (size_t)L.cap_ent);
    put(L.o_l1pair, 4 * (size_t)L.cap_ent);
    L.total = o;
    return L;
}

// First touch of fresh pageable host memory on all cores: the tables'
// pages are faulted in by CPU threads instead of one by one under the
// device-to-host copies.
void touch_pages(void *p, size_t bytes)
{
    constexpr size_t kPage = 4096;
    const int64_t n = (int64_t)((bytes + kPage - 1) / kPage);
    parallel_for(n, 0, [p](int64_t lo, int64_t hi, int) {
        volatile char *c = (volatile char *)p;
        for (int64_t x = lo; x < hi; ++x) c[(size_t)x * kPage] = 0;
    });
}

// The two largest tables, allocated and faulted in on a host thread while
// the first passes run on the device (joined before any return: the thread
// touches only its own arrays).
struct Prefault {
    HostArray<uint32_t> td;
    HostArray<int16_t> w;
    std::thread th;
    bool bad = false;
    void start(int64_t E)
    {
        th = std::thread([this, E] {
            try {
                td.alloc(E);
                w.alloc(E);
                touch_pages(td.data(), 4 * (size_t)E);
                touch_pages(w.data(), 2 * (size_t)E);
            } catch (...) {
                bad = true;
            }
        });
    }
    void join()
    {
        if (th.joinable()) th.join();
    }
    ~Prefault() { join(); }
};

#define RCK(x)                                          \
    do {                                                \
        if ((x) != cudaSuccess) {                       \
            delete rt;                                  \
            return SNN_E_CUDA;                          \
        }                                               \
    } while (0)

}  // namespace

extern "C" int snn_routing_build_device_workspace_bytes(const snn_network *net, int32_t P, int32_t n_vn,
                                                        size_t *bytes)
{
    if (!net || !net->syn_ptr || net->n_neurons <= 0 || !bytes || P < 1 || n_vn < 1) return SNN_E_ARG;
    const long long M = net->n_neurons;
    *bytes = r_layout(M, net->syn_ptr[M], P, n_vn, max_degree(net)).total;
    return SNN_OK;
}

extern "C" int snn_routing_build_device(const snn_network *net, const int32_t *part_of, int32_t P, int32_t n_vn,
                                        const snn_routing_params *prm, void *workspace, size_t workspace_bytes,
                                        void *stream, snn_routing **out)
{
    if (!out) return SNN_E_ARG;
    *out = nullptr;
    if (!net || !net->syn_ptr || !net->v0 || !part_of || !prm || !workspace) return SNN_E_ARG;
    const long long M = net->n_neurons;
    if (M <= 0 || net->syn_ptr[0] != 0) return SNN_E_ARG;
    const long long E = net->syn_ptr[M];
    if (E > 0 && (!net->syn_tgt || !net->syn_w || !net->syn_d)) return SNN_E_ARG;
    if (P < 1 || n_vn < 1 || P % n_vn || P > M) return SNN_E_ARG;
    if (P > 4096) return SNN_E_RANGE;
    if (prm->grouping != SNN_GROUP_CONTIGUOUS && prm->grouping != SNN_GROUP_GREEDY) return SNN_E_ARG;
    if (prm->relay < SNN_RELAY_PER_VN || prm->relay > SNN_RELAY_BALANCED) return SNN_E_ARG;
    if (prm->grouping == SNN_GROUP_GREEDY && prm->iters < 1) return SNN_E_ARG;
    if (M >= (1ll << kTgtBits)) return SNN_E_RANGE;
    if (E >= (1ll << 40)) return SNN_E_RANGE;
    long long maxdeg = 0;
    for (long long i = 0; i < M; ++i) {
        const long long dg = net->syn_ptr[i + 1] - net->syn_ptr[i];
        if (dg < 0) return SNN_E_ARG;
        maxdeg = std::max(maxdeg, dg);
    }
    if (maxdeg >= (1ll << kLenBits)) return SNN_E_RANGE;
    if (maxdeg > kCapBig) return SNN_E_RANGE;
    std::vector<int64_t> sizes((size_t)P, 0);
    for (long long i = 0; i < M; ++i) {
        if (part_of[i] < 0 || part_of[i] >= P) return SNN_E_ARG;
        sizes[part_of[i]]++;
    }
    for (int32_t p = 0; p < P; ++p)
        if (sizes[p] == 0) return SNN_E_ARG;
    const RLayout L = r_layout(M, E, P, n_vn, maxdeg);
    if (workspace_bytes < L.total || ((uintptr_t)workspace & 255)) return SNN_E_NOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SNN_E_CUDA;

    snn_routing *rt = nullptr;
    try {
        rt = new snn_routing();
    } catch (const std::bad_alloc &) {
        return SNN_E_NOMEM;
    }
    rt->M = M;
    rt->E = E;
    rt->P = P;
    rt->n_vn = n_vn;
    rt->vn_size = P / n_vn;
    const int s = rt->vn_size;

    Prefault pf;
    try {
        pf.start(E);
    } catch (const std::system_error &) {
        delete rt;
        return SNN_E_NOMEM;
    }
    RDev d;
    std::memset(&d, 0, sizeof(d));
    d.sp = (const long long *)(ws + L.sp);
    d.tgt = (const uint32_t *)(ws + L.tgt);
    d.w = (const int16_t *)(ws + L.w);
    d.d = (const uint8_t *)(ws + L.d);
    d.part_of = (const int32_t *)(ws + L.part_of);
    d.perm_fwd = (const uint32_t *)(ws + L.perm_fwd);
    d.perm_inv = (const uint32_t *)(ws + L.perm_inv);
    d.ipo = (const uint16_t *)(ws + L.ipo);
    d.flags = (unsigned int *)(ws + L.flags);
    d.PG = (unsigned long long *)(ws + L.PG);
    d.nseg = (uint32_t *)(ws + L.nseg);
    d.nvn = (uint32_t *)(ws + L.nvn);
    d.bc = (uint32_t *)(ws + L.bc);
    d.ic = (uint32_t *)(ws + L.ic);
    d.csr = (const long long *)(ws + L.csr);
    d.l2p = (const long long *)(ws + L.l2p);
    d.l1p = (const uint32_t *)(ws + L.l1p);
    d.o_td = (uint32_t *)(ws + L.o_td);
    d.o_w = (int16_t *)(ws + L.o_w);
    d.o_l2 = (L2Entry *)(ws + L.o_l2);
    d.o_l2pair = (uint32_t *)(ws + L.o_l2pair);
    d.o_l1vn = (uint16_t *)(ws + L.o_l1vn);
    d.o_l1l2 = (uint32_t *)(ws + L.o_l1l2);
    d.o_l1pair = (uint32_t *)(ws + L.o_l1pair);
    d.M = M;
    d.E = E;
    d.P = P;
    d.n_vn = n_vn;
    d.s = s;
    const int grid = sms * 8;

    try {
        // ---- pass A: checks, largest delay, inter-partition synapse counts
        RCK(cudaMemcpyAsync((void *)d.sp, net->syn_ptr, 8 * (size_t)(M + 1), cudaMemcpyHostToDevice, st));
        if (E > 0) {
            RCK(cudaMemcpyAsync((void *)d.tgt, net->syn_tgt, 4 * (size_t)E, cudaMemcpyHostToDevice, st));
            RCK(cudaMemcpyAsync((void *)d.w, net->syn_w, 2 * (size_t)E, cudaMemcpyHostToDevice, st));
            RCK(cudaMemcpyAsync((void *)d.d, net->syn_d, (size_t)E, cudaMemcpyHostToDevice, st));
        }
        RCK(cudaMemcpyAsync((void *)d.part_of, part_of, 4 * (size_t)M, cudaMemcpyHostToDevice, st));
        RCK(cudaMemsetAsync(d.flags, 0, 64, st));
        RCK(cudaMemsetAsync(d.PG, 0, 8 * (size_t)P * P, st));
        k_route_scan<<<grid, kRT, 0, st>>>(d);
        RCK(cudaGetLastError());
        std::vector<unsigned long long> PGu((size_t)P * P);
        unsigned int fl[2];
        RCK(cudaMemcpyAsync(PGu.data(), d.PG, 8 * (size_t)P * P, cudaMemcpyDeviceToHost, st));
        RCK(cudaMemcpyAsync(fl, d.flags, sizeof(fl), cudaMemcpyDeviceToHost, st));
        RCK(cudaStreamSynchronize(st));
        if (fl[0] & kRBadId) { delete rt; return SNN_E_ARG; }
        if (fl[0] & kRBadDelay) { delete rt; return SNN_E_RANGE; }
        rt->max_delay = E > 0 ? (int32_t)fl[1] : 1;

        // ---- host: grouping, internal orders
        std::vector<int64_t> PG(PGu.begin(), PGu.end()), WG((size_t)P, 0);
        for (long long i = 0; i < M; ++i) WG[part_of[i]] += net->syn_ptr[i + 1] - net->syn_ptr[i];
        route_groups(rt, prm, PG, WG);
        route_order(rt, net, part_of, sizes);
        std::vector<uint16_t> ipo((size_t)P);
        for (int32_t p = 0; p < P; ++p) ipo[p] = (uint16_t)rt->ip_of_part[p];

        // ---- pass B: per-neuron segment and VN counts, pair worst cases
        RCK(cudaMemcpyAsync((void *)d.perm_fwd, rt->perm_fwd.data(), 4 * (size_t)M, cudaMemcpyHostToDevice, st));
        RCK(cudaMemcpyAsync((void *)d.perm_inv, rt->perm_inv.data(), 4 * (size_t)M, cudaMemcpyHostToDevice, st));
        RCK(cudaMemcpyAsync((void *)d.ipo, ipo.data(), 2 * (size_t)P, cudaMemcpyHostToDevice, st));
        RCK(cudaMemsetAsync(d.bc, 0, 4 * (size_t)P * n_vn, st));
        RCK(cudaMemsetAsync(d.ic, 0, 4 * (size_t)P * P, st));
        const size_t bm = (size_t)kRW * (((P + 31) / 32) + ((n_vn + 31) / 32)) * 4;
        k_route_count<<<grid, kRT, bm, st>>>(d);
        RCK(cudaGetLastError());
        std::vector<uint32_t> nseg((size_t)M), nvn((size_t)M), bc((size_t)P * n_vn), ic((size_t)P * P);
        RCK(cudaMemcpyAsync(nseg.data(), d.nseg, 4 * (size_t)M, cudaMemcpyDeviceToHost, st));
        RCK(cudaMemcpyAsync(nvn.data(), d.nvn, 4 * (size_t)M, cudaMemcpyDeviceToHost, st));
        RCK(cudaMemcpyAsync(bc.data(), d.bc, 4 * bc.size(), cudaMemcpyDeviceToHost, st));
        RCK(cudaMemcpyAsync(ic.data(), d.ic, 4 * ic.size(), cudaMemcpyDeviceToHost, st));
        RCK(cudaStreamSynchronize(st));

        // ---- host: offsets, capacities, connections, pair numbering
        rt->csr.assign((size_t)M + 1, 0);
        std::vector<int64_t> l2p((size_t)M + 1, 0);
        rt->l1_ptr.alloc(M + 1);
        rt->l1_ptr[0] = 0;
        int64_t n_l1 = 0;
        for (long long k = 0; k < M; ++k) {
            const uint32_t i = rt->perm_inv[k];
            rt->csr[k + 1] = rt->csr[k] + (net->syn_ptr[i + 1] - net->syn_ptr[i]);
            l2p[k + 1] = l2p[k] + nseg[k];
            n_l1 += nvn[k];
            if (n_l1 >= (1ll << 32)) { delete rt; return SNN_E_RANGE; }
            rt->l1_ptr[k + 1] = (uint32_t)n_l1;
        }
        const int64_t n_l2 = l2p[M];
        if (n_l2 >= (1ll << 32)) { delete rt; return SNN_E_RANGE; }
        rt->n_l1 = n_l1;
        rt->n_l2 = n_l2;
        rt->bucket_cap.assign((size_t)n_vn, 0);
        rt->inbox_cap.assign((size_t)P, 0);
        std::vector<uint8_t> conn((size_t)P * P, 0);
        for (int32_t ip = 0; ip < P; ++ip) {
            for (int32_t g = 0; g < n_vn; ++g) rt->bucket_cap[g] += bc[(size_t)ip * n_vn + g];
            for (int32_t q = 0; q < P; ++q) {
                rt->inbox_cap[q] += ic[(size_t)ip * P + q];
                conn[(size_t)ip * P + q] = ic[(size_t)ip * P + q] != 0;
            }
        }
        route_connections(rt, conn);
        route_number_pairs(rt, bc, ic);
        RCK(cudaMemcpyAsync(d.bc, bc.data(), 4 * bc.size(), cudaMemcpyHostToDevice, st));
        RCK(cudaMemcpyAsync(d.ic, ic.data(), 4 * ic.size(), cudaMemcpyHostToDevice, st));
        RCK(cudaMemcpyAsync((void *)d.csr, rt->csr.data(), 8 * (size_t)(M + 1), cudaMemcpyHostToDevice, st));
        RCK(cudaMemcpyAsync((void *)d.l2p, l2p.data(), 8 * (size_t)(M + 1), cudaMemcpyHostToDevice, st));
        RCK(cudaMemcpyAsync((void *)d.l1p, rt->l1_ptr.data(), 4 * (size_t)(M + 1), cudaMemcpyHostToDevice, st));

        // ---- pass C in chunks of internal neurons, each copied back
        rt->l1_vn.alloc(n_l1);
        rt->l1_l2.alloc(n_l1 + 1);
        rt->l2.alloc(n_l2);
        rt->l1_pair.alloc(n_l1);
        rt->l2_pair.alloc(n_l2);
        touch_pages(rt->l1_vn.data(), 2 * (size_t)n_l1);
        touch_pages(rt->l1_l2.data(), 4 * (size_t)(n_l1 + 1));
        touch_pages(rt->l2.data(), sizeof(L2Entry) * (size_t)n_l2);
        touch_pages(rt->l1_pair.data(), 4 * (size_t)n_l1);
        touch_pages(rt->l2_pair.data(), 4 * (size_t)n_l2);
        rt->l1_l2[n_l1] = (uint32_t)n_l2;
        pf.join();
        if (pf.bad) { delete rt; return SNN_E_NOMEM; }
        rt->syn_td = std::move(pf.td);
        rt->syn_w = std::move(pf.w);
        if (cudaFuncSetAttribute(k_route_emit_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBigSmem) !=
            cudaSuccess) {
            delete rt;
            return SNN_E_CUDA;
        }
        for (long long k0 = 0; k0 < M;) {
            long long k1 = k0;
            long long big = 0;
            while (k1 < M && rt->csr[k1 + 1] - rt->csr[k0] <= L.cap_syn && l2p[k1 + 1] - l2p[k0] <= L.cap_ent &&
                   (long long)rt->l1_ptr[k1 + 1] - (long long)rt->l1_ptr[k0] <= L.cap_ent) {
                big += (rt->csr[k1 + 1] - rt->csr[k1]) > kCapSmall;
                ++k1;
            }
            if (k1 == k0) { delete rt; return SNN_E_RANGE; }  // (a neuron larger than a chunk: not reached)
            d.k0 = k0;
            d.k1 = k1;
            d.syn0 = rt->csr[k0];
            d.l20 = l2p[k0];
            d.l10 = rt->l1_ptr[k0];
            const int nb = (int)std::min<long long>(k1 - k0, (long long)sms * 8);
            k_route_emit_small<<<nb, kRT, 0, st>>>(d);
            if (big) k_route_emit_big<<<(int)std::min<long long>(big, (long long)sms), kRT, kBigSmem, st>>>(d);
            RCK(cudaGetLastError());
            const long long ns = rt->csr[k1] - rt->csr[k0], n2 = l2p[k1] - l2p[k0];
            const long long n1 = (long long)rt->l1_ptr[k1] - (long long)rt->l1_ptr[k0];
            if (ns) {
                RCK(cudaMemcpyAsync(rt->syn_td.data() + d.syn0, d.o_td, 4 * (size_t)ns, cudaMemcpyDeviceToHost, st));
                RCK(cudaMemcpyAsync(rt->syn_w.data() + d.syn0, d.o_w, 2 * (size_t)ns, cudaMemcpyDeviceToHost, st));
            }
            if (n2) {
                RCK(cudaMemcpyAsync(rt->l2.data() + d.l20, d.o_l2, sizeof(L2Entry) * (size_t)n2,
                                    cudaMemcpyDeviceToHost, st));
                RCK(cudaMemcpyAsync(rt->l2_pair.data() + d.l20, d.o_l2pair, 4 * (size_t)n2, cudaMemcpyDeviceToHost,
                                    st));
            }
            if (n1) {
                RCK(cudaMemcpyAsync(rt->l1_vn.data() + d.l10, d.o_l1vn, 2 * (size_t)n1, cudaMemcpyDeviceToHost, st));
                RCK(cudaMemcpyAsync(rt->l1_l2.data() + d.l10, d.o_l1l2, 4 * (size_t)n1, cudaMemcpyDeviceToHost, st));
                RCK(cudaMemcpyAsync(rt->l1_pair.data() + d.l10, d.o_l1pair, 4 * (size_t)n1, cudaMemcpyDeviceToHost,
                                    st));
            }
            // the chunk buffers are reused by the next chunk
            RCK(cudaStreamSynchronize(st));
            k0 = k1;
        }
        RCK(cudaMemcpyAsync(fl, d.flags, sizeof(fl), cudaMemcpyDeviceToHost, st));
        RCK(cudaStreamSynchronize(st));
        if (fl[0] & (kRCap | kRCount)) { delete rt; return SNN_E_STATE; }
        route_relays(rt, prm->relay, resolve_threads(prm->n_threads));
    } catch (const std::bad_alloc &) {
        delete rt;
        return SNN_E_NOMEM;
    }
    *out = rt;
    return SNN_OK;
}
