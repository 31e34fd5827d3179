// Host side of the library: neuron partitioning (Algorithm 1), partition
// grouping (Algorithm 2) and the two-level routing tables in the device
// layout.  Setup work, run once before a simulation; nothing here is timed
// in a step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <new>
#include <queue>
#include <string>

#include "snn_internal.h"

namespace snn {

int resolve_threads(int requested)
{
    int hw = (int)std::thread::hardware_concurrency();
    if (hw < 1) hw = 1;
    if (requested <= 0 || requested > hw) return hw;
    return requested;
}

void parallel_for(int64_t n, int nthreads, const std::function<void(int64_t, int64_t, int)> &f)
{
    if (n <= 0) return;
    int nt = resolve_threads(nthreads);
    if ((int64_t)nt > n) nt = (int)n;
    if (nt <= 1) {
        f(0, n, 0);
        return;
    }
    std::vector<std::thread> th;
    th.reserve((size_t)nt);
    for (int k = 0; k < nt; ++k) {
        int64_t lo = n * k / nt, hi = n * (k + 1) / nt;
        th.emplace_back([&f, lo, hi, k] { f(lo, hi, k); });
    }
    for (auto &t : th) t.join();
}

// Philox4x32-10 (Salmon et al., SC 2011), host copy for the random choices
// of Algorithms 1 and 2; word 0 of the output block.
static uint32_t philox_w0(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2)
{
    uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = 0;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        uint64_t a = (uint64_t)0xD2511F53u * x0, b = (uint64_t)0xCD9E8D57u * x2;
        uint32_t y0 = (uint32_t)(b >> 32) ^ x1 ^ k0, y2 = (uint32_t)(a >> 32) ^ x3 ^ k1;
        x1 = (uint32_t)b;
        x3 = (uint32_t)a;
        x0 = y0;
        x2 = y2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return x0;
}

// The same word for the device partitioner's seeds (snn_part.cu).
uint32_t philox_word0(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2)
{
    return philox_w0(seed, c0, c1, c2);
}

static int check_network(const snn_network *net)
{
    if (!net || net->n_neurons <= 0 || !net->syn_ptr || !net->v0) return SNN_E_ARG;
    const int64_t M = net->n_neurons;
    if (net->syn_ptr[0] != 0) return SNN_E_ARG;
    for (int64_t i = 0; i < M; ++i)
        if (net->syn_ptr[i + 1] < net->syn_ptr[i]) return SNN_E_ARG;
    if (net->syn_ptr[M] > 0 && (!net->syn_tgt || !net->syn_w || !net->syn_d)) return SNN_E_ARG;
    return SNN_OK;
}

}  // namespace snn

using namespace snn;

extern "C" const char *snn_strerror(int code)
{
    switch (code) {
    case SNN_OK: return "ok";
    case SNN_E_ARG: return "invalid argument";
    case SNN_E_NOMEM: return "out of memory or workspace too small";
    case SNN_E_CAPACITY: return "device buffer capacity exceeded";
    case SNN_E_CUDA: return "CUDA runtime error";
    case SNN_E_RANGE: return "network exceeds a layout limit";
    case SNN_E_STATE: return "invalid state for this call";
    case SNN_E_NODEV: return "no usable CUDA device";
    case SNN_E_TIMEOUT: return "a bounded device-side wait gave up";
    default: return "unknown error";
    }
}

// ------------------------------------------------------------ Algorithm 1
namespace {

struct GreedyAlg1 {
    int64_t M;
    const int64_t *ptr;
    const uint32_t *tgt;
    std::vector<int64_t> in_ptr;
    std::vector<uint32_t> in_src;
    std::vector<int64_t> W;  // out-degree

    explicit GreedyAlg1(const snn_network *net) : M(net->n_neurons), ptr(net->syn_ptr), tgt(net->syn_tgt)
    {
        const int64_t E = ptr[M];
        in_ptr.assign((size_t)M + 1, 0);
        in_src.resize((size_t)E);
        for (int64_t e = 0; e < E; ++e) in_ptr[tgt[e] + 1]++;
        for (int64_t i = 0; i < M; ++i) in_ptr[i + 1] += in_ptr[i];
        std::vector<int64_t> fill(in_ptr.begin(), in_ptr.end() - 1);
        for (int64_t i = 0; i < M; ++i)
            for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) in_src[(size_t)fill[tgt[e]]++] = (uint32_t)i;
        W.resize((size_t)M);
        for (int64_t i = 0; i < M; ++i) W[i] = ptr[i + 1] - ptr[i];
    }

    int64_t objective(const int32_t *lab) const
    {
        int64_t c = 0;
        for (int64_t i = 0; i < M; ++i)
            for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e)
                if (lab[i] != lab[tgt[e]]) c += W[i] * W[tgt[e]];
        return c;
    }

    // One greedy pass t; heap keyed by (gain desc, id asc) over unassigned
    // neurons with positive gain; zero-gain picks fall back to the lowest
    // unassigned id, which is what a full scan with ties to the lowest id gives.
    void pass(int32_t P, int32_t t, uint64_t seed, std::vector<int32_t> &lab) const
    {
        lab.assign((size_t)M, -1);
        std::vector<int64_t> gain((size_t)M, 0);
        std::vector<int64_t> touched;
        int64_t Wtot = 0;
        for (int64_t i = 0; i < M; ++i) Wtot += W[i];
        int64_t n_un = M;
        int64_t low = 0;  // lowest possibly unassigned id
        typedef std::pair<int64_t, int64_t> Item;  // (gain, -id): max-heap => max gain, min id
        for (int32_t k = 0; k < P; ++k) {
            if (k == P - 1) {
                for (int64_t i = 0; i < M; ++i)
                    if (lab[i] < 0) lab[i] = k;
                break;
            }
            if (n_un == 0) break;
            while (low < M && lab[low] >= 0) ++low;
            int64_t s;
            if (t == 1) {
                s = low;
            } else {
                int64_t r = (int64_t)(philox_w0(seed, (uint32_t)t, (uint32_t)k, 0xA1u) % (uint64_t)n_un);
                s = -1;
                for (int64_t i = low; i < M; ++i)
                    if (lab[i] < 0) {
                        if (r == 0) { s = i; break; }
                        --r;
                    }
            }
            for (int64_t j : touched) gain[j] = 0;
            touched.clear();
            std::priority_queue<Item> heap;
            int64_t wk = 0, add = s;
            while (add >= 0) {
                lab[add] = k;
                --n_un;
                const int64_t wa = W[add];
                wk += wa;
                auto bump = [&](int64_t j) {
                    int64_t inc = wa * W[j];
                    if (gain[j] == 0) touched.push_back(j);
                    gain[j] += inc;
                    if (lab[j] < 0 && gain[j] > 0) heap.push(Item(gain[j], -j));
                };
                for (int64_t e = ptr[add]; e < ptr[add + 1]; ++e) bump(tgt[e]);
                for (int64_t e = in_ptr[add]; e < in_ptr[add + 1]; ++e) bump(in_src[e]);
                if (!(wk * (int64_t)P < Wtot) || n_un == 0) break;
                add = -1;
                while (!heap.empty()) {
                    Item it = heap.top();
                    int64_t j = -it.second;
                    if (lab[j] >= 0 || gain[j] != it.first) {
                        heap.pop();
                        continue;
                    }
                    add = j;
                    break;
                }
                if (add < 0) {
                    while (low < M && lab[low] >= 0) ++low;
                    add = low;
                }
            }
        }
    }
};

}  // namespace

extern "C" int snn_partition(const snn_network *net, int32_t P, const snn_partition_params *prm,
                             int32_t *part_of, snn_partition_stats *stats)
{
    if (check_network(net) != SNN_OK || !prm || !part_of) return SNN_E_ARG;
    const int64_t M = net->n_neurons;
    if (P < 1 || P > M) return SNN_E_ARG;
    try {
        if (prm->mode == SNN_PART_PLANTED) {
            for (int32_t p = 0; p < P; ++p)
                for (int64_t i = (int64_t)p * M / P; i < (int64_t)(p + 1) * M / P; ++i) part_of[i] = p;
        } else if (prm->mode == SNN_PART_RANDOM) {
            // balanced random: a seeded shuffle of the ids cut into P runs
            std::vector<uint32_t> ids((size_t)M);
            for (int64_t i = 0; i < M; ++i) ids[i] = (uint32_t)i;
            uint64_t st = prm->seed ^ 0x5DEECE66DULL;
            for (int64_t i = M - 1; i > 0; --i) {
                st += 0x9E3779B97F4A7C15ULL;
                uint64_t z = st;
                z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
                z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
                z ^= z >> 31;
                int64_t j = (int64_t)(((unsigned __int128)z * (uint64_t)(i + 1)) >> 64);
                std::swap(ids[i], ids[j]);
            }
            for (int32_t p = 0; p < P; ++p)
                for (int64_t x = (int64_t)p * M / P; x < (int64_t)(p + 1) * M / P; ++x) part_of[ids[x]] = p;
        } else if (prm->mode == SNN_PART_GREEDY) {
            if (prm->iters < 1) return SNN_E_ARG;
            for (int64_t i = 0; i < M; ++i)
                if (net->syn_ptr[i + 1] > net->syn_ptr[i])
                    for (int64_t e = net->syn_ptr[i]; e < net->syn_ptr[i + 1]; ++e)
                        if (net->syn_tgt[e] >= (uint64_t)M) return SNN_E_ARG;
            GreedyAlg1 g(net);
            std::vector<int32_t> lab;
            int64_t best = -1;
            for (int32_t t = 1; t <= prm->iters; ++t) {
                g.pass(P, t, prm->seed, lab);
                int64_t c = g.objective(lab.data());
                if (best < 0 || c < best) {
                    best = c;
                    std::memcpy(part_of, lab.data(), sizeof(int32_t) * (size_t)M);
                }
            }
        } else {
            return SNN_E_ARG;
        }
        if (stats) {
            std::vector<int64_t> wsum((size_t)P, 0);
            int64_t obj = 0;
            for (int64_t i = 0; i < M; ++i) {
                int64_t wi = net->syn_ptr[i + 1] - net->syn_ptr[i];
                wsum[part_of[i]] += wi;
                for (int64_t e = net->syn_ptr[i]; e < net->syn_ptr[i + 1]; ++e) {
                    uint32_t j = net->syn_tgt[e];
                    if (part_of[i] != part_of[j]) obj += wi * (net->syn_ptr[j + 1] - net->syn_ptr[j]);
                }
            }
            stats->objective = obj;
            stats->min_weight = *std::min_element(wsum.begin(), wsum.end());
            stats->max_weight = *std::max_element(wsum.begin(), wsum.end());
        }
    } catch (const std::bad_alloc &) {
        return SNN_E_NOMEM;
    }
    return SNN_OK;
}

// ------------------------------------------------------------ Algorithm 2
namespace {

typedef unsigned __int128 u128;

// Greedy grouping of P partitions into n_vn groups of size s.
static void group_greedy(int32_t P, int32_t n_vn, int32_t iters, uint64_t seed,
                         const std::vector<int64_t> &PG, const std::vector<int64_t> &WG,
                         std::vector<int32_t> &best_grp, u128 &best_cost)
{
    const int32_t s = P / n_vn;
    std::vector<int32_t> grp((size_t)P);
    bool have = false;
    for (int32_t t = 1; t <= iters; ++t) {
        std::fill(grp.begin(), grp.end(), -1);
        int32_t n_un = P;
        for (int32_t g = 0; g < n_vn; ++g) {
            if (g == n_vn - 1) {
                for (int32_t p = 0; p < P; ++p)
                    if (grp[p] < 0) grp[p] = g;
                break;
            }
            int32_t seedp = -1;
            if (t == 1) {
                for (int32_t p = 0; p < P; ++p)
                    if (grp[p] < 0 && (seedp < 0 || WG[p] > WG[seedp])) seedp = p;
            } else {
                uint32_t r = philox_w0(seed, (uint32_t)t, (uint32_t)g, 0xA2u) % (uint32_t)n_un;
                for (int32_t p = 0; p < P; ++p)
                    if (grp[p] < 0) {
                        if (r == 0) { seedp = p; break; }
                        --r;
                    }
            }
            grp[seedp] = g;
            --n_un;
            std::vector<int32_t> members(1, seedp);
            while ((int32_t)members.size() < s) {
                int32_t bq = -1;
                u128 bg = 0;
                for (int32_t q = 0; q < P; ++q) {
                    if (grp[q] >= 0) continue;
                    u128 gq = 0;
                    for (int32_t m : members)
                        gq += (u128)(PG[(size_t)m * P + q] + PG[(size_t)q * P + m]) * (u128)WG[m] * (u128)WG[q];
                    if (bq < 0 || gq > bg) { bq = q; bg = gq; }
                }
                grp[bq] = g;
                --n_un;
                members.push_back(bq);
            }
        }
        u128 cost = 0;
        for (int32_t p = 0; p < P; ++p)
            for (int32_t q = 0; q < P; ++q)
                if (grp[p] != grp[q]) cost += (u128)PG[(size_t)p * P + q] * (u128)WG[p] * (u128)WG[q];
        if (!have || cost < best_cost) {
            best_cost = cost;
            best_grp = grp;
            have = true;
        }
    }
}

}  // namespace

namespace snn {

void route_groups(snn_routing *rt, const snn_routing_params *prm, const std::vector<int64_t> &PG,
                  const std::vector<int64_t> &WG)
{
    const int32_t P = rt->P, n_vn = rt->n_vn, s = rt->vn_size;
    rt->vn_of_part.assign((size_t)P, 0);
    if (prm->grouping == SNN_GROUP_CONTIGUOUS) {
        for (int32_t p = 0; p < P; ++p) rt->vn_of_part[p] = p / s;
        u128 c = 0;
        for (int32_t p = 0; p < P; ++p)
            for (int32_t q = 0; q < P; ++q)
                if (p / s != q / s) c += (u128)PG[(size_t)p * P + q] * (u128)WG[p] * (u128)WG[q];
        rt->group_cost = c;
    } else {
        group_greedy(P, n_vn, prm->iters, prm->seed, PG, WG, rt->vn_of_part, rt->group_cost);
    }
}

void route_order(snn_routing *rt, const snn_network *net, const int32_t *part_of, const std::vector<int64_t> &sizes)
{
    const int32_t P = rt->P, n_vn = rt->n_vn, s = rt->vn_size;
    const int64_t M = rt->M;
    // internal partition order: by (VN, label)
    rt->part_of_ip.resize((size_t)P);
    rt->ip_of_part.resize((size_t)P);
    {
        std::vector<int32_t> fill((size_t)n_vn, 0);
        for (int32_t p = 0; p < P; ++p) {
            int32_t g = rt->vn_of_part[p];
            int32_t ip = g * s + fill[g]++;
            rt->ip_of_part[p] = ip;
            rt->part_of_ip[ip] = p;
        }
    }
    // relay of VN g for source VN h: ((h - g) mod s)-th member of g in label order,
    // which is internal partition g*s + (h - g) mod s
    rt->relay.resize((size_t)n_vn * n_vn);
    for (int32_t g = 0; g < n_vn; ++g)
        for (int32_t h = 0; h < n_vn; ++h) rt->relay[(size_t)g * n_vn + h] = rt->part_of_ip[g * s + vn_rank(h, g, s)];

    // internal neuron order: partition-major, ascending global id
    rt->pbase.assign((size_t)P + 1, 0);
    for (int32_t p = 0; p < P; ++p) rt->pbase[rt->ip_of_part[p] + 1] = sizes[p];
    for (int32_t ip = 0; ip < P; ++ip) rt->pbase[ip + 1] += rt->pbase[ip];
    rt->perm_inv.resize((size_t)M);
    rt->perm_fwd.resize((size_t)M);
    {
        std::vector<int64_t> fill(rt->pbase.begin(), rt->pbase.end() - 1);
        for (int64_t i = 0; i < M; ++i) {
            int64_t k = fill[rt->ip_of_part[part_of[i]]]++;
            rt->perm_inv[k] = (uint32_t)i;
            rt->perm_fwd[i] = (uint32_t)k;
        }
    }
    rt->identity = true;
    for (int64_t i = 0; i < M; ++i)
        if (rt->perm_fwd[i] != (uint32_t)i) { rt->identity = false; break; }
    rt->v0.resize((size_t)M);
    for (int64_t k = 0; k < M; ++k) rt->v0[k] = net->v0[rt->perm_inv[k]];
    rt->src_part.resize((size_t)M);
    for (int32_t ip = 0; ip < P; ++ip)
        for (int64_t k = rt->pbase[ip]; k < rt->pbase[ip + 1]; ++k) rt->src_part[k] = (uint16_t)ip;
}

void route_connections(snn_routing *rt, const std::vector<uint8_t> &conn)
{
    const int32_t P = rt->P, n_vn = rt->n_vn, s = rt->vn_size;
    // static connections per partition (label order)
    rt->conn_direct.assign((size_t)P, 0);
    rt->conn_two.assign((size_t)P, 0);
    for (int32_t p = 0; p < P; ++p) {
        int32_t ip = rt->ip_of_part[p], h = ip / s;
        std::vector<uint8_t> gr((size_t)n_vn, 0);
        for (int32_t q = 0; q < P; ++q) {
            if (q == ip || !conn[(size_t)ip * P + q]) continue;
            rt->conn_direct[p]++;
            if (q / s == h) rt->conn_two[p]++;
            else gr[q / s] = 1;
        }
        for (int32_t g = 0; g < n_vn; ++g) rt->conn_two[p] += gr[g];
    }
}

void route_number_pairs(snn_routing *rt, std::vector<uint32_t> &bc, std::vector<uint32_t> &ic)
{
    const int32_t P = rt->P;
    // number the pairs; the dense tables then hold each pair's id
    auto number = [P](std::vector<uint32_t> &dense, int32_t n_dst, std::vector<uint32_t> &ptr,
                      std::vector<uint16_t> &dst, std::vector<uint32_t> &cap) {
        ptr.assign((size_t)P + 1, 0);
        dst.clear();
        cap.clear();
        for (int32_t ip = 0; ip < P; ++ip) {
            for (int32_t x = 0; x < n_dst; ++x) {
                uint32_t &v = dense[(size_t)ip * n_dst + x];
                if (!v) continue;
                dst.push_back((uint16_t)x);
                cap.push_back(v);
                v = (uint32_t)(cap.size() - 1);
            }
            ptr[ip + 1] = (uint32_t)cap.size();
        }
    };
    number(bc, rt->n_vn, rt->bpair_ptr, rt->bpair_dst, rt->bpair_cap);
    number(ic, P, rt->ipair_ptr, rt->ipair_dst, rt->ipair_cap);
}

void route_relay_map(const snn_routing *rt, int32_t policy, std::vector<int32_t> &relay_ip)
{
    const int32_t P = rt->P, n_vn = rt->n_vn, s = rt->vn_size;
    relay_ip.assign((size_t)n_vn * P, -1);
    for (int32_t g = 0; g < n_vn; ++g)
        for (int32_t ip = 0; ip < P; ++ip) {
            if (ip / s == g) continue;
            // internal partitions are VN-major, by ascending label inside a VN:
            // the rank of ip in its VN is ip mod s, member k of g is g*s + k
            relay_ip[(size_t)g * P + ip] = policy == SNN_RELAY_PER_VN ? g * s + vn_rank(ip / s, g, s) : g * s + ip % s;
        }
    if (policy != SNN_RELAY_BALANCED) return;
    // static load of (g, source ip): its level-2 pairs into the partitions of g
    std::vector<int64_t> load((size_t)n_vn * P, 0);
    for (int32_t ip = 0; ip < P; ++ip)
        for (uint32_t k = rt->ipair_ptr[ip]; k < rt->ipair_ptr[ip + 1]; ++k) {
            const int32_t q = rt->ipair_dst[k];
            if (q / s != ip / s) load[(size_t)(q / s) * P + ip] += rt->ipair_cap[k];
        }
    std::vector<int32_t> src;
    std::vector<int64_t> acc((size_t)s);
    for (int32_t g = 0; g < n_vn; ++g) {
        src.clear();
        for (int32_t ip = 0; ip < P; ++ip)
            if (ip / s != g && load[(size_t)g * P + ip] > 0) src.push_back(ip);
        const int64_t *lg = &load[(size_t)g * P];
        std::sort(src.begin(), src.end(), [&](int32_t a, int32_t b) {
            if (lg[a] != lg[b]) return lg[a] > lg[b];
            return rt->part_of_ip[a] < rt->part_of_ip[b];
        });
        std::fill(acc.begin(), acc.end(), 0);
        for (int32_t ip : src) {
            int32_t k = 0;
            for (int32_t m = 1; m < s; ++m)
                if (acc[m] < acc[k]) k = m;
            acc[k] += lg[ip];
            relay_ip[(size_t)g * P + ip] = g * s + k;
        }
    }
}

void route_relays(snn_routing *rt, int32_t policy, int nthreads)
{
    const int32_t P = rt->P, n_vn = rt->n_vn, s = rt->vn_size;
    rt->relay_policy = policy;
    route_relay_map(rt, policy, rt->relay_ip);
    if (policy != SNN_RELAY_PER_VN) std::fill(rt->relay.begin(), rt->relay.end(), -1);
    if (policy == SNN_RELAY_PER_VN) return;  // the builders' classes already follow it
    // the relay classes of the level-2 entries under the policy's relays
    parallel_for(P, nthreads, [&](int64_t plo, int64_t phi, int) {
        for (int64_t ip = plo; ip < phi; ++ip) {
            const int32_t hs = (int32_t)ip / s;
            for (int64_t k = rt->pbase[ip]; k < rt->pbase[ip + 1]; ++k)
                for (uint32_t e = rt->l1_ptr[k]; e < rt->l1_ptr[k + 1]; ++e) {
                    const int32_t g = rt->l1_vn[e];
                    if (g == hs) continue;
                    const int32_t r = rt->relay_ip[(size_t)g * P + ip];
                    for (uint32_t f = rt->l1_l2[e]; f < rt->l1_l2[e + 1]; ++f)
                        rt->l2[f].cls = rt->l2[f].q == r ? kClsRelayLocal : kClsRelayRemote;
                }
        }
    });
    (void)n_vn;
}

}  // namespace snn

extern "C" int snn_routing_build(const snn_network *net, const int32_t *part_of, int32_t P,
                                 int32_t n_vn, const snn_routing_params *prm, snn_routing **out)
{
    if (!out) return SNN_E_ARG;
    *out = nullptr;
    if (check_network(net) != SNN_OK || !part_of || !prm) return SNN_E_ARG;
    const int64_t M = net->n_neurons, E = net->syn_ptr[M];
    if (P < 1 || n_vn < 1 || P % n_vn || P > M) return SNN_E_ARG;
    if (P > 4096) return SNN_E_RANGE;
    if (prm->grouping != SNN_GROUP_CONTIGUOUS && prm->grouping != SNN_GROUP_GREEDY) return SNN_E_ARG;
    if (prm->grouping == SNN_GROUP_GREEDY && prm->iters < 1) return SNN_E_ARG;
    if (prm->relay < SNN_RELAY_PER_VN || prm->relay > SNN_RELAY_BALANCED) return SNN_E_ARG;
    if (M >= (int64_t)1 << kTgtBits) return SNN_E_RANGE;
    if (E >= (int64_t)1 << 40) return SNN_E_RANGE;
    const int nt = resolve_threads(prm->n_threads);
    const int64_t *sp = net->syn_ptr;
    const uint32_t *tg = net->syn_tgt;
    const uint8_t *dd = net->syn_d;

    snn_routing *rt = nullptr;
    try {
        rt = new snn_routing();
        rt->M = M;
        rt->E = E;
        rt->P = P;
        rt->n_vn = n_vn;
        rt->vn_size = P / n_vn;
        const int32_t s = rt->vn_size;

        // ---- validation and per-thread partition graph
        std::vector<int64_t> sizes((size_t)P, 0);
        for (int64_t i = 0; i < M; ++i) {
            if (part_of[i] < 0 || part_of[i] >= P) { delete rt; return SNN_E_ARG; }
            sizes[part_of[i]]++;
        }
        for (int32_t p = 0; p < P; ++p)
            if (sizes[p] == 0) { delete rt; return SNN_E_ARG; }
        std::vector<std::vector<int64_t>> pg_t((size_t)nt);
        std::vector<int> bad((size_t)nt, 0), maxd((size_t)nt, 1);
        std::vector<int64_t> WG((size_t)P, 0);
        parallel_for(M, nt, [&](int64_t lo, int64_t hi, int k) {
            std::vector<int64_t> &pg = pg_t[k];
            pg.assign((size_t)P * P, 0);
            for (int64_t i = lo; i < hi; ++i) {
                int64_t deg = sp[i + 1] - sp[i];
                if (deg >= ((int64_t)1 << kLenBits)) bad[k] = SNN_E_RANGE;
                int32_t p = part_of[i];
                for (int64_t e = sp[i]; e < sp[i + 1]; ++e) {
                    if (tg[e] >= (uint64_t)M) { bad[k] = SNN_E_ARG; continue; }
                    if (dd[e] < 1 || dd[e] > kMaxDelay) { bad[k] = SNN_E_RANGE; continue; }
                    if (dd[e] > maxd[k]) maxd[k] = dd[e];
                    int32_t q = part_of[tg[e]];
                    if (q != p) pg[(size_t)p * P + q]++;
                }
            }
        });
        for (int k = 0; k < nt; ++k)
            if (bad[k]) { int rc = bad[k]; delete rt; return rc; }
        std::vector<int64_t> PG((size_t)P * P, 0);
        for (int k = 0; k < nt; ++k) {
            if (pg_t[k].empty()) continue;
            for (size_t x = 0; x < PG.size(); ++x) PG[x] += pg_t[k][x];
            rt->max_delay = std::max(rt->max_delay, maxd[k]);
        }
        pg_t.clear();
        for (int64_t i = 0; i < M; ++i) WG[part_of[i]] += sp[i + 1] - sp[i];

        // ---- Algorithm 2: groups; internal order
        route_groups(rt, prm, PG, WG);
        route_order(rt, net, part_of, sizes);

        // ---- pass 1: per internal neuron, segment and VN counts
        std::vector<int64_t> csr((size_t)M + 1, 0), l2p((size_t)M + 1, 0);
        std::vector<uint32_t> nl1((size_t)M + 1, 0);
        std::vector<std::vector<uint64_t>> bcap_t((size_t)nt), icap_t((size_t)nt);
        std::vector<std::vector<uint8_t>> conn_t((size_t)nt);
        parallel_for(M, nt, [&](int64_t lo, int64_t hi, int k) {
            std::vector<int32_t> cnt((size_t)P, 0);
            std::vector<uint8_t> gm((size_t)n_vn, 0);
            bcap_t[k].assign((size_t)n_vn, 0);
            icap_t[k].assign((size_t)P, 0);
            conn_t[k].assign((size_t)P * P, 0);
            for (int64_t kk = lo; kk < hi; ++kk) {
                int64_t i = rt->perm_inv[kk];
                int32_t ps = rt->ip_of_part[part_of[i]];
                int64_t nseg = 0, nvn = 0;
                for (int64_t e = sp[i]; e < sp[i + 1]; ++e) {
                    int32_t q = rt->ip_of_part[part_of[tg[e]]];
                    if (cnt[q]++ == 0) {
                        ++nseg;
                        icap_t[k][q]++;
                        conn_t[k][(size_t)ps * P + q] = 1;
                        int32_t g = q / s;
                        if (!gm[g]) { gm[g] = 1; ++nvn; bcap_t[k][g]++; }
                    }
                }
                for (int64_t e = sp[i]; e < sp[i + 1]; ++e) {
                    int32_t q = rt->ip_of_part[part_of[tg[e]]];
                    cnt[q] = 0;
                    gm[q / s] = 0;
                }
                csr[kk + 1] = sp[i + 1] - sp[i];
                l2p[kk + 1] = nseg;
                nl1[kk + 1] = (uint32_t)nvn;
            }
        });
        for (int64_t k = 0; k < M; ++k) {
            csr[k + 1] += csr[k];
            l2p[k + 1] += l2p[k];
        }
        int64_t n_l1 = 0;
        rt->l1_ptr.alloc(M + 1);
        rt->l1_ptr[0] = 0;
        for (int64_t k = 0; k < M; ++k) {
            n_l1 += nl1[k + 1];
            if (n_l1 >= ((int64_t)1 << 32)) { delete rt; return SNN_E_RANGE; }
            rt->l1_ptr[k + 1] = (uint32_t)n_l1;
        }
        const int64_t n_l2 = l2p[M];
        if (n_l2 >= ((int64_t)1 << 32)) { delete rt; return SNN_E_RANGE; }
        rt->n_l1 = n_l1;
        rt->n_l2 = n_l2;
        rt->bucket_cap.assign((size_t)n_vn, 0);
        rt->inbox_cap.assign((size_t)P, 0);
        std::vector<uint8_t> conn((size_t)P * P, 0);
        for (int k = 0; k < nt; ++k) {
            if (bcap_t[k].empty()) continue;
            for (int32_t g = 0; g < n_vn; ++g) rt->bucket_cap[g] += bcap_t[k][g];
            for (int32_t q = 0; q < P; ++q) rt->inbox_cap[q] += icap_t[k][q];
            for (size_t x = 0; x < conn.size(); ++x) conn[x] |= conn_t[k][x];
        }
        bcap_t.clear();
        icap_t.clear();
        conn_t.clear();

        route_connections(rt, conn);

        // ---- pass 2: fill the CSR and the level-1 / level-2 tables
        rt->syn_td.alloc(E);
        rt->syn_w.alloc(E);
        rt->l1_vn.alloc(n_l1);
        rt->l1_l2.alloc(n_l1 + 1);
        rt->l2.alloc(n_l2);
        rt->l1_l2[n_l1] = (uint32_t)n_l2;
        rt->csr = csr;
        parallel_for(M, nt, [&](int64_t lo, int64_t hi, int) {
            std::vector<int32_t> cnt((size_t)P, 0), pos((size_t)P, 0);
            std::vector<int32_t> qs;
            std::vector<uint64_t> key;
            for (int64_t kk = lo; kk < hi; ++kk) {
                int64_t i = rt->perm_inv[kk];
                int32_t ps = rt->ip_of_part[part_of[i]], hs = ps / s;
                qs.clear();
                for (int64_t e = sp[i]; e < sp[i + 1]; ++e) {
                    int32_t q = rt->ip_of_part[part_of[tg[e]]];
                    if (cnt[q]++ == 0) qs.push_back(q);
                }
                std::sort(qs.begin(), qs.end());
                int64_t base = csr[kk];
                int32_t run = 0;
                for (int32_t q : qs) {
                    pos[q] = run;
                    run += cnt[q];
                }
                int64_t f = l2p[kk];
                uint32_t e1 = rt->l1_ptr[kk];
                int32_t lastg = -1;
                for (int32_t q : qs) {
                    int32_t g = q / s;
                    if (g != lastg) {
                        rt->l1_vn[e1] = (uint16_t)g;
                        rt->l1_l2[e1] = (uint32_t)f;
                        ++e1;
                        lastg = g;
                    }
                    L2Entry &l = rt->l2[f++];
                    l.off = (uint64_t)(base + pos[q]);
                    l.len = (uint32_t)cnt[q];
                    l.q = (uint16_t)q;
                    l.pad = 0;
                    if (g == hs) l.cls = (q == ps) ? kClsLocal : kClsPeer;
                    else l.cls = (q == g * s + vn_rank(hs, g, s)) ? kClsRelayLocal : kClsRelayRemote;
                }
                for (int64_t e = sp[i]; e < sp[i + 1]; ++e) {
                    int32_t q = rt->ip_of_part[part_of[tg[e]]];
                    int64_t o = base + pos[q]++;
                    rt->syn_td[o] = rt->perm_fwd[tg[e]] | ((uint32_t)(dd[e] - 1) << kTgtBits);
                    rt->syn_w[o] = net->syn_w[e];
                }
                // each segment by (delay, target): the delay-1 synapses first
                for (int64_t x = l2p[kk]; x < f; ++x) {
                    L2Entry &l = rt->l2[x];
                    key.clear();
                    for (uint32_t k = 0; k < l.len; ++k)
                        key.push_back(((uint64_t)rt->syn_td[l.off + k] << 16) | (uint16_t)rt->syn_w[l.off + k]);
                    std::sort(key.begin(), key.end());
                    uint64_t n1 = 0;
                    for (uint32_t k = 0; k < l.len; ++k) {
                        rt->syn_td[l.off + k] = (uint32_t)(key[k] >> 16);
                        rt->syn_w[l.off + k] = (int16_t)(uint16_t)(key[k] & 0xFFFFu);
                        n1 += (key[k] >> (16 + kTgtBits)) == 0;
                    }
                    l.off |= n1 << kOffBits;
                }
                for (int32_t q : qs) cnt[q] = 0;
            }
        });

        // ---- exchange pairs and their exact worst cases by source partition
        // (each partition's neurons are contiguous in the internal order)
        std::vector<uint32_t> bc((size_t)P * n_vn, 0), ic((size_t)P * P, 0);
        parallel_for(P, nt, [&](int64_t plo, int64_t phi, int) {
            for (int64_t ip = plo; ip < phi; ++ip) {
                uint32_t *b = &bc[(size_t)ip * n_vn];
                uint32_t *c = &ic[(size_t)ip * P];
                for (int64_t k = rt->pbase[ip]; k < rt->pbase[ip + 1]; ++k) {
                    for (uint32_t e = rt->l1_ptr[k]; e < rt->l1_ptr[k + 1]; ++e) b[rt->l1_vn[e]]++;
                    const uint32_t f0 = rt->l1_l2[rt->l1_ptr[k]], f1 = rt->l1_l2[rt->l1_ptr[k + 1]];
                    for (uint32_t f = f0; f < f1; ++f) c[rt->l2[f].q]++;
                }
            }
        });
        route_number_pairs(rt, bc, ic);
        rt->l1_pair.alloc(n_l1);
        rt->l2_pair.alloc(n_l2);
        parallel_for(P, nt, [&](int64_t plo, int64_t phi, int) {
            for (int64_t ip = plo; ip < phi; ++ip)
                for (int64_t k = rt->pbase[ip]; k < rt->pbase[ip + 1]; ++k)
                    for (uint32_t e = rt->l1_ptr[k]; e < rt->l1_ptr[k + 1]; ++e) {
                        rt->l1_pair[e] = bc[(size_t)ip * n_vn + rt->l1_vn[e]];
                        for (uint32_t f = rt->l1_l2[e]; f < rt->l1_l2[e + 1]; ++f)
                            rt->l2_pair[f] = ic[(size_t)ip * P + rt->l2[f].q];
                    }
        });
        route_relays(rt, prm->relay, nt);
    } catch (const std::bad_alloc &) {
        delete rt;
        return SNN_E_NOMEM;
    }
    *out = rt;
    return SNN_OK;
}

extern "C" int snn_routing_info_get(const snn_routing *rt, snn_routing_info *o)
{
    if (!rt || !o) return SNN_E_ARG;
    std::memset(o, 0, sizeof(*o));
    o->n_neurons = rt->M;
    o->n_synapses = rt->E;
    o->n_parts = rt->P;
    o->n_vn = rt->n_vn;
    o->vn_size = rt->vn_size;
    o->max_delay = rt->max_delay;
    o->n_l1 = rt->n_l1;
    o->n_l2 = rt->n_l2;
    o->group_cost_lo = (uint64_t)rt->group_cost;
    o->group_cost_hi = (uint64_t)(rt->group_cost >> 64);
    for (int32_t p = 0; p < rt->P; ++p) {
        o->conn_direct_sum += rt->conn_direct[p];
        o->conn_two_level_sum += rt->conn_two[p];
        o->conn_direct_max = std::max(o->conn_direct_max, rt->conn_direct[p]);
        o->conn_two_level_max = std::max(o->conn_two_level_max, rt->conn_two[p]);
    }
    o->identity_order = rt->identity ? 1 : 0;
    return SNN_OK;
}

extern "C" int snn_routing_groups(const snn_routing *rt, int32_t *vn_of_part, int32_t *relay)
{
    if (!rt) return SNN_E_ARG;
    if (vn_of_part) std::memcpy(vn_of_part, rt->vn_of_part.data(), sizeof(int32_t) * (size_t)rt->P);
    if (relay) std::memcpy(relay, rt->relay.data(), sizeof(int32_t) * rt->relay.size());
    return SNN_OK;
}

extern "C" int snn_routing_traffic(const snn_routing *rt, const uint32_t *ids, int64_t n, int32_t relay_policy,
                                   int64_t *direct_out, int64_t *direct_in, int64_t *two_out, int64_t *two_in)
{
    if (!rt || n < 0 || (n > 0 && !ids)) return SNN_E_ARG;
    if (relay_policy < -1 || relay_policy > SNN_RELAY_BALANCED) return SNN_E_ARG;
    std::vector<int32_t> own;
    if (relay_policy >= 0 && relay_policy != rt->relay_policy) route_relay_map(rt, relay_policy, own);
    const std::vector<int32_t> &relay_ip = own.empty() ? rt->relay_ip : own;
    for (int64_t x = 0; x < n; ++x)
        if ((int64_t)ids[x] >= rt->M) return SNN_E_ARG;
    const int32_t P = rt->P, s = rt->vn_size;
    const int nt = resolve_threads(0);
    // per thread: [4][P] in internal partition order
    std::vector<std::vector<int64_t>> acc((size_t)nt);
    parallel_for(n, nt, [&](int64_t lo, int64_t hi, int k) {
        std::vector<int64_t> &a = acc[k];
        a.assign((size_t)4 * P, 0);
        int64_t *dout = a.data(), *din = dout + P, *tout = din + P, *tin = tout + P;
        for (int64_t x = lo; x < hi; ++x) {
            const int64_t i = rt->perm_fwd[ids[x]];
            const int32_t ps = rt->src_part[i], hs = ps / s;
            for (uint32_t e = rt->l1_ptr[i]; e < rt->l1_ptr[i + 1]; ++e) {
                const int32_t g = rt->l1_vn[e];
                const int32_t r = g == hs ? -1 : relay_ip[(size_t)g * P + ps];
                if (g != hs) {  // level 1: one message to the relay of g
                    ++tout[ps];
                    ++tin[r];
                }
                for (uint32_t f = rt->l1_l2[e]; f < rt->l1_l2[e + 1]; ++f) {
                    const int32_t q = rt->l2[f].q;
                    if (q == ps) continue;
                    ++dout[ps];
                    ++din[q];
                    if (g == hs) {  // peer of the own VN: direct
                        ++tout[ps];
                        ++tin[q];
                    } else if (q != r) {  // level 2: the relay forwards
                        ++tout[r];
                        ++tin[q];
                    }
                }
            }
        }
    });
    int64_t *outs[4] = {direct_out, direct_in, two_out, two_in};
    for (int c = 0; c < 4; ++c) {
        if (!outs[c]) continue;
        for (int32_t p = 0; p < P; ++p) outs[c][p] = 0;
        for (int k = 0; k < nt; ++k)
            if (!acc[k].empty())
                for (int32_t ip = 0; ip < P; ++ip) outs[c][rt->part_of_ip[ip]] += acc[k][(size_t)c * P + ip];
    }
    return SNN_OK;
}

extern "C" int snn_routing_relays(const snn_routing *rt, int32_t policy, int32_t *relay)
{
    if (!rt || !relay || policy < -1 || policy > SNN_RELAY_BALANCED) return SNN_E_ARG;
    std::vector<int32_t> own;
    if (policy >= 0 && policy != rt->relay_policy) route_relay_map(rt, policy, own);
    const std::vector<int32_t> &rip = own.empty() ? rt->relay_ip : own;
    const int32_t P = rt->P;
    for (int32_t g = 0; g < rt->n_vn; ++g)
        for (int32_t p = 0; p < P; ++p) {
            const int32_t r = rip[(size_t)g * P + rt->ip_of_part[p]];
            relay[(size_t)g * P + p] = r < 0 ? -1 : rt->part_of_ip[r];
        }
    return SNN_OK;
}

extern "C" int snn_routing_connections(const snn_routing *rt, int32_t *direct, int32_t *two_level)
{
    if (!rt) return SNN_E_ARG;
    if (direct) std::memcpy(direct, rt->conn_direct.data(), sizeof(int32_t) * (size_t)rt->P);
    if (two_level) std::memcpy(two_level, rt->conn_two.data(), sizeof(int32_t) * (size_t)rt->P);
    return SNN_OK;
}

extern "C" int snn_routing_export(const snn_routing *rt, const char *name, void *out, size_t cap, size_t *bytes)
{
    if (!rt || !name) return SNN_E_ARG;
    const void *src = nullptr;
    size_t n = 0;
    auto take = [&](const void *p, size_t b) {
        src = p;
        n = b;
    };
    const std::string k(name);
    if (k == "syn_td") take(rt->syn_td.data(), 4 * (size_t)rt->E);
    else if (k == "syn_w") take(rt->syn_w.data(), 2 * (size_t)rt->E);
    else if (k == "csr") take(rt->csr.data(), 8 * rt->csr.size());
    else if (k == "l1_ptr") take(rt->l1_ptr.data(), 4 * (size_t)(rt->M + 1));
    else if (k == "l1_vn") take(rt->l1_vn.data(), 2 * (size_t)rt->n_l1);
    else if (k == "l1_l2") take(rt->l1_l2.data(), 4 * (size_t)(rt->n_l1 + 1));
    else if (k == "l2") take(rt->l2.data(), sizeof(L2Entry) * (size_t)rt->n_l2);
    else if (k == "l1_pair") take(rt->l1_pair.data(), 4 * (size_t)rt->n_l1);
    else if (k == "l2_pair") take(rt->l2_pair.data(), 4 * (size_t)rt->n_l2);
    else if (k == "bpair_ptr") take(rt->bpair_ptr.data(), 4 * rt->bpair_ptr.size());
    else if (k == "bpair_dst") take(rt->bpair_dst.data(), 2 * rt->bpair_dst.size());
    else if (k == "bpair_cap") take(rt->bpair_cap.data(), 4 * rt->bpair_cap.size());
    else if (k == "ipair_ptr") take(rt->ipair_ptr.data(), 4 * rt->ipair_ptr.size());
    else if (k == "ipair_dst") take(rt->ipair_dst.data(), 2 * rt->ipair_dst.size());
    else if (k == "ipair_cap") take(rt->ipair_cap.data(), 4 * rt->ipair_cap.size());
    else if (k == "bucket_cap") take(rt->bucket_cap.data(), 8 * rt->bucket_cap.size());
    else if (k == "inbox_cap") take(rt->inbox_cap.data(), 8 * rt->inbox_cap.size());
    else if (k == "perm_inv") take(rt->perm_inv.data(), 4 * rt->perm_inv.size());
    else if (k == "perm_fwd") take(rt->perm_fwd.data(), 4 * rt->perm_fwd.size());
    else if (k == "src_part") take(rt->src_part.data(), 2 * rt->src_part.size());
    else if (k == "pbase") take(rt->pbase.data(), 8 * rt->pbase.size());
    else if (k == "v0") take(rt->v0.data(), 4 * rt->v0.size());
    else if (k == "vn_of_part") take(rt->vn_of_part.data(), 4 * rt->vn_of_part.size());
    else if (k == "relay") take(rt->relay.data(), 4 * rt->relay.size());
    else return SNN_E_ARG;
    if (bytes) *bytes = n;
    if (!out) return SNN_OK;
    if (cap < n) return SNN_E_NOMEM;
    if (n) std::memcpy(out, src, n);
    return SNN_OK;
}

extern "C" void snn_routing_destroy(snn_routing *rt)
{
    delete rt;
}
