// Internal structures shared by the host routing build (snn_host.cpp) and
// the device simulation (snn_sim.cu).  Not part of the public ABI.
#pragma once

#include <atomic>
#include <cstdint>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/snn.h"

namespace snn {

// Packed synapse target word: internal target index (28 bits) | (delay-1) << 28.
constexpr uint32_t kTgtBits = 28;
constexpr uint32_t kTgtMask = (1u << kTgtBits) - 1u;
constexpr int kMaxDelay = 16;
// Level-2 inbox entry: synapse offset << 24 | segment length.
constexpr int kLenBits = 24;
constexpr uint64_t kLenMask = (1ull << kLenBits) - 1ull;
// Delivery work: segments of up to kShortSeg synapses are walked by one
// lane; longer segments are cut into pieces of kPiece synapses, one warp each.
constexpr uint32_t kShortSeg = 8;
constexpr uint32_t kPiece = 128;

// Level-2 entry classes (message accounting of the two-level route).
enum : uint8_t {
    kClsLocal = 0,        // destination is the source partition
    kClsPeer = 1,         // other partition of the source's VN: direct message
    kClsRelayLocal = 2,   // destination VN != source VN, destination is the relay
    kClsRelayRemote = 3,  // destination VN != source VN, forwarded by the relay
};

// One (neuron, destination partition) entry of the level-2 table.  The
// segment's synapses are ordered by delay, so the ones of delay 1 (the only
// ones the next step reads) come first.
constexpr int kOffBits = 40;  // E < 2^40
constexpr uint64_t kOffMask = (1ull << kOffBits) - 1ull;
struct L2Entry {
    uint64_t off;   // bits 0-39: first synapse of the segment in the internal CSR;
                    // bits 40-63: synapses of delay 1 at the segment's start
    uint32_t len;   // synapses in the segment
    uint16_t q;     // internal destination partition
    uint8_t cls;    // kCls*
    uint8_t pad;
};
static_assert(sizeof(L2Entry) == 16, "L2Entry layout");

template <class T>
struct HostArray {
    std::unique_ptr<T[]> p;
    int64_t n = 0;
    void alloc(int64_t count) {
        p.reset(count > 0 ? new T[(size_t)count] : nullptr);
        n = count;
    }
    T *data() { return p.get(); }
    const T *data() const { return p.get(); }
    T &operator[](int64_t i) { return p[(size_t)i]; }
    const T &operator[](int64_t i) const { return p[(size_t)i]; }
};

}  // namespace snn

struct snn_routing {
    int64_t M = 0, E = 0;
    int32_t P = 0, n_vn = 0, vn_size = 0, max_delay = 1;
    bool identity = true;
    unsigned __int128 group_cost = 0;

    std::vector<int32_t> vn_of_part;  // label -> VN
    std::vector<int32_t> ip_of_part;  // label -> internal partition
    std::vector<int32_t> part_of_ip;  // internal partition -> label
    std::vector<int32_t> relay;       // [g*n_vn + h] -> label (per-VN relay policy; -1 otherwise)
    std::vector<int32_t> relay_ip;    // [g*P + ip] relay (internal partition) of VN g for source ip
    int32_t relay_policy = 0;         // SNN_RELAY_*
    std::vector<int64_t> pbase;       // [P+1] first internal neuron of each internal partition
    std::vector<uint32_t> perm_inv;   // internal -> global
    std::vector<uint32_t> perm_fwd;   // global -> internal
    std::vector<int32_t> conn_direct, conn_two;  // per label

    // device-layout tables, host copies (internal order)
    snn::HostArray<uint32_t> syn_td;   // [E]
    snn::HostArray<int16_t> syn_w;     // [E]
    snn::HostArray<uint32_t> l1_ptr;   // [M+1]
    snn::HostArray<uint16_t> l1_vn;    // [n_l1]
    snn::HostArray<uint32_t> l1_l2;    // [n_l1+1]
    snn::HostArray<snn::L2Entry> l2;   // [n_l2]
    std::vector<uint64_t> bucket_cap;  // [n_vn] exact worst case
    std::vector<uint64_t> inbox_cap;   // [P] (internal partitions)
    // Exchange pairs: (internal source partition p, destination VN g) of
    // level 1 and (p, destination partition q) of level 2 that carry at least
    // one entry, numbered by p then destination, each with its exact worst
    // case (every neuron of p spiking).
    std::vector<uint32_t> bpair_ptr;      // [P+1] level-1 pairs of p
    std::vector<uint16_t> bpair_dst;      // [n_bpair] g
    std::vector<uint32_t> bpair_cap;      // [n_bpair]
    std::vector<uint32_t> ipair_ptr;      // [P+1] level-2 pairs of p
    std::vector<uint16_t> ipair_dst;      // [n_ipair] q
    std::vector<uint32_t> ipair_cap;      // [n_ipair]
    snn::HostArray<uint32_t> l1_pair;     // [n_l1] level-1 pair of each entry
    snn::HostArray<uint32_t> l2_pair;     // [n_l2] level-2 pair of each entry
    std::vector<float> v0;             // [M] internal order
    std::vector<int64_t> csr;          // [M+1] first synapse of each internal neuron
    std::vector<uint16_t> src_part;    // [M] internal partition of each internal neuron
    int64_t n_l1 = 0, n_l2 = 0;
    // Delivery by arrival step, from the level-2 entries (computed once, on
    // first use): the longest segment; segments holding a synapse of delay
    // >= 2; the sum over segments of min(max_delay - 1, synapses of delay >= 2)
    // (-1: not computed yet).
    mutable std::atomic<int64_t> seg_maxlen{-1}, seg_delayed{-1}, seg_runs{-1};
    // Partition-owned delivery, per internal destination partition q: the
    // segments into q and the sum over them of min(max_delay, length)
    // (computed once, on first use).
    mutable std::once_flag own_once;
    mutable std::vector<int64_t> own_segs, own_runs;
};

namespace snn {
// Rank of the relay of destination VN g for source VN h under the per-VN
// relay policy: (h - g) mod s, which depends only on the VNs' distance, so
// networks concatenated into a batch get each its own relays.
#if defined(__CUDACC__)
#define SNN_HOST_DEVICE __host__ __device__
#else
#define SNN_HOST_DEVICE
#endif
SNN_HOST_DEVICE inline int32_t vn_rank(int32_t h, int32_t g, int32_t s)
{
    const int32_t r = (h - g) % s;
    return r < 0 ? r + s : r;
}

// Run f(lo, hi) over [0, n) split into contiguous chunks on up to nthreads threads.
void parallel_for(int64_t n, int nthreads, const std::function<void(int64_t, int64_t, int)> &f);
int resolve_threads(int requested);

// Steps of the routing build shared by the host and device builders
// (snn_host.cpp): Algorithm 2 grouping from the inter-partition synapse
// counts PG[p*P+q] (label order) and partition weights WG; the internal
// partition and neuron order, relay map, initial state and source
// partitions; the static connections from the connection matrix
// conn[ip*P+q] (internal order); the exchange-pair numbering from the dense
// worst cases bc[ip*n_vn+g] and ic[ip*P+q], which become pair ids.
void route_groups(snn_routing *rt, const snn_routing_params *prm, const std::vector<int64_t> &PG,
                  const std::vector<int64_t> &WG);
void route_order(snn_routing *rt, const snn_network *net, const int32_t *part_of, const std::vector<int64_t> &sizes);
void route_connections(snn_routing *rt, const std::vector<uint8_t> &conn);
void route_number_pairs(snn_routing *rt, std::vector<uint32_t> &bc, std::vector<uint32_t> &ic);
// Relays of a relay policy (SNN_RELAY_*): relay_ip[g*P + ip] = the internal
// partition of VN g relaying source ip's traffic (-1 for ip in g); the
// balanced policy weighs the level-2 pair worst cases (after
// route_number_pairs).  route_relays sets the routing's own map and the
// relay classes of its level-2 entries under it.
void route_relay_map(const snn_routing *rt, int32_t policy, std::vector<int32_t> &relay_ip);
void route_relays(snn_routing *rt, int32_t policy, int nthreads);
uint32_t philox_word0(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2);
}  // namespace snn
