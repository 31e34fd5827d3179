/*
 * snn.h — C ABI of the GB300 partitioned spiking-network step library
 * (libsnn.so).
 *
 * The calls follow the paper's statement of the problem (arXiv 2205.07125,
 * Sec. I and Sec. IV): a network is generated, its neurons are mapped to
 * partitions (Algorithm 1, Sec. IV.A), the partitions are grouped and a
 * two-level routing table is built (Algorithm 2, Sec. IV.B), and the
 * simulation then alternates computation with spike exchange.  Here all
 * partitions ("GPUs" in the paper) live on one GPU: the spike exchange of
 * the two-level route becomes level-1 buckets per destination group
 * ("virtual node", VN) and level-2 relay expansion into per-partition
 * inboxes, all in device memory.
 *
 * Conventions
 *   - Every call returns int: SNN_OK (0) or a negative SNN_E_* code;
 *     snn_strerror() names it.  No call aborts the process.
 *   - Host arrays passed in are borrowed for the duration of the call
 *     unless a call says otherwise; output arrays are caller-owned with an
 *     explicit capacity.
 *   - Opaque handles are owned by the library and freed by the matching
 *     *_destroy call (which accepts NULL).
 *   - Device memory comes only from the caller: snn_sim_create carves a
 *     caller-allocated device workspace; the library never calls
 *     cudaMalloc for simulation state.  Work is issued asynchronously on the
 *     caller's CUDA stream.
 *   - Neuron ids are the caller's global ids 0..M-1 in every input and
 *     output; the internal partition-major order is never exposed.
 */
#ifndef SNN_H
#define SNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- errors */
#define SNN_OK          0
#define SNN_E_ARG      -1   /* invalid argument or inconsistent sizes */
#define SNN_E_NOMEM    -2   /* host allocation failed / workspace too small */
#define SNN_E_CAPACITY -3   /* a device bucket, inbox or record buffer overflowed */
#define SNN_E_CUDA     -4   /* a CUDA runtime call failed */
#define SNN_E_RANGE    -5   /* network exceeds a layout limit (ids, delays, lengths) */
#define SNN_E_STATE    -6   /* call not valid in the object's current state */
#define SNN_E_NODEV    -7   /* no usable CUDA device */
#define SNN_E_TIMEOUT  -8   /* a bounded device-side wait gave up; the sim state is inconsistent */

const char *snn_strerror(int code);

/* ---------------------------------------------------------------- network */
/*
 * A network as a source-major synapse list (host memory, borrowed):
 * neuron i owns synapses syn_ptr[i] .. syn_ptr[i+1]-1, each with a global
 * target id, an int16 fixed-point weight (units of 2^-10 mV) and a delay in
 * steps (1..16).  v0 holds the initial membrane potentials (mV).
 * Limits: M < 2^28 neurons, out-degree < 2^24 per neuron.
 */
typedef struct {
    int64_t n_neurons;
    const int64_t *syn_ptr;   /* [M+1], syn_ptr[0] == 0, nondecreasing */
    const uint32_t *syn_tgt;  /* [E] */
    const int16_t *syn_w;     /* [E] */
    const uint8_t *syn_d;     /* [E] */
    const float *v0;          /* [M] */
} snn_network;

/* ------------------------------------------------------------------ model */
/*
 * The first setup stage of the paper's statement of the problem (Sec. I:
 * a simulation model is generated, then dispersed over the GPUs; the
 * partitioning and routing of Sec. IV take it as input).  The paper's model
 * is a scanned human brain, which is not available; snn_model_build makes a
 * seeded synthetic LIF network in its place:
 *   - M neurons in n_parts planted partitions of contiguous ids (partition p
 *     holds ids floor(pM/P) .. floor((p+1)M/P)-1), planted VNs = runs of
 *     vn_size partitions; the first round(frac_exc * size) ids of each
 *     planted partition are excitatory;
 *   - exactly syn_per_neuron out-synapses per neuron, drawn with replacement,
 *     no autapses: uniform over all other neurons (uniform = 1), or
 *     n_same_part in the own partition, n_same_vn in the other partitions of
 *     the own VN and n_remote outside it;
 *   - int16 weights in units of 2^-10 mV: excitatory lround(mu_e + sd_e z)
 *     clamped to [1, 32767], inhibitory -lround(mu_i + sd_i z) clamped to
 *     [-32768, -1], z = (sum of 12 uniforms) - 6 computed exactly in double;
 *   - delays uniform in 1..max_delay steps; V0 = v_reset + u (v_th - v_reset);
 *   - randomness: splitmix64 seeded per neuron from `seed`, so the network
 *     has the same bits for any thread count and on any host.
 * The model owns its arrays; snn_model_network gives a borrowed
 * snn_network view of them (valid until snn_model_destroy) for
 * snn_partition, snn_routing_build and snn_sim_create.
 */
typedef struct {
    int64_t n_neurons;
    int32_t n_parts, vn_size;
    int32_t syn_per_neuron;
    int32_t uniform;                             /* 1: targets uniform over all other neurons */
    int32_t n_same_part, n_same_vn, n_remote;    /* locality mix (sum = syn_per_neuron) */
    int32_t max_delay;                           /* 1..16 */
    uint64_t seed;
    double v_reset, v_th;                        /* range of the initial potentials (mV) */
    double frac_exc, mu_e, sd_e, mu_i, sd_i;
} snn_model_params;

typedef struct snn_model snn_model;

/* Workloads: 4,096 neurons / 4 partitions / 100 uniform synapses, delay 1;
 * 1,048,576 / 64 partitions in VNs of 4 / 1,000 synapses (70/20/10 locality,
 * delays 1-8); the per-GPU share of the paper's 10-billion-neuron run on
 * 2,000 GPUs (Sec. V): 5,000,000 / 256 partitions in VNs of 4 / 1,000
 * synapses; the adjoint network: 131,072 / 8 partitions in VNs of 4 / 500
 * synapses (the same mix). */
#define SNN_WORKLOAD_TINY        0
#define SNN_WORKLOAD_SCALE       1
#define SNN_WORKLOAD_PAPER_SHARE 2
#define SNN_WORKLOAD_ADJOINT     4
/* Fill p with a workload's recipe.  Errors: SNN_E_ARG (unknown workload). */
int snn_model_params_preset(int32_t workload, snn_model_params *p);
/* Generate the network (host, all cores).  Errors: SNN_E_ARG (invalid
 * parameters: M < 2 or >= 2^28, a mix that does not sum to syn_per_neuron,
 * n_parts not a multiple of vn_size, E >= 2^40), SNN_E_NOMEM. */
int snn_model_build(const snn_model_params *params, snn_model **out);
/* Borrowed view of the model's arrays; is_exc (may be NULL) receives the
 * [M] excitatory flags (snn_adjoint_create takes them).  Errors: SNN_E_ARG. */
int snn_model_network(const snn_model *model, snn_network *net, const uint8_t **is_exc);
/*
 * Write the model as an edge-list file: 8 magic bytes "SNNMODL1", then
 * little-endian u64 M, u64 E, u32 max_delay, u32 0, then syn_ptr i64[M+1],
 * syn_tgt u32[E], syn_w i16[E], syn_d u8[E], v0 f32[M], is_exc u8[M]
 * (source-major: neuron i's synapses are syn_ptr[i] .. syn_ptr[i+1]-1).
 * Errors: SNN_E_ARG (NULL arguments, the file cannot be written).
 */
int snn_model_save(const snn_model *model, const char *path);
/* Read a file written by snn_model_save, checking that the synapse list is
 * well formed (offsets, target ids < M, delays within 1..max_delay).
 * Errors: SNN_E_ARG (unreadable or malformed file), SNN_E_NOMEM. */
int snn_model_load(const char *path, snn_model **out);
void snn_model_destroy(snn_model *model);

/* -------------------------------------------------------------- partition */
#define SNN_PART_PLANTED 0   /* contiguous id ranges: part(i) = p, floor(pM/P) <= i < floor((p+1)M/P) */
#define SNN_PART_GREEDY  1   /* Algorithm 1 (greedy growth, best of `iters`) */
#define SNN_PART_RANDOM  2   /* balanced random mapping (the paper's baseline) */

typedef struct {
    int32_t mode;      /* SNN_PART_* */
    int32_t iters;     /* Algorithm 1 iterations T (>= 1) */
    uint64_t seed;     /* seed of the random choices */
} snn_partition_params;

typedef struct {
    int64_t objective;    /* sum over cut synapses i->j of W_i*W_j, W = out-degree */
    int64_t min_weight;   /* smallest / largest per-part sum of W */
    int64_t max_weight;
} snn_partition_stats;

/*
 * Map neurons to n_parts partitions (Algorithm 1, Sec. IV.A).  Greedy
 * reading: for t = 1..iters, parts 0..P-2 are grown one at a time from a
 * seed (t = 1: lowest unassigned id; t > 1: a Philox4x32-10-chosen
 * unassigned neuron, counter (t, k, 0xA1, 0), key = seed), adding the
 * unassigned neuron with the largest sum_{i in part} (c_ij + c_ji) W_i W_j
 * (ties: lowest id) while the part's weight is below sum(W)/P; the last part
 * takes the rest; the mapping with the smallest objective is kept.
 * part_of: caller-owned [M], receives partition labels.  stats may be NULL.
 * Errors: SNN_E_ARG (bad sizes), SNN_E_NOMEM.
 */
int snn_partition(const snn_network *net, int32_t n_parts, const snn_partition_params *params,
                  int32_t *part_of, snn_partition_stats *stats);

/*
 * Algorithm 1 on the GPU with batched growth (the parallel form of the
 * greedy that the paper names as future work, Sec. VII).  Seeds, stopping
 * rule, last part, iterations and objective are those of snn_partition's
 * greedy; a part grows in rounds: the `need` unassigned neurons with the
 * largest gains (ties: lowest id) are ranked on the gains at the start of
 * the round and join the part one at a time in that order until its weight
 * reaches sum(W)/P; the gains of the round's members are added before the
 * next round.  need = min(batch, unassigned, max(1, n_k / grow)) with n_k the
 * part's size so far (grow = 0 drops the last term).  batch = 1 gives the
 * sequential greedy of snn_partition bit for bit; every batch gives the same
 * mapping on every run (integer gains, order-free sums).
 */
typedef struct {
    int32_t iters;     /* Algorithm 1 iterations T (>= 1) */
    int32_t batch;     /* largest round, 1 .. 2048 */
    int32_t grow;      /* round <= max(1, n_k / grow) while the part is small; 0: off */
    int32_t reserved;
    uint64_t seed;     /* seed of the t > 1 starting neurons (as snn_partition) */
} snn_partition_device_params;

/* Defaults: iters 4, batch 2048, grow 2, seed 7. */
void snn_partition_device_params_default(snn_partition_device_params *p);
/* Device workspace for a network of M neurons and E synapses: 8E + ~44M
 * bytes (out- and in-synapse lists, per-neuron state of the growth). */
int snn_partition_device_workspace_bytes(const snn_network *net, int32_t n_parts, size_t *bytes);
/*
 * workspace: caller-owned device memory of at least the bytes above,
 * 256-byte aligned; stream: the caller's cudaStream_t (the call copies the
 * synapse lists in, runs on the stream and synchronises it before
 * returning).  part_of: caller-owned host [M], receives the labels of the
 * iteration with the smallest objective (the first one on ties).  stats may
 * be NULL.  Errors: SNN_E_ARG (bad sizes or parameters, a target id >= M),
 * SNN_E_NOMEM (workspace too small or misaligned), SNN_E_RANGE (M >= 2^28,
 * or the largest possible gain and the id need more than 64 key bits),
 * SNN_E_NODEV (no cooperative launch), SNN_E_CUDA, SNN_E_TIMEOUT (a bounded
 * grid-barrier wait ran out; part_of is not written), SNN_E_STATE (a
 * device-side consistency check failed: a round of the wrong size or no
 * seed; the kernel skips the access and ends; part_of is not written).
 */
int snn_partition_device(const snn_network *net, int32_t n_parts, const snn_partition_device_params *params,
                         void *workspace, size_t workspace_bytes, void *stream, int32_t *part_of,
                         snn_partition_stats *stats);

/* ---------------------------------------------------------------- routing */
#define SNN_GROUP_CONTIGUOUS 0  /* VN g = partitions g*s .. g*s+s-1, s = P/n_vn */
#define SNN_GROUP_GREEDY     1  /* Algorithm 2 grouping (best of `iters`) */

/*
 * Relay ("bridge") of destination VN g for a source partition p in another
 * VN (paper Sec. IV.B: traffic to another group goes through one bridge;
 * which member of g relays whose traffic is the design choice behind the
 * peak level-2 traffic of Sec. V, Fig. 3(b)).  Members of a VN are ranked
 * by ascending partition label.
 *   PER_VN (default): member ((vn(p) - g) mod s) of g, one relay per pair of
 *     VNs (it depends on the VNs' distance only, so each network of a batch
 *     gets the relays it has alone);
 *   PER_PARTITION: member (rank of p in its own VN, mod s) of g, which
 *     spreads the s partitions of a VN over the s members of g;
 *   BALANCED: per g, the sources p in decreasing static load (ties: lower
 *     label) each go to the member of g with the least load so far (ties:
 *     lower rank) -- longest-processing-time first -- where the static
 *     load of (g, p) is the number of (neuron of p, partition of g) pairs
 *     with synapses, the level-2 entries p sends into g; sources of load 0
 *     take the PER_PARTITION member.
 * The relay decides only which level-2 entries the relay forwards (message
 * accounting and connections); delivery and results are the same.
 */
#define SNN_RELAY_PER_VN        0
#define SNN_RELAY_PER_PARTITION 1
#define SNN_RELAY_BALANCED      2

typedef struct {
    int32_t grouping;   /* SNN_GROUP_* */
    int32_t iters;      /* Algorithm 2 iterations T (>= 1) */
    uint64_t seed;      /* seed of the random choices */
    int32_t n_threads;  /* host threads for the build (0 = all) */
    int32_t relay;      /* SNN_RELAY_* */
} snn_routing_params;

typedef struct {
    int64_t n_neurons, n_synapses;
    int32_t n_parts, n_vn, vn_size, max_delay;
    int64_t n_l1;              /* (neuron, destination VN) entries */
    int64_t n_l2;              /* (neuron, destination partition) entries */
    uint64_t group_cost_lo;    /* Algorithm 2 objective: sum over inter-group */
    uint64_t group_cost_hi;    /*   partition pairs of PG[p][q]*WG[p]*WG[q] (128 bit) */
    int64_t conn_direct_sum;   /* static outgoing connections summed over partitions: */
    int64_t conn_two_level_sum;/*   direct route vs two-level route (Sec. V, Fig. 4) */
    int32_t conn_direct_max;
    int32_t conn_two_level_max;
    int32_t identity_order;    /* 1 if the internal neuron order equals the global order */
    int32_t reserved;
} snn_routing_info;

typedef struct snn_routing snn_routing;

/*
 * Group partitions into n_vn virtual nodes of equal size (Algorithm 2,
 * Sec. IV.B) and build the two-level routing table and the device layout:
 *   - level 1: per source neuron, the destination VNs holding its targets
 *     (one message per VN, deduplicated);
 *   - level 2: per (neuron, VN), the destination partitions of that VN
 *     with the neuron's synapse segment for each;
 *   - relay ("bridge") of destination VN g for a source partition of
 *     another VN: by relay policy (snn_routing_params.relay, below); inside
 *     the own VN the source partition sends directly.
 * Greedy grouping reading: for t = 1..iters, groups 0..n_vn-2 are grown
 * from a seed (t = 1: heaviest ungrouped partition by WG, ties lowest label;
 * t > 1: Philox-chosen, counter (t, g, 0xA2, 0)) by adding the ungrouped q
 * with the largest sum_{m in g} (PG[m][q] + PG[q][m]) WG[m] WG[q] (ties:
 * lowest q), PG = inter-partition synapse counts, WG = summed out-degree.
 * part_of: [M] labels 0..n_parts-1 (each partition non-empty);
 * n_parts % n_vn == 0.  The network arrays are read during the call only.
 * Errors: SNN_E_ARG, SNN_E_RANGE (delay outside 1..16, M >= 2^28,
 * out-degree >= 2^24), SNN_E_NOMEM.
 */
int snn_routing_build(const snn_network *net, const int32_t *part_of, int32_t n_parts,
                      int32_t n_vn, const snn_routing_params *params, snn_routing **out);
int snn_routing_info_get(const snn_routing *rt, snn_routing_info *out);
/* vn_of_part: caller-owned [n_parts]; relay: caller-owned [n_vn*n_vn],
 * relay[g*n_vn + h] = partition label relaying VN h's traffic inside VN g
 * (SNN_RELAY_PER_VN; -1 under the other policies, see snn_routing_relays). */
int snn_routing_groups(const snn_routing *rt, int32_t *vn_of_part, int32_t *relay);
/* relay: caller-owned [n_vn*n_parts], relay[g*n_parts + p] = partition label
 * relaying the traffic of source partition p (label) inside VN g, or -1 for
 * p in g.  policy: SNN_RELAY_* to compute that policy's map for this
 * routing, or -1 for the routing's own.  Errors: SNN_E_ARG. */
int snn_routing_relays(const snn_routing *rt, int32_t policy, int32_t *relay);
/* Per-partition static connection counts (caller-owned [n_parts] each). */
int snn_routing_connections(const snn_routing *rt, int32_t *direct, int32_t *two_level);
/*
 * Messages per partition that a multiset of spikes causes, on the direct
 * route and on the two-level route (the per-GPU traffic whose peak the
 * paper compares, Sec. V, Fig. 3).  A message is one (spike, destination)
 * pair.  Direct route: a spike of partition p sends one message to every
 * partition q != p holding targets of it.  Two-level route: p sends one
 * message to each own-VN peer holding targets and one to the relay of each
 * other VN holding targets (level 1); the relay forwards one to every other
 * partition of its VN holding targets (level 2), counted as the relay's
 * traffic.  ids: host uint32 [n] global spike ids (repeats count again,
 * e.g. a raster over many steps).  relay_policy: SNN_RELAY_* (the relays of
 * that policy on this routing's groups), or -1 for the routing's own.  Outputs (caller-owned [n_parts], label
 * order, each may be NULL): messages sent and received per partition on
 * each route.  Errors: SNN_E_ARG (NULL arrays with n > 0, an id >= M).
 */
int snn_routing_traffic(const snn_routing *rt, const uint32_t *ids, int64_t n, int32_t relay_policy,
                        int64_t *direct_out, int64_t *direct_in, int64_t *two_level_out, int64_t *two_level_in);
/*
 * Copy one of the routing's tables (host memory, internal order) into the
 * caller's buffer `out` of `cap` bytes; *bytes receives the table's size.
 * With out == NULL only the size is returned.  Names and element types:
 * "syn_td" u32 [E] (internal target | (delay-1) << 28), "syn_w" i16 [E],
 * "csr" i64 [M+1], "l1_ptr" u32 [M+1], "l1_vn" u16 [n_l1], "l1_l2" u32
 * [n_l1+1], "l2" 16-byte entries [n_l2] {u64 offset | delay-1 count << 40,
 * u32 length, u16 partition, u8 class, u8 0}, "l1_pair" u32 [n_l1],
 * "l2_pair" u32 [n_l2], "bpair_ptr" / "ipair_ptr" u32 [P+1], "bpair_dst" /
 * "ipair_dst" u16, "bpair_cap" / "ipair_cap" u32, "bucket_cap" u64 [n_vn],
 * "inbox_cap" u64 [P], "perm_inv" / "perm_fwd" u32 [M], "src_part" u16 [M],
 * "pbase" i64 [P+1], "v0" f32 [M], "vn_of_part" / "relay" i32.
 * Errors: SNN_E_ARG (unknown name), SNN_E_NOMEM (cap too small).
 */
int snn_routing_export(const snn_routing *rt, const char *name, void *out, size_t cap, size_t *bytes);

/*
 * The same routing built on the GPU (the table building of the parallel
 * design the paper names as future work, Sec. VII): the synapse scans
 * (inter-partition counts, per-neuron segment and VN counts, exchange-pair
 * worst cases) and the per-neuron sort of the synapses by (destination
 * partition, delay, target, weight) with the level-1 / level-2 entries run
 * on the device; grouping (Algorithm 2), orders and pair numbering on the
 * host.  The tables equal snn_routing_build's byte for byte.  The result is
 * an ordinary routing (host tables, copied back chunk by chunk).
 * workspace: caller-owned device memory of snn_routing_build_device_
 * workspace_bytes, 256-byte aligned; stream: the caller's cudaStream_t (the
 * call synchronises it).  Limits beyond snn_routing_build's: out-degree <=
 * 16384.  Errors: as snn_routing_build, plus SNN_E_NOMEM (workspace), SNN_E_CUDA.
 */
int snn_routing_build_device_workspace_bytes(const snn_network *net, int32_t n_parts, int32_t n_vn, size_t *bytes);
int snn_routing_build_device(const snn_network *net, const int32_t *part_of, int32_t n_parts, int32_t n_vn,
                             const snn_routing_params *params, void *workspace, size_t workspace_bytes,
                             void *stream, snn_routing **out);
void snn_routing_destroy(snn_routing *rt);

/* ------------------------------------------------------------- simulation */
typedef struct {
    /* LIF dynamics.  Update of a non-refractory neuron (FP32, no fused
     * multiply-add, this order): u = V - e_l; V = e_l + alpha*u;
     * V = V + float(I) * 2^-10, alpha = fl32(exp(-dt_ms/tau_ms)); spike if
     * V >= v_th, then V = v_reset and ref = t_ref.  A refractory neuron
     * (ref > 0) is held at v_reset and ref decreases by one. */
    double dt_ms, tau_ms;
    float e_l, v_th, v_reset;
    int32_t t_ref;               /* 0..255 */
    /* input I = recurrent int32 input + k*w_ext + i_bias, k ~ Poisson(lambda)
     * drawn by inverse CDF from word (j mod 4) of the Philox4x32-10 block
     * with key = drive_seed, counter = (j div 4, step, 0, 0), j = global id */
    double drive_lambda;         /* 0..16 */
    int32_t w_ext, i_bias;
    uint64_t drive_seed;
    /* records */
    int64_t raster_cap;          /* spike ids kept for snn_read_raster */
    int64_t raster_steps;        /* steps whose raster offsets are kept */
    int64_t hash_steps;          /* steps whose state hashes are kept */
    int32_t cur_every;           /* snapshot consumed input every k-th step (0 = off) */
    int32_t cur_slots;           /* number of snapshots kept */
    /* capacities of level-1 buckets / level-2 inboxes as a fraction of
     * their exact worst case (every neuron spiking); 1.0 never overflows */
    float bucket_frac, inbox_frac;
    int32_t steps_per_graph;     /* steps unrolled per CUDA graph (1..256) */
    int32_t pin_host_tables;     /* page-lock the routing tables for uploads */
    int32_t defer_delayed;       /* 0/1: minimum-delay batching on the persistent shared-memory shape:
                                  * each step's delay >= 2 synapses are delivered during the next
                                  * step's table walk (exact; slower on GB300 for the scale
                                  * workload, off by default) */
    /* SNN_DELIVER_*: when a spike's synapses reach their targets' input.
     *   RING (default): every delay at the spike's step, into a delay ring
     *     of max_delay + 1 slots of M int32 (the slots a step writes span
     *     the whole ring);
     *   ARRIVAL: each step writes only the next step's input slot: the
     *     delay-1 run of each routed segment at once, the run of delay d >= 2
     *     queued on the list of step t + d - 1 and delivered by that step
     *     (segments are sorted by delay).  Two input slots of M int32 stay
     *     hot in L2 however large the ring would be.  Needs max_delay <= 8
     *     and segments of at most 65535 synapses (else SNN_E_RANGE);
     *   OWNER: every run of a routed segment, of every delay, is queued on
     *     its destination partition's list of its arrival step; at step t
     *     the block that owns a partition adds that partition's runs into a
     *     shared-memory accumulator and updates the partition's neurons
     *     from it, so no global input slot and no global reductions remain
     *     (each partition receives its messages and delivers them into its
     *     own neurons).  Persistent kernel only; needs cooperative launch,
     *     max_delay <= 8, segments of at most 65535 synapses and the
     *     largest partition's accumulator in one block's shared memory
     *     (else SNN_E_RANGE);
     *   AUTO: the workspace holds every available mode; snn_autotune picks
     *     the fastest (until then ARRIVAL when it is available, else RING).
     * Sums are integers, so every mode gives the same results bit for bit. */
    int32_t delivery;
    /* capacity of each arrival list (ARRIVAL and OWNER) as a fraction of its
     * exact worst case (1.0, the default, never overflows; overflow sets
     * SNN_E_CAPACITY) */
    float arrival_frac;
} snn_sim_params;

#define SNN_DELIVER_RING    0
#define SNN_DELIVER_ARRIVAL 1
#define SNN_DELIVER_AUTO    2
#define SNN_DELIVER_OWNER   3

/* Fill p with the defaults (no records, exact capacities, 32 steps/graph). */
void snn_sim_params_default(snn_sim_params *p);

typedef struct {
    uint64_t steps;             /* steps simulated */
    uint64_t spikes;            /* spikes emitted */
    uint64_t events;            /* synaptic events delivered */
    uint64_t direct;            /* direct route: (spike, partition q != own) messages */
    uint64_t direct_xvn;        /*   of which cross a VN boundary */
    uint64_t l1_local;          /* level 1: own-VN bucket entries (no message) */
    uint64_t l1_xvn;            /* level 1: cross-VN messages (one per spike and VN) */
    uint64_t l2_local;          /* level 2: own partition (no message) */
    uint64_t l2_peer;           /* level 2: direct messages to own-VN peers */
    uint64_t l2_relay_local;    /* level 2: relay is itself a destination (no message) */
    uint64_t l2_relay_remote;   /* level 2: relay forwards to another partition */
} snn_counts;

typedef struct snn_sim snn_sim;

/* Device workspace size for a routing and parameters.  Errors: SNN_E_ARG. */
int snn_sim_workspace_bytes(const snn_routing *rt, const snn_sim_params *p, size_t *bytes);

/*
 * Create a simulation: carve `workspace` (device memory of at least
 * snn_sim_workspace_bytes, 256-byte aligned, caller-owned, must outlive the
 * sim), upload the routing tables and the initial state (V = v0, ref = 0,
 * empty delay ring, t = 0) on `stream` (a cudaStream_t, NULL = legacy
 * default stream).  `rt` must outlive the sim.  Uses the current device.
 * Errors: SNN_E_ARG, SNN_E_NOMEM (workspace too small), SNN_E_CUDA, SNN_E_NODEV.
 *
 * Environment variables read here (launch-shape and tuning switches; none
 * changes a result, every combination is bit-exact):
 *   SNN_PERSIST=0               CUDA-graph path instead of the persistent kernel
 *   SNN_PERSIST_SMEM=0          persistent kernel on global neuron state only
 *   SNN_PERSIST_BLOCKS_PER_SM=b at most b (1..4) resident blocks per SM
 *   SNN_PERSIST_DEFER=1         minimum-delay batching, as defer_delayed = 1
 *   SNN_DELIVERY=0..3           overrides snn_sim_params.delivery
 *   SNN_PDL=0                   graph kernels in plain stream order (no
 *                               programmatic dependent launch)
 *   SNN_BAR_GROUPS=G            two-level grid-barrier arrival over G (2..16)
 *                               group words (default: one word)
 *   SNN_PREFETCH_STATE=0        no L2 prefetch of the next step's neuron state
 *                               (global-state persistent kernel)
 *   SNN_ASYNC_RECORDS=0         queued runs delivered with plain loads instead
 *                               of asynchronous copies into shared memory
 *   SNN_VEC_PIECES=1            staged pieces delivered with 16- / 8-byte loads
 *   SNN_BARRIER_LIMIT_NS=n      bound of each grid-barrier wait (default 1 s);
 *                               one that runs out is reported by
 *                               snn_sync_status as SNN_E_TIMEOUT
 *   SNN_TEST_SKIP_BARRIER=1     tests only: block 0 skips its first arrival,
 *                               so the others' bounded wait runs out
 */
int snn_sim_create(const snn_network *net, const snn_routing *rt, const snn_sim_params *p,
                   void *workspace, size_t workspace_bytes, void *stream, snn_sim **out);

/*
 * Batches (no counterpart in the paper, which simulates one network):
 * n independent networks of any sizes stepped together by one sim, so one
 * snn_step runs all of them in one persistent launch (or one graph).
 * The caller concatenates the networks into `net`: network k owns ids
 * [off[k], off[k+1]) (off[0] = 0, off[n] = M, every off[k] a multiple of 4,
 * n <= 65535) and no synapse leaves its network; the partition vector gives
 * each network its own partitions and the routing is built once on the
 * concatenation, with every VN inside one network (contiguous grouping and a
 * multiple of the VN size partitions per network).  params[k] gives network
 * k its drive (drive_lambda, drive_seed: the Philox stream of network k counts
 * its own ids from 0); all other fields come from params[0].  Routing,
 * delivery and records are those of the concatenation: network k's spikes
 * are the raster ids in [off[k], off[k+1]), the counts are sums over the
 * networks.  `off` and `params` are copied.
 * Errors: SNN_E_ARG (a check above fails, M % 4 != 0), plus those of
 * snn_sim_create.
 */
int snn_batch_workspace_bytes(const snn_routing *rt, int32_t n, const snn_sim_params *params, size_t *bytes);
int snn_batch_create(const snn_network *net, const snn_routing *rt, int32_t n, const int64_t *off,
                     const snn_sim_params *params, void *workspace, size_t workspace_bytes, void *stream,
                     snn_sim **out);

/*
 * Advance T steps: the paper's simulation loop, in which every step is the
 * GPUs' computation followed by the spike exchange between them (Sec. I,
 * Sec. III), with the exchange taking the two-level route (Sec. IV.B): a
 * spike goes once to each destination group (level 1) and is forwarded
 * inside that group to the partitions that hold its targets (level 2).  The
 * neuron model is LIF, the one the paper lists for its simulators (Table I).
 * Each step: (a1) consume the step's input (delay-ring slot, or input slot
 * with SNN_DELIVER_ARRIVAL), add the
 * Poisson drive; (a2) LIF update and threshold; (a3) warp-ballot/prefix-sum
 * spike compaction; (a4) level-1 bucketing by destination VN; (a5) level-2
 * relay expansion into per-partition inboxes; (a6) CSR fan-out of int16
 * weights into int32 accumulators.  Asynchronous on the sim's stream.
 * A step runs in two halves: a1-a3 over the neurons into the step's spike
 * list, then a4-a6 over equal shares of that list (a step's deliveries
 * write only the ring slots of later steps).  On a GPU with cooperative
 * launch the T steps run in one persistent kernel (every block resident, a
 * grid barrier after each half, each barrier wait bounded by one second);
 * otherwise, or with the environment variable SNN_PERSIST=0 at
 * snn_sim_create, as replays of captured CUDA graphs of two kernels per
 * step.  Both give the same results bit for bit.
 * Errors raised on the device are reported by snn_sync_status.
 * Errors: SNN_E_ARG, SNN_E_CUDA.
 */
int snn_step(snn_sim *sim, int32_t T);

/* Wait for the sim's stream and return the device status:
 * SNN_OK, SNN_E_CAPACITY (bucket/inbox overflow; the affected steps are
 * wrong, the raster overflow alone is reported by snn_read_raster),
 * SNN_E_TIMEOUT (a grid barrier of the persistent step kernel waited past its
 * one-second bound and the run stopped), or SNN_E_CUDA. */
int snn_sync_status(snn_sim *sim);

/*
 * Read-outs of a simulation (the spikes, inputs, message counts and state
 * the paper's evaluation is made of, Sec. V: the messages of each route and
 * their traffic).
 * Spikes of steps t0 .. t1-1 (global ids, ascending within a step):
 * ids[step_off[k] .. step_off[k+1]) for step t0+k; step_off has t1-t0+1
 * entries; *n receives the total.  Synchronises the stream.
 * Errors: SNN_E_ARG; SNN_E_CAPACITY with *n = -1 when a step was not
 * recorded, with *n = the total when it exceeds cap (ids may be NULL then).
 */
int snn_read_raster(snn_sim *sim, int64_t t0, int64_t t1, uint32_t *ids, int64_t cap,
                    int64_t *step_off, int64_t *n);
/* Recurrent int32 input consumed at step t (global order, [M]); t must be a
 * snapshot step (t % cur_every == 0, t / cur_every < cur_slots). */
int snn_read_currents(snn_sim *sim, int64_t t, int32_t *out);
/* Order-free hashes of steps t0..t1-1: cur = sum_j mix(j<<32 | I_rec_j),
 * v = sum_j mix(j<<32 | bits(V_j)) mod 2^64 over global ids j, mix the
 * splitmix64 finaliser. */
int snn_read_hashes(snn_sim *sim, int64_t t0, int64_t t1, uint64_t *cur, uint64_t *v);
/* Counters since the start (or the last reset/restore): spikes, synaptic
 * events, and the messages of the direct route and of the two-level route by
 * kind (Sec. IV.B: level-1 messages to other groups, direct messages inside
 * the group, level-2 forwards by the relay; the comparison of Sec. V,
 * Fig. 3).  With SNN_DELIVER_ARRIVAL the events are counted when routed. */
int snn_read_counts(snn_sim *sim, snn_counts *out);
/* Current state in global order: V [M], ref [M]; *t = next step index. */
int snn_read_state(snn_sim *sim, float *V, uint8_t *ref, int64_t *t);
/* (spike id << 32 | destination partition label) pairs held in the
 * level-2 inboxes after the last step, unsorted; *n = total (may exceed cap):
 * the spikes each partition received over the two-level route (Sec. IV.B),
 * which must be the pairs of the direct route. */
int snn_read_inbox_pairs(snn_sim *sim, uint64_t *pairs, int64_t cap, int64_t *n);

/* Checkpoint: V, ref, delay ring, step index, counters (bytes from
 * snn_state_bytes).  Restoring continues bit-exactly (the drive is
 * counter-based).  Records are not part of the checkpoint: after a restore
 * the raster stays off and the hash slots from the restored step on are
 * cleared. */
int snn_state_bytes(snn_sim *sim, size_t *bytes);
int snn_save_state(snn_sim *sim, void *host_buf, size_t cap);
int snn_load_state(snn_sim *sim, const void *host_buf, size_t bytes);

/* Return to the initial state and clear counters and records; with
 * reupload != 0 the routing tables are copied to the device again. */
int snn_sim_reset(snn_sim *sim, int32_t reupload);

/*
 * Launch-shape autotuner (no counterpart in the paper): time `steps` steps
 * (after steps/4 warm-up steps) of every shape this GPU can run -- the
 * persistent kernel with 4, 3, 2 or 1 blocks per SM and the neuron state in
 * shared memory, in global memory with 16-byte accesses or one neuron per
 * thread, the CUDA-graph path, each with delivery into the delay ring and
 * (workspace of SNN_DELIVER_AUTO) by arrival step, and the partition-owned
 * kernel -- each from the sim's current state, and keep the fastest (shapes
 * excluded by SNN_PERSIST=0 / SNN_PERSIST_SMEM=0 at creation are not
 * tried).  Every shape gives the same results bit for bit.  The exchange
 * capacities need no tuning: they are the exact worst case of the routing
 * tables.  Leaves the sim in the state it had (records included), so it can
 * be called after a pre-roll into the regime that is to be timed.
 * choice (may be NULL): 0 = graph path, else 100 * mode + blocks per SM
 * (mode 2 shared-memory state, 1 global 16-byte, 0 global one neuron per
 * thread), + 1000 with delivery by arrival step; 2000 + blocks per SM for
 * the partition-owned kernel; best_ms (may be NULL): the chosen shape's time
 * per step.  Synchronises the stream.  Host memory: a copy of the neuron
 * state and the delay ring.
 * Errors: SNN_E_ARG, SNN_E_CUDA.
 */
int snn_autotune(snn_sim *sim, int32_t steps, int32_t *choice, double *best_ms);

/* ---------------------------------------------------------------- adjoint */
/*
 * Surrogate-gradient adjoint (no counterpart in the paper, which simulates
 * but does not train).  The differentiable step keeps the routing and the
 * integer delivery and adds parameters: population-pair gains G[a][b]
 * (n_pop x n_pop, row = target population) and drive rates lam[a] (arrivals
 * per step), populations pop(j) = 2 vn(j) + (1 if j is inhibitory), n_pop =
 * 2 n_vn <= 8.  Forward step (fp32, fixed order, no FMA):
 *   A_jb = int32 sum of the weights from population b arriving at j;
 *   I_j  = (((G[a][0] A_j0 + G[a][1] A_j1) + ...) + w_ext (lam_a + sigma xi_j(t)),
 *   xi_j(t) = (sum of the 12 bytes of words 0..2 of Philox4x32-10(counter
 *   (global id j, t, 0xAD, 0), key = drive_seed) - 1530) / 256;
 *   V_pre = (E_L + alpha (V - E_L)) + I 2^-10, spike V_pre >= V_th, reset and
 *   refractory as the plain step.
 * Rates r_a = (spikes of population a) / (T N_a).  Backward: surrogate
 * dS/dV_pre = 1 / (1 + beta |V_pre - V_th|)^2, reset detached; each neuron
 * gathers its targets' adjoints along its own level-2 entries (the
 * transpose of the routed delivery).  Backward step t gathers the newest
 * adjoint plane only, h(t + 1) = G[pop k][b] * dL/dV_pre of k at t + 1, and
 * adds each synapse's term to a per-step partial sum by its delay; the
 * float32 terms are summed in a fixed order per neuron, so the gradients do
 * not depend on the checkpoint interval.  Gradients are accumulated in
 * float64 (per-warp float pairs first).
 */
typedef struct {
    int32_t T;            /* forward steps per run (>= 1) */
    int32_t ckpt_every;   /* membrane checkpoint interval K: state saved every K steps */
    float sigma;          /* noise scale (0.9) */
    float beta;           /* surrogate slope, 1/mV (5) */
    int64_t reserved[2];
} snn_adjoint_params;

typedef struct snn_adjoint snn_adjoint;

void snn_adjoint_params_default(snn_adjoint_params *ap);
/* Device workspace: state, tables, one recorded segment of K steps and
 * ceil(T/K) checkpoints of (V, ref, delay ring).  Errors: SNN_E_ARG,
 * SNN_E_RANGE (n_pop > 8). */
int snn_adjoint_workspace_bytes(const snn_routing *rt, const snn_sim_params *p, const snn_adjoint_params *ap,
                                size_t *bytes);
/* is_exc: [M] global order (1 excitatory).  p gives the LIF constants,
 * w_ext, drive_seed and raster_cap (spike record of the forward).
 * Workspace and stream as snn_sim_create.  Errors: SNN_E_ARG, SNN_E_NOMEM,
 * SNN_E_CUDA, SNN_E_NODEV, SNN_E_STATE (a neuron's level-2 entries do not
 * tile its synapse run: routing tables not built by this library). */
int snn_adjoint_create(const snn_network *net, const uint8_t *is_exc, const snn_routing *rt,
                       const snn_sim_params *p, const snn_adjoint_params *ap, void *workspace,
                       size_t workspace_bytes, void *stream, snn_adjoint **out);
/* T steps from the initial state with parameters G [n_pop*n_pop], lam
 * [n_pop] (host); rates [n_pop] (may be NULL), *spikes = total (may be
 * NULL).  Synchronises the stream. */
int snn_adjoint_forward(snn_adjoint *adj, const float *G, const float *lam, float *rates, int64_t *spikes);
/* Gradients of a loss with dL/dr = grates [n_pop] through the last
 * forward: dG [n_pop*n_pop], dlam [n_pop] (host, float64).  Recomputes each
 * K-step segment from its checkpoint.  Errors: SNN_E_STATE (no forward). */
int snn_adjoint_backward(snn_adjoint *adj, const double *grates, double *dG, double *dlam);
/* Spikes of the last forward as (t << 32 | global id), unordered; *n = total. */
int snn_adjoint_read_spikes(snn_adjoint *adj, uint64_t *out, int64_t cap, int64_t *n);
void snn_adjoint_destroy(snn_adjoint *adj);

/* Kernels of one step on the graph path: 2 (a1-a3, a4-a6). */
int64_t snn_launches_per_step(const snn_sim *sim);
/* Kernel launches one snn_step(sim, T) issues: 1 on the persistent path,
 * 2 per step plus one per replayed graph on the graph path. */
int64_t snn_launches(const snn_sim *sim, int32_t T);

/*
 * Advance T steps like snn_step and return, in milliseconds summed over the
 * steps, the time of the parts of a step (phase_ms: caller-owned [7]).
 * Persistent path, as seen by block 0 (GPU global timer): [0] the neurons'
 * update (a1-a2), [1] the spike compaction (a3), [2] the prefetch of its own
 * spikes' tables and its share of the runs queued for the step (delivery by
 * arrival step), [3] the rest of the wait at the first grid barrier, [4] the
 * routing walk (a4-a5), [5] the routing rounds' deliveries and copies (a6),
 * [6] the next step's input-free update and the wait at the second barrier.
 * Graph path: [0] the k_update kernel and [4] the k_route kernel of every
 * step (CUDA events between them, which add a little time), the rest 0.
 * Synchronises the stream.  Errors: SNN_E_ARG, SNN_E_CUDA.
 */
int snn_profile_phases(snn_sim *sim, int32_t T, double *phase_ms);

/*
 * Route a caller-given set of spikes through the two-level route (level-1
 * entries per destination VN, level-2 relay expansion into partition
 * segments, Sec. IV.B) and fan them out:
 *     out[(d-1)*M + j] += sum of w over synapses i -> j with delay d,
 * summed over the listed source neurons i (global ids; a repeated id is
 * delivered once per occurrence).  Use: external stimulation, or the
 * synaptic input a spike pattern produces, without advancing the sim.
 *   ids: device uint32 [n]; out: device int32 [max_delay * M], global
 *   neuron order, accumulated into (the call does not clear it); both
 *   caller-owned.  counts (host uint64 [3], may be NULL) receives the
 *   level-1 entries, level-2 entries and synaptic events of this call.
 * Scratch: the level-1 bucket and level-2 inbox regions of the sim's
 * workspace, so the call must not overlap snn_step on the same sim.
 * Runs on the sim's stream, with the sim's device current (the caller's
 * current device is restored), and synchronises the stream before returning.
 * Errors: SNN_E_ARG (n < 0, NULL pointers with n > 0, an id >= M),
 * SNN_E_CAPACITY (the spikes need more bucket/inbox room than the
 * workspace holds), SNN_E_CUDA.
 */
int snn_deliver_spikes(snn_sim *sim, const uint32_t *ids, int64_t n, int32_t *out,
                       uint64_t *counts);

/*
 * snn_deliver_spikes without any device allocation.  The paper has no
 * counterpart: this is for callers that cannot allocate device memory while
 * they run, such as a host program that hands out all device memory itself
 * from a fixed budget, or a real-time stimulation loop that may not stall
 * in an allocator call.  It computes exactly what snn_deliver_spikes
 * computes (same arguments, same output, same counts) but keeps its scratch
 * in a fixed array built into the library, of snn_static_scratch_bytes()
 * (8 MiB) per GPU; every GPU that loads the library holds that array until
 * the process exits.  The call itself allocates nothing: no cudaMalloc,
 * no cudaFree.
 *   - The first call on a device looks up the array's device address once
 *     (cudaGetSymbolAddress, with that device current); make that first
 *     call before any stream capture.  The address stays cached for the
 *     life of the process: after cudaDeviceReset (or a reset of the
 *     device's primary context) the library's module is unloaded and this
 *     call must not be used again in that process.
 *   - Size limit: n * (4 B * longest level-1 row + 8 B * most level-2
 *     entries of any neuron) + 512 B must fit in the array; larger calls
 *     return SNN_E_RANGE and do nothing.
 *   - All calls share the one array and each call clears its counters
 *     first, so calls that overlap on the GPU (other streams, other threads,
 *     other sims on the same GPU) race and give wrong results: serialise
 *     them.  The array keeps the last call's contents.
 * Errors: as snn_deliver_spikes, plus SNN_E_RANGE.
 */
int snn_deliver_spikes_static(snn_sim *sim, const uint32_t *ids, int64_t n, int32_t *out,
                              uint64_t *counts);
/* Size in bytes of the fixed scratch array of snn_deliver_spikes_static. */
size_t snn_static_scratch_bytes(void);

void snn_sim_destroy(snn_sim *sim);

#ifdef __cplusplus
}
#endif

#endif /* SNN_H */
