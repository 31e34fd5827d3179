/*
 * CPU ORACLE — test infrastructure only.
 *
 * A plain, sequential, deliberately slow simulator of one step of a
 * partitioned LIF network with the paper's message structure (arXiv
 * 2205.07125, "A Low-latency Communication Design for Brain Simulations").
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may call it; the GPU library never links or calls it, and it shares no
 * code, header or table with the GPU library.
 *
 * What it computes, per step t (state V, ref, ring; all sizes in neurons):
 *   1. for every partition p in order, for every neuron j of p in ascending
 *      id: take the recurrent input ring[t mod D][j] and zero it, add the
 *      Poisson drive and the bias, run the LIF update (FP32, fixed operation
 *      order) and the threshold test; a spiking neuron is put on the
 *      partition's out-queue.  (The paper leaves the neuron model open; its
 *      only neuron-model statement is LIF as a model family, Table I.)
 *   2. the direct route (the peer-to-peer baseline the paper compares
 *      against, Sec. II and Table II "Random/P2P"): every spike i of p is
 *      appended to the inbox of every partition q that holds at least one
 *      target of i.
 *   3. delivery: every partition q walks its inbox and adds, for each
 *      synapse (i -> j in q, weight w, delay d), w into ring[(t+d) mod D][j]
 *      (int32).
 *   4. message counts of the direct route and of the two-level route
 *      (Sec. IV.B: GPUs grouped into virtual nodes; traffic inside a group
 *      goes directly, traffic to another group goes to one relay ("bridge")
 *      partition of the destination group which forwards it), computed from
 *      their definitions with a fresh scan of each spike's synapses,
 *      independently of steps 2-3.
 *   5. an FP64 shadow membrane driven by the same integer inputs, for the
 *      FP32-vs-FP64 membrane error.
 *
 * It also holds the partitioning (Algorithm 1, sequential and batched
 * growth) and grouping (Algorithm 2) readings as plain greedy loops, for the
 * partition tests, the device partitioner's parity and the message counts
 * of a greedy mapping.
 *
 * Readings of points the paper leaves open (all are listed with the design
 * notes):
 *   - LIF: u = V - E_L; V = E_L + alpha*u; V = V + I*2^-10 mV with
 *     alpha = fl32(exp(-dt/tau)); spike if V >= V_th, then V = V_reset and
 *     ref = t_ref; while ref > 0 the neuron is clamped to V_reset, ref
 *     decreases by one, and its input is consumed and discarded.
 *   - Poisson drive: k ~ Poisson(lambda) by inverse CDF on one 32-bit
 *     Philox4x32-10 word (Salmon et al., SC'11): neuron j at step t takes word
 *     (j mod 4) of the block with key = drive seed and counter =
 *     (j div 4, step, 0, 0), so one block serves four consecutive neurons;
 *     thresholds floor(2^32 * CDF(k)) in double.
 *   - relay of destination group g for a source partition p of another
 *     group (the "bridge" of Sec. IV.B; which member relays whose traffic
 *     is the design choice the paper's level-2 traffic result rests on,
 *     Sec. V, Fig. 3(b)), members of a group ranked by ascending partition
 *     index, by policy:
 *       per group (default): the ((h - g) mod |g|)-th member of g, h = group
 *       of p (it depends only on the groups' distance, so networks placed
 *       side by side in one mapping get each their own relays);
 *       per partition: the (rank of p in its own group mod |g|)-th member;
 *       balanced: longest-processing-time first -- the sources of g in
 *       decreasing static load (ties: lower index) each join the member of
 *       g with the least load so far (ties: lower rank); the static load of
 *       (g, p) is the number of (neuron of p, partition of g) pairs with
 *       synapses; sources of load 0 take the per-partition member;
 *     for the own group the source partition sends directly.
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:  */
/* as easy as 1, 2, 3", SC 2011): ten rounds of the 4x32 Philox S-box    */
/* with round multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key bumps     */
/* 0x9E3779B9 / 0xBB67AE85.                                              */
/* ------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Drive word of neuron j at step t: word j mod 4 of block (j div 4, t, 0, 0). */
static uint32_t drive_word(uint64_t seed, uint32_t j, uint32_t t)
{
    uint32_t ctr[4] = {j >> 2, t, 0u, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return out[j & 3u];
}

static uint32_t philox_word(uint64_t seed, uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t ctr[4] = {a, b, c, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return out[0];
}

/* ------------------------------------------------------------------ */
/* Poisson inverse-CDF thresholds: th[k] = floor(2^32 * P(X <= k)),     */
/* pmf by the recurrence p_0 = e^-lambda, p_k = p_{k-1} * lambda / k,   */
/* closed by a final 2^32.  A draw is k = #{m : th[m] <= u}.            */
/* ------------------------------------------------------------------ */
#define OR_PTAB 32

int or_poisson_table(double lambda, uint64_t *th, int32_t *len)
{
    if (!(lambda >= 0.0) || lambda > 16.0) return -1;
    double pmf = exp(-lambda), cdf = pmf;
    int n = 0;
    for (int k = 0; k < OR_PTAB; ++k) {
        if (k > 0) {
            pmf = pmf * lambda / (double)k;
            cdf = cdf + pmf;
        }
        double x = floor(cdf * 4294967296.0);
        /* the table closes at the first k whose threshold reaches 2^32 - 1:
         * that entry becomes 2^32, so every 32-bit word maps below it */
        uint64_t v = x >= 4294967295.0 ? 4294967296ULL : (uint64_t)x;
        th[k] = v;
        n = k + 1;
        if (v >= 4294967296ULL) break;
    }
    *len = n;
    return 0;
}

static int32_t poisson_draw(const uint64_t *th, int32_t len, uint32_t u)
{
    int32_t k = 0;
    for (int32_t m = 0; m < len; ++m)
        if (th[m] <= (uint64_t)u) ++k;
    return k;
}

/* splitmix64 finaliser (Steele, Lea, Flood, OOPSLA 2014), used for the    */
/* order-free per-step hashes h = sum_j mix((j << 32) | bits(x_j)).        */
static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t or_mix64(uint64_t z) { return mix64(z); }

/* ------------------------------------------------------------------ */
/* Partitions                                                          */
/* ------------------------------------------------------------------ */

/* Planted contiguous partition: part(i) = p with floor(pM/P) <= i < floor((p+1)M/P). */
int or_partition_planted(int64_t M, int32_t P, int32_t *part_of)
{
    if (M <= 0 || P <= 0 || P > M) return -1;
    for (int32_t p = 0; p < P; ++p) {
        int64_t s = ((int64_t)p * M) / P, e = ((int64_t)(p + 1) * M) / P;
        for (int64_t i = s; i < e; ++i) part_of[i] = p;
    }
    return 0;
}

/* Objective of Algorithm 1: sum over synapses i->j whose ends lie in
 * different parts of W_i * W_j, with W_i the out-degree of i (the paper's
 * neuron weight: the data volume a neuron generates, uniform rates). */
int64_t or_cut(int64_t M, const int64_t *syn_ptr, const uint32_t *tgt, const int32_t *part_of)
{
    int64_t cut = 0;
    for (int64_t i = 0; i < M; ++i) {
        int64_t wi = syn_ptr[i + 1] - syn_ptr[i];
        for (int64_t e = syn_ptr[i]; e < syn_ptr[i + 1]; ++e) {
            int64_t j = tgt[e];
            if (part_of[i] != part_of[j]) cut += wi * (syn_ptr[j + 1] - syn_ptr[j]);
        }
    }
    return cut;
}

/*
 * Algorithm 1 (Sec. IV.A), greedy reading.  For t = 1..T: grow parts
 * k = 0..P-2 one at a time from a seed (t = 1: lowest unassigned id;
 * t > 1: a Philox-chosen unassigned neuron), repeatedly adding the
 * unassigned neuron j with the largest gain sum_{i in k} (c_ij + c_ji) W_i W_j
 * (ties: lowest id) while W(k) < sum(W)/P; the last part takes the rest.
 * Keep the mapping with the smallest objective (first one on ties).
 * Naive O(M) scan per added neuron.
 */
int or_partition_greedy(int64_t M, const int64_t *syn_ptr, const uint32_t *tgt, int32_t P,
                        int32_t iters, uint64_t seed, int32_t *part_of, int64_t *best_cut)
{
    if (M <= 0 || P <= 0 || P > M || iters < 1) return -1;
    int64_t E = syn_ptr[M];
    /* in-edge lists */
    int64_t *in_ptr = calloc((size_t)M + 1, sizeof(int64_t));
    uint32_t *in_src = malloc((size_t)(E > 0 ? E : 1) * sizeof(uint32_t));
    int64_t *gain = malloc((size_t)M * sizeof(int64_t));
    int32_t *cur = malloc((size_t)M * sizeof(int32_t));
    if (!in_ptr || !in_src || !gain || !cur) return -2;
    for (int64_t e = 0; e < E; ++e) in_ptr[tgt[e] + 1]++;
    for (int64_t i = 0; i < M; ++i) in_ptr[i + 1] += in_ptr[i];
    {
        int64_t *fill = malloc((size_t)M * sizeof(int64_t));
        memcpy(fill, in_ptr, (size_t)M * sizeof(int64_t));
        for (int64_t i = 0; i < M; ++i)
            for (int64_t e = syn_ptr[i]; e < syn_ptr[i + 1]; ++e) in_src[fill[tgt[e]]++] = (uint32_t)i;
        free(fill);
    }
    int64_t Wtot = E;
    int64_t best = -1;
    for (int32_t t = 1; t <= iters; ++t) {
        for (int64_t i = 0; i < M; ++i) cur[i] = -1;
        int64_t n_un = M;
        for (int32_t k = 0; k < P; ++k) {
            if (k == P - 1) {
                for (int64_t i = 0; i < M; ++i) if (cur[i] < 0) cur[i] = k;
                break;
            }
            if (n_un == 0) break;
            int64_t s = -1;
            if (t == 1) {
                for (int64_t i = 0; i < M; ++i) if (cur[i] < 0) { s = i; break; }
            } else {
                int64_t r = (int64_t)(philox_word(seed, (uint32_t)t, (uint32_t)k, 0xA1u) % (uint64_t)n_un);
                for (int64_t i = 0; i < M; ++i) if (cur[i] < 0) { if (r == 0) { s = i; break; } --r; }
            }
            for (int64_t i = 0; i < M; ++i) gain[i] = 0;
            int64_t wk = 0;
            int64_t add = s;
            while (add >= 0) {
                cur[add] = k;
                --n_un;
                int64_t wa = syn_ptr[add + 1] - syn_ptr[add];
                wk += wa;
                for (int64_t e = syn_ptr[add]; e < syn_ptr[add + 1]; ++e) {
                    int64_t j = tgt[e];
                    gain[j] += wa * (syn_ptr[j + 1] - syn_ptr[j]);
                }
                for (int64_t e = in_ptr[add]; e < in_ptr[add + 1]; ++e) {
                    int64_t j = in_src[e];
                    gain[j] += wa * (syn_ptr[j + 1] - syn_ptr[j]);
                }
                if (!(wk * (int64_t)P < Wtot) || n_un == 0) break;
                add = -1;
                int64_t bg = -1;
                for (int64_t j = 0; j < M; ++j)
                    if (cur[j] < 0 && gain[j] > bg) { bg = gain[j]; add = j; }
            }
        }
        int64_t c = or_cut(M, syn_ptr, tgt, cur);
        if (best < 0 || c < best) {
            best = c;
            memcpy(part_of, cur, (size_t)M * sizeof(int32_t));
        }
    }
    *best_cut = best;
    free(in_ptr); free(in_src); free(gain); free(cur);
    return 0;
}

/*
 * Algorithm 1 (Sec. IV.A) with batched growth, the parallel form of the
 * greedy the paper proposes as future work (Sec. VII, parallelization of
 * algorithms).  Seeds, stopping rule, last part, iterations and objective
 * are those of or_partition_greedy.  The difference is in how a part grows:
 * in each round the `need` unassigned neurons with the largest gains (ties:
 * lowest id) are taken, ranked by the gains of that round (no update inside
 * the round); they join the part one at a time in rank order, the stopping
 * rule checked after each; the gains of the ones that joined are added
 * before the next round.  need = min(B, unassigned, max(1, n_k / g)) with
 * n_k the neurons already in the part: with g > 0 a round grows with the
 * part (a part's first rounds, whose gains rest on few members, stay small);
 * g = 0 drops that term.  With B = 1 this is or_partition_greedy step for
 * step.
 * Naive: the batch is taken by `need` argmax scans, O(M * need) per round.
 */
int or_partition_greedy_batched(int64_t M, const int64_t *syn_ptr, const uint32_t *tgt, int32_t P,
                                int32_t iters, uint64_t seed, int32_t B, int32_t g, int32_t *part_of,
                                int64_t *best_cut)
{
    if (M <= 0 || P <= 0 || P > M || iters < 1 || B < 1 || g < 0) return -1;
    int64_t E = syn_ptr[M];
    int64_t *in_ptr = calloc((size_t)M + 1, sizeof(int64_t));
    uint32_t *in_src = malloc((size_t)(E > 0 ? E : 1) * sizeof(uint32_t));
    int64_t *gain = malloc((size_t)M * sizeof(int64_t));
    int32_t *cur = malloc((size_t)M * sizeof(int32_t));
    char *picked = calloc((size_t)M, 1);
    int64_t *batch = malloc((size_t)B * sizeof(int64_t));
    if (!in_ptr || !in_src || !gain || !cur || !picked || !batch) return -2;
    for (int64_t e = 0; e < E; ++e) in_ptr[tgt[e] + 1]++;
    for (int64_t i = 0; i < M; ++i) in_ptr[i + 1] += in_ptr[i];
    {
        int64_t *fill = malloc((size_t)M * sizeof(int64_t));
        memcpy(fill, in_ptr, (size_t)M * sizeof(int64_t));
        for (int64_t i = 0; i < M; ++i)
            for (int64_t e = syn_ptr[i]; e < syn_ptr[i + 1]; ++e) in_src[fill[tgt[e]]++] = (uint32_t)i;
        free(fill);
    }
    int64_t Wtot = E;
    int64_t best = -1;
    for (int32_t t = 1; t <= iters; ++t) {
        for (int64_t i = 0; i < M; ++i) cur[i] = -1;
        int64_t n_un = M;
        for (int32_t k = 0; k < P; ++k) {
            if (k == P - 1) {
                for (int64_t i = 0; i < M; ++i) if (cur[i] < 0) cur[i] = k;
                break;
            }
            if (n_un == 0) break;
            int64_t s = -1;
            if (t == 1) {
                for (int64_t i = 0; i < M; ++i) if (cur[i] < 0) { s = i; break; }
            } else {
                int64_t r = (int64_t)(philox_word(seed, (uint32_t)t, (uint32_t)k, 0xA1u) % (uint64_t)n_un);
                for (int64_t i = 0; i < M; ++i) if (cur[i] < 0) { if (r == 0) { s = i; break; } --r; }
            }
            for (int64_t i = 0; i < M; ++i) gain[i] = 0;
            /* the seed is a round of one */
            int64_t n_b = 1;
            batch[0] = s;
            int64_t wk = 0, n_k = 0;
            int stop = 0;
            while (!stop) {
                /* members join in rank order until the part is full */
                int64_t joined = 0;
                for (int64_t r = 0; r < n_b; ++r) {
                    int64_t a = batch[r];
                    cur[a] = k;
                    --n_un;
                    wk += syn_ptr[a + 1] - syn_ptr[a];
                    ++joined;
                    ++n_k;
                    if (!(wk * (int64_t)P < Wtot) || n_un == 0) { stop = 1; break; }
                }
                if (stop) break;
                /* gains of the members that joined: (c_aj + c_ja) W_a W_j */
                for (int64_t r = 0; r < joined; ++r) {
                    int64_t a = batch[r];
                    int64_t wa = syn_ptr[a + 1] - syn_ptr[a];
                    for (int64_t e = syn_ptr[a]; e < syn_ptr[a + 1]; ++e) {
                        int64_t j = tgt[e];
                        gain[j] += wa * (syn_ptr[j + 1] - syn_ptr[j]);
                    }
                    for (int64_t e = in_ptr[a]; e < in_ptr[a + 1]; ++e) {
                        int64_t j = in_src[e];
                        gain[j] += wa * (syn_ptr[j + 1] - syn_ptr[j]);
                    }
                }
                /* next round: the need best unassigned neurons, in rank order */
                int64_t need = n_un < (int64_t)B ? n_un : (int64_t)B;
                if (g > 0 && n_k / g < need) need = n_k / g > 1 ? n_k / g : 1;
                for (n_b = 0; n_b < need; ++n_b) {
                    int64_t add = -1, bg = -1;
                    for (int64_t j = 0; j < M; ++j)
                        if (cur[j] < 0 && !picked[j] && gain[j] > bg) { bg = gain[j]; add = j; }
                    picked[add] = 1;
                    batch[n_b] = add;
                }
                for (int64_t r = 0; r < n_b; ++r) picked[batch[r]] = 0;
            }
        }
        int64_t c = or_cut(M, syn_ptr, tgt, cur);
        if (best < 0 || c < best) {
            best = c;
            memcpy(part_of, cur, (size_t)M * sizeof(int32_t));
        }
    }
    *best_cut = best;
    free(in_ptr); free(in_src); free(gain); free(cur); free(picked); free(batch);
    return 0;
}

/* Inter-partition synapse counts PG[p*P+q] (p != q) and weights WG[p]. */
static void part_graph(int64_t M, const int64_t *syn_ptr, const uint32_t *tgt,
                       const int32_t *part_of, int32_t P, int64_t *PG, int64_t *WG)
{
    memset(PG, 0, sizeof(int64_t) * (size_t)P * (size_t)P);
    memset(WG, 0, sizeof(int64_t) * (size_t)P);
    for (int64_t i = 0; i < M; ++i) {
        int32_t p = part_of[i];
        WG[p] += syn_ptr[i + 1] - syn_ptr[i];
        for (int64_t e = syn_ptr[i]; e < syn_ptr[i + 1]; ++e) {
            int32_t q = part_of[tgt[e]];
            if (q != p) PG[(int64_t)p * P + q]++;
        }
    }
}

/*
 * Algorithm 2 (Sec. IV.B), greedy grouping reading.  Group size s = P/n_vn.
 * For t = 1..T: form groups g = 0..n_vn-2 one at a time from a seed
 * (t = 1: the heaviest ungrouped partition, ties lowest index; t > 1: a
 * Philox-chosen ungrouped partition), adding the ungrouped q with the
 * largest sum_{m in g} (PG[m][q] + PG[q][m]) WG[m] WG[q] (ties: lowest q)
 * until the group has s members; the last group takes the rest.  Keep the
 * grouping with the smallest inter-group sum of PG[p][q] WG[p] WG[q].
 * cost_out receives that sum as two 64-bit halves (lo, hi).
 */
int or_group_greedy(int64_t M, const int64_t *syn_ptr, const uint32_t *tgt,
                    const int32_t *part_of, int32_t P, int32_t n_vn, int32_t iters,
                    uint64_t seed, int32_t *vn_of_part, uint64_t *cost_out)
{
    if (P <= 0 || n_vn <= 0 || P % n_vn || iters < 1) return -1;
    int32_t s = P / n_vn;
    int64_t *PG = malloc(sizeof(int64_t) * (size_t)P * (size_t)P);
    int64_t *WG = malloc(sizeof(int64_t) * (size_t)P);
    int32_t *cur = malloc(sizeof(int32_t) * (size_t)P);
    part_graph(M, syn_ptr, tgt, part_of, P, PG, WG);
    unsigned __int128 best = 0;
    int have = 0;
    for (int32_t t = 1; t <= iters; ++t) {
        for (int32_t p = 0; p < P; ++p) cur[p] = -1;
        int32_t n_un = P;
        for (int32_t g = 0; g < n_vn; ++g) {
            if (g == n_vn - 1) {
                for (int32_t p = 0; p < P; ++p) if (cur[p] < 0) cur[p] = g;
                break;
            }
            int32_t sd = -1;
            if (t == 1) {
                for (int32_t p = 0; p < P; ++p)
                    if (cur[p] < 0 && (sd < 0 || WG[p] > WG[sd])) sd = p;
            } else {
                int32_t r = (int32_t)(philox_word(seed, (uint32_t)t, (uint32_t)g, 0xA2u) % (uint32_t)n_un);
                for (int32_t p = 0; p < P; ++p) if (cur[p] < 0) { if (r == 0) { sd = p; break; } --r; }
            }
            cur[sd] = g; --n_un;
            for (int32_t m = 1; m < s; ++m) {
                int32_t bq = -1;
                unsigned __int128 bgain = 0;
                for (int32_t q = 0; q < P; ++q) {
                    if (cur[q] >= 0) continue;
                    unsigned __int128 gq = 0;
                    for (int32_t x = 0; x < P; ++x)
                        if (cur[x] == g)
                            gq += (unsigned __int128)(PG[(int64_t)x * P + q] + PG[(int64_t)q * P + x])
                                  * (unsigned __int128)WG[x] * (unsigned __int128)WG[q];
                    if (bq < 0 || gq > bgain) { bq = q; bgain = gq; }
                }
                cur[bq] = g; --n_un;
            }
        }
        unsigned __int128 c = 0;
        for (int32_t p = 0; p < P; ++p)
            for (int32_t q = 0; q < P; ++q)
                if (cur[p] != cur[q])
                    c += (unsigned __int128)PG[(int64_t)p * P + q] * (unsigned __int128)WG[p]
                         * (unsigned __int128)WG[q];
        if (!have || c < best) {
            best = c; have = 1;
            memcpy(vn_of_part, cur, sizeof(int32_t) * (size_t)P);
        }
    }
    cost_out[0] = (uint64_t)best;
    cost_out[1] = (uint64_t)(best >> 64);
    free(PG); free(WG); free(cur);
    return 0;
}

/* The k-th partition of group g in ascending index (k taken mod |g|). */
static int32_t member_of(const int32_t *vn_of_part, int32_t P, int32_t g, int32_t k)
{
    int32_t sz = 0;
    for (int32_t p = 0; p < P; ++p) if (vn_of_part[p] == g) ++sz;
    int32_t want = k % sz;
    for (int32_t p = 0; p < P; ++p)
        if (vn_of_part[p] == g) { if (want == 0) return p; --want; }
    return -1;
}

/* relay(g, h): the ((h - g) mod |g|)-th partition of group g, ascending index. */
static int32_t relay_of(const int32_t *vn_of_part, int32_t P, int32_t g, int32_t h)
{
    int32_t sz = 0;
    for (int32_t p = 0; p < P; ++p) if (vn_of_part[p] == g) ++sz;
    int32_t k = (h - g) % sz;
    if (k < 0) k += sz;
    return member_of(vn_of_part, P, g, k);
}

/* Rank of partition p among the partitions of its own group (ascending index). */
static int32_t rank_in_group(const int32_t *vn_of_part, int32_t p)
{
    int32_t r = 0;
    for (int32_t x = 0; x < p; ++x) r += vn_of_part[x] == vn_of_part[p];
    return r;
}

/* ------------------------------------------------------------------ */
/* Simulator                                                           */
/* ------------------------------------------------------------------ */
typedef struct {
    double dt_ms, tau_ms;
    float e_l, v_th, v_reset;
    int32_t t_ref;
    double drive_lambda;
    int32_t w_ext;
    int32_t i_bias;
    uint64_t drive_seed;
} or_dyn;

enum {
    OC_STEPS = 0, OC_SPIKES, OC_EVENTS, OC_DIRECT, OC_DIRECT_XVN,
    OC_L1_LOCAL, OC_L1_XVN, OC_L2_LOCAL, OC_L2_PEER, OC_L2_RELAY_LOCAL, OC_L2_RELAY_REMOTE,
    OC_N
};

typedef struct {
    int64_t M, E;
    const int64_t *syn_ptr;
    const uint32_t *tgt;
    const int16_t *w;
    const uint8_t *d;
    int32_t P, n_vn;
    int32_t *part_of;      /* copy */
    int32_t *vn_of_part;   /* copy */
    int32_t *relay;        /* [n_vn * P]: relay[g * P + p] of source partition p, -1 for p in g */
    or_dyn dyn;
    float alpha;
    double alpha64;
    uint64_t th[OR_PTAB];
    int32_t th_len;
    /* per-neuron synapses grouped by destination partition */
    uint32_t *ord;         /* [E] within-row indices, stable-sorted by part_of[tgt] */
    int64_t *seg_ptr;      /* [M+1] */
    int32_t *seg_q;
    uint32_t *seg_beg, *seg_len;
    /* partition membership lists (ascending ids) */
    int64_t *mem_ptr;      /* [P+1] */
    uint32_t *mem;         /* [M] */
} or_net;

void or_destroy(void *hv)
{
    or_net *h = (or_net *)hv;
    if (!h) return;
    free(h->part_of); free(h->vn_of_part); free(h->relay); free(h->ord); free(h->seg_ptr);
    free(h->seg_q); free(h->seg_beg); free(h->seg_len); free(h->mem_ptr); free(h->mem);
    free(h);
}

void *or_create(int64_t M, const int64_t *syn_ptr, const uint32_t *tgt, const int16_t *w,
                const uint8_t *d, int32_t P, const int32_t *part_of, int32_t n_vn,
                const int32_t *vn_of_part, const or_dyn *dyn)
{
    if (M <= 0 || P <= 0 || n_vn <= 0) return NULL;
    or_net *h = calloc(1, sizeof(or_net));
    h->M = M; h->E = syn_ptr[M];
    h->syn_ptr = syn_ptr; h->tgt = tgt; h->w = w; h->d = d;
    h->P = P; h->n_vn = n_vn; h->dyn = *dyn;
    h->part_of = malloc(sizeof(int32_t) * (size_t)M);
    memcpy(h->part_of, part_of, sizeof(int32_t) * (size_t)M);
    h->vn_of_part = malloc(sizeof(int32_t) * (size_t)P);
    memcpy(h->vn_of_part, vn_of_part, sizeof(int32_t) * (size_t)P);
    for (int32_t p = 0; p < P; ++p)
        if (vn_of_part[p] < 0 || vn_of_part[p] >= n_vn) { or_destroy(h); return NULL; }
    for (int64_t i = 0; i < M; ++i)
        if (part_of[i] < 0 || part_of[i] >= P) { or_destroy(h); return NULL; }
    h->relay = malloc(sizeof(int32_t) * (size_t)n_vn * (size_t)P);
    for (int32_t g = 0; g < n_vn; ++g)
        for (int32_t p = 0; p < P; ++p)
            h->relay[g * P + p] = vn_of_part[p] == g ? -1 : relay_of(vn_of_part, P, g, vn_of_part[p]);
    h->alpha = (float)exp(-dyn->dt_ms / dyn->tau_ms);
    h->alpha64 = exp(-dyn->dt_ms / dyn->tau_ms);
    if (or_poisson_table(dyn->drive_lambda, h->th, &h->th_len)) { or_destroy(h); return NULL; }

    /* group each neuron's synapses by destination partition (counting sort) */
    int64_t E = h->E;
    h->ord = malloc(sizeof(uint32_t) * (size_t)(E > 0 ? E : 1));
    h->seg_ptr = malloc(sizeof(int64_t) * (size_t)(M + 1));
    int32_t *cnt = calloc((size_t)P, sizeof(int32_t));
    int64_t nseg = 0;
    for (int64_t i = 0; i < M; ++i) {
        h->seg_ptr[i] = nseg;
        for (int64_t e = syn_ptr[i]; e < syn_ptr[i + 1]; ++e) {
            int32_t q = part_of[tgt[e]];
            if (cnt[q]++ == 0) ++nseg;
        }
        for (int64_t e = syn_ptr[i]; e < syn_ptr[i + 1]; ++e) cnt[part_of[tgt[e]]] = 0;
    }
    h->seg_ptr[M] = nseg;
    h->seg_q = malloc(sizeof(int32_t) * (size_t)(nseg + 1));
    h->seg_beg = malloc(sizeof(uint32_t) * (size_t)(nseg + 1));
    h->seg_len = malloc(sizeof(uint32_t) * (size_t)(nseg + 1));
    uint32_t *pos = malloc(sizeof(uint32_t) * (size_t)P);
    for (int64_t i = 0; i < M; ++i) {
        int64_t b = syn_ptr[i], n = syn_ptr[i + 1] - b;
        for (int64_t k = 0; k < n; ++k) cnt[part_of[tgt[b + k]]]++;
        int64_t sg = h->seg_ptr[i];
        uint32_t run = 0;
        for (int32_t q = 0; q < P; ++q) {
            if (!cnt[q]) continue;
            h->seg_q[sg] = q; h->seg_beg[sg] = run; h->seg_len[sg] = (uint32_t)cnt[q];
            pos[q] = run; run += (uint32_t)cnt[q]; ++sg;
        }
        for (int64_t k = 0; k < n; ++k) h->ord[b + pos[part_of[tgt[b + k]]]++] = (uint32_t)k;
        for (int64_t k = 0; k < n; ++k) cnt[part_of[tgt[b + k]]] = 0;
    }
    free(cnt); free(pos);
    /* membership lists */
    h->mem_ptr = calloc((size_t)P + 1, sizeof(int64_t));
    h->mem = malloc(sizeof(uint32_t) * (size_t)M);
    for (int64_t i = 0; i < M; ++i) h->mem_ptr[part_of[i] + 1]++;
    for (int32_t p = 0; p < P; ++p) h->mem_ptr[p + 1] += h->mem_ptr[p];
    {
        int64_t *f = malloc(sizeof(int64_t) * (size_t)P);
        memcpy(f, h->mem_ptr, sizeof(int64_t) * (size_t)P);
        for (int64_t i = 0; i < M; ++i) h->mem[f[part_of[i]]++] = (uint32_t)i;
        free(f);
    }
    return h;
}

static int cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : x > y;
}

/* simple growable queue of 64-bit items */
typedef struct { int64_t *v; int64_t n, cap; } q64;
static void q_push(q64 *q, int64_t x)
{
    if (q->n == q->cap) {
        q->cap = q->cap ? 2 * q->cap : 64;
        q->v = realloc(q->v, sizeof(int64_t) * (size_t)q->cap);
    }
    q->v[q->n++] = x;
}

/*
 * Run T steps starting at global step t0.  State (V, ref, ring[D][M],
 * v64) is caller-owned and updated in place; D must exceed no delay minus
 * one, i.e. D >= max delay.  Optional records (NULL to skip):
 *   raster_ids/raster_off: spikes of step t0+k, ascending ids, in
 *     raster_ids[raster_off[k] .. raster_off[k+1]) (raster_off has T+1 slots)
 *   cur_hash/v_hash [T]: order-free hashes of the consumed recurrent input
 *     and of V after the update
 *   rec_steps[n_rec] / rec_cur[n_rec][M]: consumed recurrent input of the
 *     listed global steps
 *   counts[OC_N]: accumulated
 *   fp64[3]: max relative error, compared samples, threshold disagreements
 *   pairs: the (spike, destination partition) pairs of the last step's
 *     direct route, packed (i << 32) | q
 * Returns 0, -1 bad argument, -3 raster capacity exceeded.
 */
int or_run(void *hv, int64_t t0, int32_t T, int32_t D,
           float *V, uint8_t *ref, int32_t *ring, double *v64,
           uint32_t *raster_ids, int64_t raster_cap, int64_t *raster_off,
           uint64_t *cur_hash, uint64_t *v_hash,
           int32_t n_rec, const int64_t *rec_steps, int32_t *rec_cur,
           uint64_t *counts, double *fp64,
           uint64_t *pairs, int64_t pairs_cap, int64_t *n_pairs)
{
    or_net *h = (or_net *)hv;
    if (!h || T < 0 || D < 1) return -1;
    const int64_t M = h->M;
    const int32_t P = h->P;
    for (int64_t e = 0; e < h->E; ++e)
        if (h->d[e] < 1 || h->d[e] > D) return -1;
    const or_dyn *dy = &h->dyn;
    const float alpha = h->alpha, e_l = dy->e_l, v_th = dy->v_th, v_reset = dy->v_reset;
    const float scale = 0.0009765625f; /* 2^-10 mV per unit */
    q64 *outq = calloc((size_t)P, sizeof(q64));
    q64 *inbox = calloc((size_t)P, sizeof(q64));
    uint8_t *mark = calloc((size_t)P, 1);
    uint8_t *gmark = calloc((size_t)h->n_vn, 1);
    int64_t nr = 0;
    if (raster_off) raster_off[0] = 0;
    int rc = 0;
    for (int32_t k = 0; k < T; ++k) {
        const int64_t t = t0 + k;
        const int64_t slot = t % D;
        int32_t *rs = ring + slot * M;
        int32_t *rec = NULL;
        for (int32_t r = 0; r < n_rec; ++r) if (rec_steps[r] == t) rec = rec_cur + (int64_t)r * M;
        uint64_t ch = 0, vh = 0;
        /* 1. update, partition by partition, ascending ids */
        for (int32_t p = 0; p < P; ++p) {
            outq[p].n = 0;
            for (int64_t m = h->mem_ptr[p]; m < h->mem_ptr[p + 1]; ++m) {
                int64_t j = h->mem[m];
                int32_t irec = rs[j];
                rs[j] = 0;
                if (rec) rec[j] = irec;
                ch += mix64(((uint64_t)j << 32) | (uint32_t)irec);
                uint32_t u = drive_word(dy->drive_seed, (uint32_t)j, (uint32_t)t);
                int32_t kd = poisson_draw(h->th, h->th_len, u);
                int32_t I = (int32_t)((uint32_t)irec + (uint32_t)kd * (uint32_t)dy->w_ext
                                      + (uint32_t)dy->i_bias);
                float v = V[j];
                if (ref[j] > 0) {
                    ref[j] = (uint8_t)(ref[j] - 1);
                    v = v_reset;
                    if (v64) v64[j] = (double)v_reset;
                } else {
                    float uu = v - e_l;
                    float au = alpha * uu;
                    v = e_l + au;
                    float x = (float)I * scale;
                    v = v + x;
                    int spk = v >= v_th;
                    if (v64) {
                        double y = (double)e_l + h->alpha64 * (v64[j] - (double)e_l)
                                   + (double)I * (1.0 / 1024.0);
                        int spk64 = y >= (double)v_th;
                        if (spk64 != spk) {
                            if (fp64) fp64[2] += 1.0;
                            y = (double)v;
                        } else if (!spk && fp64) {
                            double rel = fabs((double)v - y) / fabs(y);
                            if (rel > fp64[0]) fp64[0] = rel;
                            fp64[1] += 1.0;
                        }
                        v64[j] = spk ? (double)v_reset : y;
                    }
                    if (spk) {
                        v = v_reset;
                        ref[j] = (uint8_t)dy->t_ref;
                        q_push(&outq[p], j);
                    }
                }
                V[j] = v;
                uint32_t vb;
                memcpy(&vb, &v, 4);
                vh += mix64(((uint64_t)j << 32) | vb);
            }
        }
        if (cur_hash) cur_hash[k] = ch;
        if (v_hash) v_hash[k] = vh;
        /* raster record, ascending ids */
        int64_t S = 0;
        for (int32_t p = 0; p < P; ++p) S += outq[p].n;
        if (raster_ids) {
            if (nr + S > raster_cap) { rc = -3; break; }
            int64_t b = nr;
            for (int32_t p = 0; p < P; ++p)
                for (int64_t a = 0; a < outq[p].n; ++a) raster_ids[nr++] = (uint32_t)outq[p].v[a];
            qsort(raster_ids + b, (size_t)S, sizeof(uint32_t), cmp_u32);
            raster_off[k + 1] = nr;
        }
        /* 2. direct route: each spike to every partition holding a target */
        for (int32_t q = 0; q < P; ++q) inbox[q].n = 0;
        for (int32_t p = 0; p < P; ++p)
            for (int64_t a = 0; a < outq[p].n; ++a) {
                int64_t i = outq[p].v[a];
                for (int64_t sg = h->seg_ptr[i]; sg < h->seg_ptr[i + 1]; ++sg) q_push(&inbox[h->seg_q[sg]], sg);
            }
        if (pairs && k == T - 1) {
            int64_t np = 0;
            for (int32_t q = 0; q < P; ++q)
                for (int64_t a = 0; a < inbox[q].n; ++a) {
                    int64_t sg = inbox[q].v[a];
                    /* the source neuron of segment sg */
                    int64_t lo = 0, hi = M - 1;
                    while (lo < hi) {
                        int64_t mid = (lo + hi + 1) / 2;
                        if (h->seg_ptr[mid] <= sg) lo = mid; else hi = mid - 1;
                    }
                    if (np < pairs_cap) pairs[np] = ((uint64_t)lo << 32) | (uint32_t)q;
                    ++np;
                }
            *n_pairs = np;
        }
        /* 3. delivery by destination partition */
        uint64_t ev = 0;
        for (int32_t q = 0; q < P; ++q)
            for (int64_t a = 0; a < inbox[q].n; ++a) {
                int64_t sg = inbox[q].v[a];
                int64_t lo = 0, hi = M - 1;
                while (lo < hi) {
                    int64_t mid = (lo + hi + 1) / 2;
                    if (h->seg_ptr[mid] <= sg) lo = mid; else hi = mid - 1;
                }
                int64_t i = lo, b = h->syn_ptr[i];
                for (uint32_t x = 0; x < h->seg_len[sg]; ++x) {
                    int64_t e = b + h->ord[b + h->seg_beg[sg] + x];
                    int64_t j = h->tgt[e];
                    int64_t sl = (t + h->d[e]) % D;
                    int32_t *c = ring + sl * M + j;
                    *c = (int32_t)((uint32_t)*c + (uint32_t)(int32_t)h->w[e]);
                    ++ev;
                }
            }
        /* 4. message counts from their definitions */
        if (counts) {
            counts[OC_STEPS] += 1;
            counts[OC_SPIKES] += (uint64_t)S;
            counts[OC_EVENTS] += ev;
            for (int32_t p = 0; p < P; ++p)
                for (int64_t a = 0; a < outq[p].n; ++a) {
                    int64_t i = outq[p].v[a];
                    int32_t hv_ = h->vn_of_part[p];
                    for (int64_t e = h->syn_ptr[i]; e < h->syn_ptr[i + 1]; ++e) {
                        int32_t q = h->part_of[h->tgt[e]];
                        mark[q] = 1;
                        gmark[h->vn_of_part[q]] = 1;
                    }
                    for (int32_t q = 0; q < P; ++q) {
                        if (!mark[q]) continue;
                        int32_t g = h->vn_of_part[q];
                        if (q != p) counts[OC_DIRECT]++;
                        if (g != hv_) counts[OC_DIRECT_XVN]++;
                        if (g == hv_) {
                            if (q == p) counts[OC_L2_LOCAL]++; else counts[OC_L2_PEER]++;
                        } else {
                            if (q == h->relay[g * P + p]) counts[OC_L2_RELAY_LOCAL]++;
                            else counts[OC_L2_RELAY_REMOTE]++;
                        }
                    }
                    for (int32_t g = 0; g < h->n_vn; ++g) {
                        if (!gmark[g]) continue;
                        if (g == hv_) counts[OC_L1_LOCAL]++; else counts[OC_L1_XVN]++;
                    }
                    memset(mark, 0, (size_t)P);
                    memset(gmark, 0, (size_t)h->n_vn);
                }
        }
    }
    for (int32_t p = 0; p < P; ++p) { free(outq[p].v); free(inbox[p].v); }
    free(outq); free(inbox); free(mark); free(gmark);
    return rc;
}

/* Number of (neuron, destination partition) segments built by or_create. */
int64_t or_num_segments(void *hv)
{
    or_net *h = (or_net *)hv;
    return h ? h->seg_ptr[h->M] : -1;
}

/* Relays of a policy (0 per group, 1 per partition, 2 balanced; see the
 * header) for the network's mapping; the two-level counts of later runs use
 * them.  out (may be NULL) receives relay[g * P + p].  Returns 0, -1 on a
 * bad policy. */
int or_set_relay_policy(void *hv, int32_t policy, int32_t *out)
{
    or_net *h = (or_net *)hv;
    if (!h || policy < 0 || policy > 2) return -1;
    const int32_t P = h->P, n_vn = h->n_vn;
    const int32_t *vp = h->vn_of_part;
    for (int32_t g = 0; g < n_vn; ++g)
        for (int32_t p = 0; p < P; ++p)
            h->relay[g * P + p] = vp[p] == g ? -1
                                  : policy == 0 ? relay_of(vp, P, g, vp[p])
                                                : member_of(vp, P, g, rank_in_group(vp, p));
    if (policy == 2) {
        /* static loads: (neuron of p, partition of g) pairs with synapses */
        int64_t *load = calloc((size_t)n_vn * (size_t)P, sizeof(int64_t));
        for (int64_t i = 0; i < h->M; ++i) {
            int32_t p = h->part_of[i];
            for (int64_t sg = h->seg_ptr[i]; sg < h->seg_ptr[i + 1]; ++sg) {
                int32_t g = vp[h->seg_q[sg]];
                if (g != vp[p]) load[(int64_t)g * P + p]++;
            }
        }
        int32_t *mem = malloc(sizeof(int32_t) * (size_t)P);
        int64_t *acc = malloc(sizeof(int64_t) * (size_t)P);
        char *done = malloc((size_t)P);
        for (int32_t g = 0; g < n_vn; ++g) {
            int32_t nm = 0;
            for (int32_t p = 0; p < P; ++p)
                if (vp[p] == g) { mem[nm] = p; acc[nm] = 0; ++nm; }
            memset(done, 0, (size_t)P);
            for (;;) {
                /* the heaviest unassigned source (ties: lower index) */
                int32_t best = -1;
                for (int32_t p = 0; p < P; ++p) {
                    int64_t l = load[(int64_t)g * P + p];
                    if (vp[p] == g || done[p] || l == 0) continue;
                    if (best < 0 || l > load[(int64_t)g * P + best]) best = p;
                }
                if (best < 0) break;
                done[best] = 1;
                int32_t k = 0;
                for (int32_t m = 1; m < nm; ++m)
                    if (acc[m] < acc[k]) k = m;
                acc[k] += load[(int64_t)g * P + best];
                h->relay[g * P + best] = mem[k];
            }
        }
        free(load); free(mem); free(acc); free(done);
    }
    if (out) memcpy(out, h->relay, sizeof(int32_t) * (size_t)n_vn * (size_t)P);
    return 0;
}

/* Single-precision alpha = fl32(exp(-dt/tau)) as the oracle uses it. */
float or_alpha(double dt_ms, double tau_ms)
{
    return (float)exp(-dt_ms / tau_ms);
}

/* Poisson drive arrivals k_j(t) for neurons j0 .. j0+n-1 at step t. */
int or_drive_draws(uint64_t seed, double lambda, int64_t j0, int64_t n, int64_t t, int32_t *out)
{
    uint64_t th[OR_PTAB];
    int32_t len;
    if (or_poisson_table(lambda, th, &len)) return -1;
    for (int64_t a = 0; a < n; ++a)
        out[a] = poisson_draw(th, len, drive_word(seed, (uint32_t)(j0 + a), (uint32_t)t));
    return 0;
}
