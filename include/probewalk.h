/*
 * probewalk.h — C ABI of the GB300 ProbeWalk library (libprobewalk.so).
 *
 * ProbeWalk (arXiv 2512.05460) estimates the squared biharmonic distance
 *     beta(s,t) = || L^+ (e_s - e_t) ||^2                  (Definition 2.1, Eq. exact)
 * of two nodes of an undirected graph to a relative error eps (Problem 1) by
 * Algorithm 1: for K = B*G Paired-Sign Probes z^(k) (Definition 3.1, generated
 * statelessly as in Section 3.3) it runs R independent pairs of length-L random
 * walks from s and t, forms U_p = sum_i z_{X_i}/d_{X_i} - sum_i z_{~X_i}/d_{~X_i}
 * (Eq. hatphi-def), the U-statistic Q_R = (S1^2 - S2) / (R(R-1)) (Eq. Q-Ustat)
 * with S1 = sum_p U_p and S2 = sum_p U_p^2 evaluated exactly and rounded once
 * to FP64 (so independent of the order in which replicas finish), and returns
 * the median of the G block means of B probes each (Eq. final-estimator).  The returned value estimates the truncated
 * distance beta^(L) (Lemma 2.3), which is within eps*beta/2 of beta when L is
 * chosen by Eq. uni_l / Theorem 3.8.
 *
 * Conventions for every function:
 *   - No exception crosses this boundary.  Each function returns a pw_status;
 *     on failure pw_last_error() returns a message for the calling thread.
 *   - "host" pointers are ordinary CPU memory owned by the caller, read or
 *     written only during the call.  "device" pointers are CUDA global memory
 *     on the graph's device, owned by the caller.
 *   - The library owns the device copy of the graph and its scratch memory.
 *   - All node ids are 0-based.  Integers are little-endian native types.
 *   - A call that takes a stream (cudaStream_t passed as void*) is ordered on
 *     that stream; host-pointer calls synchronise before returning.
 *   - Calls on one pw_graph are serialised by an internal lock.
 *   - Results depend only on (graph, s, t, eps, L, seed, params): a query gives
 *     the same estimate alone or inside any batch.
 */
#ifndef PROBEWALK_H_
#define PROBEWALK_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PW_OK = 0,
  PW_PENDING = 1,        /* server ticket not finished yet */
  PW_ERR_ARG = -1,       /* invalid argument (node id, eps, L, sizes, null pointer) */
  PW_ERR_GRAPH = -2,     /* graph not sorted/simple/symmetric/connected, or an isolated node */
  PW_ERR_NOMEM = -3,     /* device or host allocation failed, or admission capacity exceeded */
  PW_ERR_CUDA = -4,      /* a CUDA runtime call failed (message in pw_last_error) */
  PW_ERR_TIMEOUT = -5,   /* a bounded wait expired */
  PW_ERR_CANCELLED = -6, /* server query cancelled or server shut down */
  PW_ERR_FULL = -7,      /* server queue full */
  PW_ERR_INTERNAL = -8   /* a self-check failed (pw_server_tune: variants gave different estimates) */
} pw_status;

/* Budget modes.  THEORY is Algorithm 1's parameter line (Eqs. B-value,
 * G-value, R-value, K-value).  The paper's experiments do not state the K and
 * R they used; SCALED scales THEORY's B and R by c_B and c_R; FIXED takes B, G,
 * R as given; PILOT (default) keeps G, takes B = ceil(c_B / eps^2)
 * (c_B = 0.5 by default: the smallest of {0.25, 0.5, 1, 2, 4} that kept >= 95% of
 * held-out queries within eps on the tiny and BA workloads) and sets R
 * from Lemma 3.7's sufficient condition R >= 4 sigma^2 / theta, with sigma^2 and
 * theta estimated by a pilot of K0 probes x R0 replicas on reserved streams
 * (theta floored by theta_0 = (1/8)(1 - eps/2)(1/d_s + 1/d_t)^2 from the proof of
 * Theorem 3.8), rounded up to a multiple of 32 and clamped to [32, R_max]. */
enum { PW_BUDGET_PILOT = 0, PW_BUDGET_THEORY = 1, PW_BUDGET_SCALED = 2, PW_BUDGET_FIXED = 3, PW_BUDGET_ADAPTIVE = 4 };
/* ADAPTIVE (the paper has no counterpart: B per query from the variance of
 * Q_R, Lemma 3.7, and the median of Eq. final-estimator): R as in PILOT; the
 * probes run in two stages.  The first stage runs B1 = ceil(B_P/4) probes per
 * block (B_P: PILOT's B); from those G B1 values of Q_R the query keeps the
 * smallest B* at which z standard errors of the median of means,
 * sqrt(pi/2) sd(Q) / sqrt(G B*), fit in eps theta (theta = max(mean Q,
 * theta_0)):  B* = ceil((pi/2) z^2 s^2 / (G eps^2 theta^2)) clamped to
 * [B1, cap B_P].  The second stage runs probes G B1 .. G B* - 1, and the
 * estimate is the median of the G contiguous blocks of B* probes.  Defaults
 * z = 3, cap = 2 (calibrated on 1024 queries per synthetic workload; the
 * variance estimate misjudges heavy-tailed Q_R, so on R-MAT graphs it does not
 * save work safely).  Not available in servers. */

/* Parameters; an all-zero struct selects every default. */
typedef struct pw_params {
  double delta;            /* failure probability of Theorem 3.8; 0 -> 0.01 */
  int32_t budget_mode;     /* PW_BUDGET_*; default PILOT */
  int32_t pilot_K0;        /* PILOT probes; 0 -> 64 */
  int32_t pilot_R0;        /* PILOT replicas per probe, 2..32; 0 -> 32 */
  int32_t reserved0;
  double c_B;              /* 0 -> 0.5 in PILOT mode (calibrated), 1.0 otherwise */
  double c_R;              /* 0 -> 1.0 */
  uint64_t B, G, R;        /* FIXED mode values (B >= 1, G >= 1, R >= 2) */
  uint64_t R_max;          /* PILOT / SCALED clamp; 0 -> 4096 */
  uint64_t seed;           /* global seed for queries that pass no seed */
  int32_t walk_mode;       /* 0 auto (graph cost model, see pw_autotune); 1 probe entries evaluated per visit; 2 per-probe shared-memory table */
  int32_t reserved1;
  double z;                /* ADAPTIVE: normal quantile of the stopping rule; 0 -> 3 */
  double cap;              /* ADAPTIVE: the most probes per block as a multiple of PILOT's B; 0 -> 2 */
} pw_params;

typedef struct pw_graph pw_graph;
typedef struct pw_server pw_server;

/* ---- graph ---------------------------------------------------------------
 * pw_graph_load: validate an undirected simple graph given as CSR and upload
 * it to CUDA device `device`.  row_ptr[0..n] (host) are row offsets with
 * row_ptr[0] = 0 and row_ptr[n] = nnz; col_idx[0..nnz) (host) are neighbour
 * ids, each row strictly increasing (so no duplicates), no self-loops, every
 * edge present in both directions, every node of degree >= 1, the graph
 * connected (Section 2.1).  Requires 2 <= n < 2^31 and nnz < 2^31.  The arrays
 * are copied; the caller keeps ownership.  flags: bit 0 skips the O(n + m)
 * connectivity check; bits 1 and 2 force the walks' graph layout, fused
 * 16-byte neighbour records (bit 1: one gather per walk step) or col_idx plus
 * 16-byte node records (bit 2: two smaller gathers per step); by default the
 * split layout is used when the fused records would take more than 64 MiB
 * (half of the L2) while col_idx plus node records take at most 160 MiB, and
 * the fused records otherwise.  Both give the same walks.  Returns
 * PW_ERR_GRAPH if a check fails.
 * On success *out holds a handle to free with pw_graph_free. */
pw_status pw_graph_load(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, int64_t nnz,
                        int32_t device, uint32_t flags, pw_graph** out);
/* Same with 32-bit row offsets. */
pw_status pw_graph_load32(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t nnz,
                          int32_t device, uint32_t flags, pw_graph** out);
/* Releases the device copy and scratch of a loaded graph (NULL is a no-op).
 * No call on g may be in flight; servers on g must be destroyed first. */
void pw_graph_free(pw_graph* g);
/* L2 access-policy window of the walk launches on g (an implementation choice:
 * the paper says nothing about caching; estimates do not depend on it).
 * which: 0 none (the default); 1 the array every walk step gathers from (the
 * fused records, or col_idx on the split layout), uniformly at stationarity;
 * 2 the split layout's node records, gathered in proportion to degree, so
 * hub nodes' records most often.  The window covers the array, up to the
 * device's maximum window size; the context's persisting-L2 set-aside is
 * raised to min(device maximum, window bytes), and the window's hit ratio is
 * set-aside / window bytes, so that the lines marked persisting fit; the
 * others are streaming.  Every later walk-kernel and server launch on g
 * carries the window as a launch attribute (the caller's streams are not
 * modified).  which = 0 returns the persisting lines to normal and the
 * set-aside to its value before; pw_graph_free does the same.  Call it with
 * no call on g in flight and no server on g.  PW_ERR_ARG for which outside
 * {0, 1, 2} or 2 on the fused layout; PW_ERR_CUDA when the device has no
 * persisting L2 or the set-aside cannot be set.  pw_autotune times the
 * windows and keeps the fastest. */
pw_status pw_graph_set_l2_window(pw_graph* g, int32_t which);
/* Graph facts: n, nnz (directed entries), minimum and maximum degree,
 * bipartite flag (1 when 2-colourable: the paper assumes non-bipartite,
 * Section 2.1; estimates then target beta^(L) only).  Any output may be NULL. */
pw_status pw_graph_info(const pw_graph* g, int64_t* n, int64_t* nnz, int32_t* d_min, int32_t* d_max,
                        int32_t* bipartite);

/* ---- budget ----------------------------------------------------------------
 * Budget of one query (Algorithm 1, line 1): writes B, G, K = B*G, R.  In
 * PILOT and ADAPTIVE modes this runs the pilot walks on the GPU; ADAPTIVE
 * reports its first stage (B = ceil(B_PILOT / 4)).  seed: host pointer to the
 * query's 64-bit seed, or NULL for pw_default_seed(params->seed, s, t, eps, L).
 * s == t gives all zeros. */
pw_status pw_budget(pw_graph* g, int64_t s, int64_t t, double eps, int32_t L, const uint64_t* seed,
                    const pw_params* params, uint64_t* B, uint64_t* G, uint64_t* K, uint64_t* R);

/* Default per-query seed: Philox4x32-10 keyed by (params seed XOR bits of eps)
 * over the counter (s, t, L, 0x5EED); first two output words.  A convention of
 * this library (the paper fixes no seeding): it makes a query's estimate
 * depend only on its own arguments, alone or in any batch. */
uint64_t pw_default_seed(uint64_t global_seed, int64_t s, int64_t t, double eps, int32_t L);

/* ---- queries ---------------------------------------------------------------
 * pw_query: Algorithm 1 for one query (Problem 1: beta(s,t) to relative error
 * eps with probability 1 - delta), one pipeline of launches (the "one query per
 * launch" form): budget (line 1), the K x R walk pairs and their U_p
 * (Eq. hatphi-def), Q_R per probe (Eq. Q-Ustat) and the median of the G block
 * means (Eq. final-estimator).  eps in (0,1), L >= 0, 0 <= s,t < n.
 * *beta_hat (host) receives the estimate of beta^(L)(s,t); it may be negative
 * for tiny distances (the U-statistic is unbiased, not positive).  s == t
 * returns exactly 0. */
pw_status pw_query(pw_graph* g, int64_t s, int64_t t, double eps, int32_t L, const uint64_t* seed,
                   const pw_params* params, double* beta_hat);

/* pw_query_batch: Algorithm 1 for `count` independent queries (host arrays of
 * length count; seeds may be NULL for default seeds), each with the result
 * pw_query gives it.  The walks of all queries run in two persistent launches
 * (the probe-table kernel for queries whose probes visit more nodes than a
 * table costs to build, the per-visit kernel for the rest; the choice is made
 * per query on the device after the pilot), and the host does not wait for the
 * device between the input copy and the result copy.  beta_hat and
 * per_query_status (host) receive the results; the return value is PW_OK when
 * the batch ran, even if some queries have a per-query error status.
 * count == 0 is a no-op. */
pw_status pw_query_batch(pw_graph* g, int64_t count, const int64_t* s, const int64_t* t, const double* eps,
                         const int32_t* L, const uint64_t* seeds, const pw_params* params, double* beta_hat,
                         int32_t* per_query_status);

/* pw_query_batch_device: as pw_query_batch with every array in device memory
 * and the work ordered on `stream` (a cudaStream_t, NULL for the legacy default
 * stream).  The call returns after the launches are enqueued; it synchronises
 * `stream` once, after the budget kernel, to read the batch's total probe count
 * K, which sizes its scratch memory (8 bytes of Q_R plus 96 of accumulator per
 * probe; nothing per replica). */
pw_status pw_query_batch_device(pw_graph* g, int64_t count, const int64_t* d_s, const int64_t* d_t,
                                const double* d_eps, const int32_t* d_L, const uint64_t* d_seeds,
                                const pw_params* params, double* d_beta_hat, int32_t* d_status, void* stream);

/* pw_query_batch_noalloc: the device-array batch of pw_query_batch_device for
 * callers that must not allocate device memory while they serve queries (for
 * example a request path where allocator calls, which can block and
 * synchronise the device, are forbidden).  The paper has no counterpart: this
 * is a deployment variant of the same computation, with the same results.
 * The call makes no cudaMalloc, cudaFree or allocating library call: all of
 * its scratch (query plans, offsets, counters, pilot sums, the Q_R values and
 * probe accumulators: about 104 bytes per probe) lives in one static 64 MiB
 * device array that the library holds on every GPU that loads it, until the
 * process exits.  A batch whose scratch exceeds 64 MiB is rejected with
 * PW_ERR_NOMEM (at eps = 0.1 and delta = 0.01 a query has K = 1,850 probes,
 * about 193 KB, so about 340 such queries fit per call; K grows as 1/eps^2).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the array and clears the counters that must start at
 * zero; calls that overlap on the GPU (other streams or threads) race on it.
 * Arguments, layout and ordering on `stream` are those of
 * pw_query_batch_device; like it, the call synchronises `stream` once, after
 * the budget kernel. */
pw_status pw_query_batch_noalloc(pw_graph* g, int64_t count, const int64_t* d_s, const int64_t* d_t,
                                 const double* d_eps, const int32_t* d_L, const uint64_t* d_seeds,
                                 const pw_params* params, double* d_beta_hat, int32_t* d_status, void* stream);

/* ---- stabilization rule (Section 4.3) ----------------------------------------
 * pw_query_stabilized: choose L per query as the paper does on graphs whose
 * spectral gap is unknown: starting from L = 1, double L (capped at L_max)
 * and accept L_stop = 2L as soon as |beta(2L) - beta(L)| <= (eps/2) |beta(2L)|;
 * when L reaches L_max without that, the estimate at L_max is returned with
 * L_stop = L_max.  Every level is a full run of Algorithm 1 keyed by
 * pw_level_seed(seed, L) (seeds: host array or NULL for
 * pw_default_seed(params->seed, s, t, eps, L_max)); all queries still doubling
 * run in one batch per level.  Host arrays of length count: s, t, eps (in),
 * beta_hat, L_stop, per_query_status (out).  L_max >= 2.  s == t gives 0. */
pw_status pw_query_stabilized(pw_graph* g, int64_t count, const int64_t* s, const int64_t* t, const double* eps,
                              int32_t L_max, const uint64_t* seeds, const pw_params* params, double* beta_hat,
                              int32_t* L_stop, int32_t* per_query_status);
/* Seed of level L of a stabilized query: first two words of Philox4x32-10
 * keyed by `seed` over the counter (L, 0, 0, 0x57AB).  A convention of this
 * library (Section 4.3 does not say how levels are seeded): levels are
 * independent runs. */
uint64_t pw_level_seed(uint64_t seed, int32_t L);

/* ---- truncated series (Lemma 2.3) --------------------------------------------
 * pw_series_batch: the deterministic beta^(L)(s,t) = ||h||^2 - (1^T h)^2 / n
 * with h = sum_{i=0}^{L} P^i D^{-1} (e_s - e_t) (Eq. tr-beta-exp-Liu), the
 * quantity the paper's PUSH baseline computes, by L sparse matrix-vector
 * products on the GPU, 32 queries of equal L per pass (each pass a CUDA graph,
 * captured once per distinct L in a call and replayed).  The steps run in
 * double-float arithmetic (FP32 pairs, 48-bit significand; GB300's FP64 rate
 * is a small fraction of its FP32 rate) and beta is reduced in FP64; results
 * agree with an FP64 evaluation to 1e-9 relative (tested; 3.3e-14 measured at
 * L = 200 on a 10^5-node graph).  Host arrays of
 * length count: s, t, L (in), beta_L (out).  s == t gives 0. */
pw_status pw_series_batch(pw_graph* g, int64_t count, const int64_t* s, const int64_t* t, const int32_t* L,
                          double* beta_L);

/* ---- sharded query (one query split across GPUs) ---------------------------
 * pw_query_blocks: the median-of-means blocks [g_begin, g_end) of one query
 * (Eq. final-estimator before the median): the same budget and the same
 * walks (probe indices keep their values) as the whole query, restricted to
 * probes g_begin*B .. g_end*B - 1.  block_means (host, g_end - g_begin) gets
 * the block means.  0 <= g_begin < g_end <= G; s != t.  Ranks that own
 * disjoint block ranges gather their means and pw_block_median gives the
 * estimate of the unsharded query, bit for bit.  Not for ADAPTIVE budgets
 * (their B is known only after the first stage): PW_ERR_ARG. */
pw_status pw_query_blocks(pw_graph* g, int64_t s, int64_t t, double eps, int32_t L, const uint64_t* seed,
                          const pw_params* params, int64_t g_begin, int64_t g_end, double* block_means);
/* pw_block_median: median of G block means (host arrays; mean of the two
 * middle values for even G), the last step of Eq. final-estimator. */
pw_status pw_block_median(const double* block_means, int64_t G, double* out);

/* ---- server (continuous batching) ----------------------------------------
 * Serving Algorithm 1 (the paper has no counterpart: a deployment of the same
 * computation).  Each query's estimate equals pw_query's for the same
 * arguments and params, alone or in any mix.  A server keeps the graph and the
 * per-query accumulators on the device and runs a persistent kernel fed by a
 * device work queue.  Queries are admitted while their accumulator memory
 * (8 bytes per probe plus 16 per pilot probe) fits in accum_bytes (at least
 * 1 MiB); later ones wait in a host queue, and a query that needs more than
 * accum_bytes alone fails with PW_ERR_NOMEM.  Requires G <= 2048 (delta above
 * about 1e-111; a larger FIXED G fails the query with PW_ERR_ARG).
 * pw_server_create: allocates the server on g's device and starts its
 *   scheduler thread; *out receives the handle.
 * pw_server_submit: queues one query (arguments as pw_query; seed NULL for
 *   the default seed) and returns its ticket in *ticket; never blocks on the
 *   GPU.  PW_ERR_CANCELLED once destruction has begun, PW_ERR_FULL past 2^24
 *   queued requests.
 * pw_server_poll: PW_OK with *beta_hat when the ticket is done (the result is
 *   then delivered and removed), PW_PENDING before, PW_ERR_ARG for an unknown
 *   ticket or one already delivered by poll or collect; a query that failed
 *   returns its error status (also delivering it). */
pw_status pw_server_create(pw_graph* g, const pw_params* params, size_t accum_bytes, pw_server** out);
pw_status pw_server_submit(pw_server* srv, int64_t s, int64_t t, double eps, int32_t L, const uint64_t* seed,
                           uint64_t* ticket);
pw_status pw_server_poll(pw_server* srv, uint64_t ticket, double* beta_hat);
/* Move up to `cap` finished results out of the server (host arrays): ticket,
 * estimate, per-query status and latency from submit to completion (ms, as
 * seen by the scheduler thread); *count receives how many were written.  A
 * collected ticket is delivered: pw_server_poll then reports PW_ERR_ARG. */
pw_status pw_server_collect(pw_server* srv, int64_t cap, uint64_t* tickets, double* beta_hat, int32_t* status,
                            double* latency_ms, int64_t* count);
/* Server tuning (an implementation choice: every policy gives the same
 * estimates).  After a query's pilot the server runs its probes either with a
 * per-probe shared-memory table of z or evaluating z at each visit; the
 * choice follows a cost model {table cost per probe, saving per visit}.
 * pw_server_tune runs the sample (host arrays as in pw_query_batch; seeds may
 * be NULL) through the server as a burst, once to warm up and once timed.
 * When the graph's probe table fits in shared memory it times each policy:
 * 0 the default model (n Feistel passes per table against 2.5 per visit), 1
 * the graph's model fitted by pw_autotune on the batch kernels (skipped when
 * the graph is untuned), 2 every query per-visit, 3 every query with the
 * table, and keeps the fastest.  When the table does not fit, every policy
 * runs the same per-visit jobs; it then times the server kernel at 2 and at 3
 * resident blocks per SM (the second with fewer registers, some spilled) and
 * keeps the faster.  Queries/s are reported for each timed case (0 for one
 * not timed).  The sums being exact, every case must give the same estimates
 * bit for bit; the tuner compares them and returns PW_ERR_INTERNAL if they
 * differ.  Call it on an idle server: the sample's tickets are consumed by
 * the tuner. */
typedef struct pw_server_tune_result {
  double queries_per_s[4];  /* per policy (table servers); [0] the kept variant otherwise */
  double occupancy_qps[2];  /* per-visit-only servers: at 2 and at 3 blocks/SM */
  int32_t policy;           /* the policy kept */
  int32_t occupancy;        /* resident blocks/SM of the kernel kept (4 for the table kernel) */
} pw_server_tune_result;
pw_status pw_server_tune(pw_server* srv, int64_t count, const int64_t* s, const int64_t* t, const double* eps,
                         const int32_t* L, const uint64_t* seeds, pw_server_tune_result* out);
/* Wait up to timeout_ms for every submitted ticket; PW_ERR_TIMEOUT otherwise. */
pw_status pw_server_drain(pw_server* srv, int64_t timeout_ms);
/* Cancels requests still waiting for admission (their tickets get
 * PW_ERR_CANCELLED), waits for the admitted ones to finish, stops the kernel
 * and frees the server.  NULL is a no-op. */
pw_status pw_server_destroy(pw_server* srv);

/* ---- debug / parity (tests) -------------------------------------------------
 * pw_debug_philox: Philox4x32-10 evaluated on the device (host arrays:
 * ctr[4], key[2], out[4]). */
pw_status pw_debug_philox(pw_graph* g, const uint32_t* ctr, const uint32_t* key, uint32_t* out);
/* pw_debug_probe: probe entries z^(k)_v for every node v (host int8 array of
 * n) of probe k under stream tag `tag` (3 main, 4 pilot) of the query keyed by
 * seed; returns the parity parameter r in *r (host, may be NULL). */
pw_status pw_debug_probe(pw_graph* g, uint64_t seed, uint32_t k, uint32_t tag, int8_t* z, int32_t* r);
/* pw_debug_gather_peak: throughput ceiling of the walk's memory side on this
 * graph: dependent random gathers with the walk's access per step (fused
 * layout: one 16-byte record uniform over the record array; split layout: one
 * col_idx entry uniform over col_idx, then the node record it names), 8 chains
 * per thread, full occupancy, no other work, best of 3 launches of `iters`
 * steps per chain.  *sectors_per_s (host) receives steps/s (each step reads one
 * 32-byte sector per gather). */
pw_status pw_debug_gather_peak(pw_graph* g, int32_t iters, double* sectors_per_s);
/* pw_debug_walk: trajectory X_0..X_L (host int64 array of L+1) of walk
 * `walk_id` under stream tag `tag` (1 main, 2 pilot). */
pw_status pw_debug_walk(pw_graph* g, int64_t start, int32_t L, uint64_t seed, uint64_t walk_id, uint32_t tag,
                        int64_t* trajectory);
/* pw_debug_query: pw_query that also returns (host arrays, each may be NULL)
 * budget[4] = (B, G, K, R), pilot[3] = (sigma2_hat, q_bar, theta_hat), q[K]
 * (Q_R per probe), u[K*R] (U_p, probe-major) and visits[n] (uint32 visit
 * counts of all main walks, X_0 included).  q_cap and u_cap are the capacities
 * of q and u in elements; PW_ERR_ARG if too small. */
pw_status pw_debug_query(pw_graph* g, int64_t s, int64_t t, double eps, int32_t L, const uint64_t* seed,
                         const pw_params* params, double* beta_hat, uint64_t* budget, double* pilot, double* q,
                         int64_t q_cap, float* u, int64_t u_cap, uint32_t* visits);
/* pw_debug_exact_sum: S1 = sum u[i] and S2 = sum u[i]^2 (host array of n FP32
 * values; results to host) through the device accumulator that the walk
 * kernels use for each probe: exact integer digits, rounded once to the
 * nearest double, ties to even.  Values must be multiples of 2^-54 below 2^33
 * in magnitude, as every replica value U_p is (1 <= d < 2^31, L < 2^31). */
pw_status pw_debug_exact_sum(pw_graph* g, const float* u, int64_t n, double* S1, double* S2);
/* pw_debug_batch_probe_q: run pw_query_batch and also copy out Q_R of
 * selected probes (host arrays of length n_sel: query index, probe index ->
 * q_sel), and the (K, R) of every query (host uint64 [count][2]). */
pw_status pw_debug_batch_probe_q(pw_graph* g, int64_t count, const int64_t* s, const int64_t* t,
                                 const double* eps, const int32_t* L, const uint64_t* seeds,
                                 const pw_params* params, double* beta_hat, int32_t* per_query_status,
                                 uint64_t* KR, int64_t n_sel, const int64_t* sel_query, const int64_t* sel_probe,
                                 double* q_sel);

/* ---- instrumentation -------------------------------------------------------
 * When enabled, batch calls on `g` record CUDA events on their launch stream
 * around the walk kernel and the finishing kernels.  pw_profile with out !=
 * NULL waits for the recorded events and writes the accumulated figures;
 * reset != 0 clears them afterwards.  transitions = sum over queries of
 * 2 K R L, the walk steps Algorithm 1 performs (pilot steps counted apart). */
typedef struct pw_profile_stats {
  double walk_ms;              /* main walk-kernel launches, summed */
  double pilot_ms;             /* pilot walk-kernel launches, summed */
  double finish_ms;            /* per-probe U-statistic + median-of-means kernels */
  uint64_t walk_launches;
  uint64_t transitions;
  uint64_t pilot_transitions;
  uint64_t queries;
  int32_t walk_mode;           /* walk kernels of the last batch: 1 per-visit probe evaluation, 2 probe table, 3 both */
  int32_t layout;              /* the graph's walk layout: 1 fused records, 2 col_idx + node records */
  double series_ms;            /* pw_series_batch passes (32 queries each), summed */
  uint64_t series_steps;       /* sparse steps of those passes: L + 1 per pass */
} pw_profile_stats;
pw_status pw_profile(pw_graph* g, int32_t enable, int32_t reset, pw_profile_stats* out);

/* Walk-kernel autotuner (implementation choice; the paper prescribes what the
 * walks compute, Algorithm 1, not which kernel runs them).  Both walk kernels
 * give bit-identical results, so the choice only changes speed.
 *
 * Runs the caller's sample batch (host arrays as in pw_query_batch, seeds may
 * be NULL, each query's s, t, L) with a FIXED budget of B = 16 probes per
 * block (8 queries give 4,736 probes at G = 37, enough to fill the GPU;
 * the policy and window checks below run at the caller's own budget, where a
 * sample of 32 queries or more stands for the batch far better than 8),
 * params' G, and R = 1024 replicas, each run after one untimed
 * warm-up: the per-visit kernel in its two register variants (compiler's
 * choice, or capped for 3 blocks of 256 per SM), keeping the faster; the
 * per-probe shared-memory table with blocks of 256, 512 and 1024 threads,
 * keeping the fastest; and that table kernel again at R = 256 (the same
 * probes, a quarter of the visits).  The kept variants are stored in the
 * graph and used by every later batch.  From the main walk kernels'
 * CUDA-event time of the kept runs it fits
 *   per-visit:  t = visits * visit_ns
 *   table:      t = probes * table_probe_ns + visits * table_visit_ns
 * (visits = 2 K R (L+1) summed over the batch) and stores the costs in the
 * graph: from then on walk_mode 0 (auto) in pw_query* uses the table when
 * probes * table_probe_ns < visits * (visit_ns - table_visit_ns).  Last,
 * the sample runs once more at the caller's own budget under three policies
 * (that model per query, every query per-visit, every query on the table),
 * and walk_mode 0 follows the fastest from then on; a single-kernel policy
 * within 1 % of the model is preferred to it (one walk launch per batch
 * instead of two).  With the table unavailable, policy 0 and 1 coincide.  Servers keep their own policy (see
 * pw_server_tune).  Costs are whole-GPU nanoseconds.  When the graph's table
 * does not fit in shared memory (one bit per node in at most 200 KB:
 * n > 1,638,336) only the per-visit runs are made and table_available = 0;
 * the model then always picks per-visit.  Finally the sample runs at the
 * caller's budget under each L2 window of pw_graph_set_l2_window (none, the
 * gathered array, and on the split layout the node records; the windows the
 * device cannot set are skipped); the fastest window is kept if it beats no
 * window by 2 % or more, else none.  A kept window raises the CUDA
 * context's persisting-L2 set-aside, which the rest of the process shares,
 * until pw_graph_set_l2_window(g, 0) or pw_graph_free(g).  Call it with no
 * server on g (server launches carry the graph's window).  params as in
 * pw_query (its walk_mode is ignored).  Errors as pw_query_batch; the
 * estimates of the runs are discarded. */
typedef struct pw_tune_result {
  double visit_ns;         /* per-visit kernel, ns per visit */
  double table_visit_ns;   /* table kernel, ns per visit (0 when unavailable) */
  double table_probe_ns;   /* table kernel, ns per probe for the table build (0 when unavailable) */
  double sample_ms[3];     /* walk-kernel time of the kept runs (per-visit; table at R = 1024; table at R = 256) */
  int32_t table_available; /* 1 when the probe table fits in shared memory */
  int32_t sample_mode;     /* walk kernel the fitted model picks for the sample: 1 per-visit, 2 table */
  int32_t visit_occupancy; /* per-visit kernel variant kept: 1 compiler-chosen registers, 3 capped for 3 blocks/SM */
  int32_t table_threads;   /* table-kernel block size kept: 256, 512 or 1024 (0 when unavailable) */
  double policy_ms[3];     /* walk time of the sample at the caller's budget: per-query model, all per-visit, all table */
  int32_t policy;          /* the policy walk_mode 0 now follows: 0 per-query model, 1 all per-visit, 2 all table */
  int32_t l2_window;       /* the L2 window kept (pw_graph_set_l2_window): 0 none, 1 gathered array, 2 node records */
  double window_ms[3];     /* walk time of the sample at the caller's budget under window 0, 1, 2 (0: not timed) */
} pw_tune_result;
pw_status pw_autotune(pw_graph* g, int64_t count, const int64_t* s, const int64_t* t, const double* eps,
                      const int32_t* L, const uint64_t* seeds, const pw_params* params, pw_tune_result* out);

/* Kernel launches issued by this thread since the last call (instrumentation). */
uint64_t pw_launch_count(int reset);
/* Message describing the last error on this thread ("" if none). */
const char* pw_last_error(void);
/* Library version string. */
const char* pw_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PROBEWALK_H_ */
