// Query pipeline of Algorithm 1 on the device:
//   budget (line 1) -> [pilot walks + pilot budget] -> per-query walk kernel and
//   offsets -> walk kernels (lines 2-11), each finishing its probes' Q_R
//   (lines 12-14) from exact replica sums -> median of block means (lines 16-20).
// No replica value is stored: a probe's S1 and S2 are exact integer sums
// (pw_exact.cuh), reduced in registers, warp shuffles and atomics in any order.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pw_budget.cuh"
#include "pw_device.cuh"
#include "pw_exact.cuh"
#include "pw_internal.h"
#include "pw_walk.cuh"

namespace pw {

constexpr int kWalkThreads = 256;

// Exact S1/S2 digits of a probe run by the per-visit kernel, whose tiles may
// land on any warp of the grid; `done` counts the probe's finished tiles.
struct ProbeAcc {
  unsigned long long d[kSumDigits];
  unsigned int done;
  unsigned int pad;
};

// ---------------------------------------------------------------------------
// Budget of every query (Algorithm 1 line 1).  PILOT queries get their pilot
// plan here and their R in pilot_budget_kernel.
// ---------------------------------------------------------------------------
__global__ void budget_init_kernel(int64_t nq, const int64_t* __restrict__ qs, const int64_t* __restrict__ qt,
                                   const double* __restrict__ qeps, const int32_t* __restrict__ qL,
                                   const uint64_t* __restrict__ qseed, BudgetArgs A, int64_t n,
                                   const int4* __restrict__ node, QPlan* __restrict__ plans,
                                   QPlan* __restrict__ pilot) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int64_t s = qs[q], t = qt[q];
  const double eps = qeps[q];
  const int32_t L = qL[q];
  const bool ok = !(s < 0 || s >= n || t < 0 || t >= n || !(eps > 0.0 && eps < 1.0) || L < 0);
  const uint64_t seed = !ok ? 0 : (qseed ? qseed[q] : default_seed(A.global_seed, s, t, eps, L));
  const int32_t ds = ok ? node[s].z : 1, dt = ok ? node[t].z : 1;
  QPlan P, PP;
  plan_query(s, t, eps, L, seed, n, ds, dt, A, &P, &PP);
  plans[q] = P;
  if (pilot) pilot[q] = PP;
}

// Q slots of the batch: the sum of K, or of G Bmax for ADAPTIVE queries
// (device-array calls size their buffers from it).
__global__ void sum_k_kernel(const QPlan* __restrict__ plans, int64_t nq, unsigned long long* __restrict__ out) {
  __shared__ unsigned long long sh[1024];
  unsigned long long acc = 0;
  for (int64_t q = threadIdx.x; q < nq; q += blockDim.x) acc += q_slots(plans[q]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// PILOT: R >= 4 sigma^2 / theta (Lemma 3.7) from the pilot probes' (S1, S2),
// summed over probes in the oracle's order.
__global__ void pilot_budget_kernel(int64_t nq, QPlan* __restrict__ plans, const QPlan* __restrict__ pilot,
                                    const double* __restrict__ pilot_s, BudgetArgs A, const int4* __restrict__ node) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const QPlan PP = pilot[q];
  if (PP.K == 0) return;
  QPlan& P = plans[q];
  double sum_var = 0.0, sum_q = 0.0;
  for (uint32_t k = 0; k < PP.K; ++k) {
    const double* sk = pilot_s + 2 * (PP.probe_begin + k);
    pilot_accumulate(sum_var, sum_q, sk[0], sk[1], PP.R);
  }
  pilot_finish(P, sum_var, sum_q, PP.K, node[P.s].z, node[P.t].z, A);
}

// Walk kernel of each query and the offsets of its work.  A query's probes run
// in the probe-table kernel when building z^(k) once is cheaper than
// evaluating it at each of the probe's 2 R (L + 1) visits, by the graph's cost
// model (forced by walk_mode 1 or 2; the table needs n/8 bytes of shared
// memory).  prefix holds three arrays of nq + 1 offsets: per-visit tiles
// (K chunks of 32 replicas), table-kernel probes, and all probes (Q slots).
struct ModeArgs {
  int32_t forced;     // 0 auto, 1 per-visit, 2 table
  int32_t table_ok;   // the table fits in shared memory
  double probe_cost;  // cost of building one probe's table
  double visit_gain;  // saving per visit when entries come from the table
};

// keep_q (the second stage of ADAPTIVE queries): the Q slots stay where the
// first stage put them.
__global__ void scan_kernel(QPlan* __restrict__ plans, int64_t nq, unsigned long long* __restrict__ prefix,
                            Totals* __restrict__ totals, ModeArgs M, int keep_q) {
  __shared__ unsigned long long sh[4][1024];
  __shared__ unsigned long long sh_steps[1024], sh_visits[1024], sh_work[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t per = (nq + nt - 1) / nt;
  const int64_t b0 = per * tid, b = b0 < nq ? b0 : nq, e = b + per < nq ? b + per : nq;
  unsigned long long a[4] = {0, 0, 0, 0}, steps = 0, visits = 0, work = 0;
  for (int64_t q = b; q < e; ++q) {
    QPlan& P = plans[q];
    const double v = 2.0 * (double)P.R * (double)(P.L + 1);
    uint32_t mode = M.forced != 0 ? (uint32_t)M.forced
                                  : (M.probe_cost < v * M.visit_gain ? 2u : 1u);
    if (!M.table_ok) mode = 1u;
    P.mode = mode;
    const unsigned long long K = P.K;
    a[0] += mode == 1u ? K * P.chunks : 0ull;  // per-visit tiles
    a[1] += mode == 1u ? K : 0ull;             // per-visit probes (accumulators)
    a[2] += mode == 2u ? K : 0ull;             // table probes
    a[3] += q_slots(P);                        // Q slots
    work += K;
    steps += K * P.R * (unsigned long long)(P.L > 0 ? P.L : 0);
    visits += 2ull * K * P.R * (unsigned long long)(P.L + 1);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) sh[j][tid] = a[j];
  sh_steps[tid] = steps;
  sh_visits[tid] = visits;
  sh_work[tid] = work;
  __syncthreads();
  if (tid == 0) {
    unsigned long long run[4] = {0, 0, 0, 0}, st = 0, vi = 0, wk = 0;
    for (int i = 0; i < nt; ++i) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const unsigned long long x = sh[j][i];
        sh[j][i] = run[j];
        run[j] += x;
      }
      st += sh_steps[i];
      vi += sh_visits[i];
      wk += sh_work[i];
    }
    totals->tiles = run[0];
    totals->visit_probes = run[1];
    totals->table_probes = run[2];
    totals->probes = wk;
    totals->steps = st;
    totals->visits = vi;
    prefix[nq] = run[0];
    prefix[(nq + 1) + nq] = run[2];
    if (!keep_q) prefix[2 * (nq + 1) + nq] = run[3];
  }
  __syncthreads();
  unsigned long long o[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) o[j] = sh[j][tid];
  for (int64_t q = b; q < e; ++q) {
    QPlan& P = plans[q];
    const unsigned long long K = P.K;
    P.tile_begin = o[0];
    P.acc_begin = o[1];
    P.table_begin = o[2];
    if (!keep_q) {
      P.probe_begin = o[3];
      P.q_begin = o[3];
      prefix[2 * (nq + 1) + q] = o[3];
    }
    prefix[q] = o[0];
    prefix[(nq + 1) + q] = o[2];
    o[0] += P.mode == 1u ? K * P.chunks : 0ull;
    o[1] += P.mode == 1u ? K : 0ull;
    o[2] += P.mode == 2u ? K : 0ull;
    o[3] += q_slots(P);
  }
}

// ADAPTIVE, between the stages: each query's B* from its first G B1 values of
// Q_R; the second stage runs probes G B1 .. G B* - 1 into the Q slots after
// the first stage's, and the median reads G blocks of B* from q_begin.
__global__ void adapt_kernel(int64_t nq, QPlan* __restrict__ plans, const double* __restrict__ qbuf, BudgetArgs A,
                             const int4* __restrict__ node) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  QPlan& P = plans[q];
  if (P.status != PW_OK || P.K == 0 || P.Bmax == 0) return;
  const uint32_t B1 = P.B, K1 = P.K;
  const uint32_t Bs = adaptive_B(qbuf + P.q_begin, B1, P.Bmax, P.G, P.eps, A.z, node[P.s].z, node[P.t].z);
  P.B = Bs;
  P.k_begin = K1;
  P.K = P.G * (Bs - B1);
  P.probe_begin = P.q_begin + K1;
}

// Accumulators of the per-visit probes start at zero.
__global__ void zero_acc_kernel(ProbeAcc* __restrict__ acc, const Totals* __restrict__ totals) {
  const unsigned long long words = totals->visit_probes * (sizeof(ProbeAcc) / 8);
  unsigned long long* w = (unsigned long long*)acc;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < words;
       i += (unsigned long long)gridDim.x * blockDim.x)
    w[i] = 0ull;
}

__device__ __forceinline__ int64_t find_segment(const unsigned long long* __restrict__ prefix, int64_t nq,
                                                unsigned long long x) {
  int64_t lo = 0, hi = nq;  // last q with prefix[q] <= x
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (prefix[mid] <= x)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

struct WalkArgs {
  const int4* rec;   // fused records (layout 1)
  const int32_t* col;  // col_idx (layout 2)
  const int4* node;
  const QPlan* plans;
  const unsigned long long* tile_prefix;   // per-visit tiles
  const unsigned long long* table_prefix;  // table-kernel probes
  const Totals* totals;
  unsigned long long* counter;  // claim cursor of this launch
  ProbeAcc* acc;                // per-visit probe accumulators (main stage)
  double* q;                    // Q_R per probe (main stage) or (S1, S2) per probe (pilot)
  float* u_debug;               // optional: replica values of query 0
  uint32_t* visits;             // optional: visit counts
  int64_t nq;
  uint32_t n;
  uint32_t walk_tag, probe_tag;
};

// Persistent per-visit walk kernel: each warp pops tiles (query, probe k, 32
// replicas) from a device counter until the work runs out; lane l runs
// replica 32c + l with probe entries evaluated at each visit.  The warp sums
// its tile's replicas exactly; a pilot tile is a whole probe (R0 <= 32) and
// writes (S1, S2); a main tile adds its digits to the probe's accumulator and
// the probe's last tile computes Q_R.
// The graph access of a launch: fused records, or col_idx plus node records.
template <bool SPLIT>
struct GraphOf;
template <>
struct GraphOf<false> {
  static __device__ __forceinline__ FusedRecords get(const WalkArgs& A) { return FusedRecords{A.rec, A.node}; }
};
template <>
struct GraphOf<true> {
  static __device__ __forceinline__ SplitRecords get(const WalkArgs& A) { return SplitRecords{A.col, A.node}; }
};

// MINB: 1 leaves the registers to the compiler (2 blocks of 256 per SM), 3
// caps them for 3 blocks per SM (more walks in flight, some spills); the
// autotuner picks one per graph.
template <bool DEBUG, bool PILOT, bool SPLIT, int MINB>
__global__ void __launch_bounds__(kWalkThreads, MINB) walk_kernel(WalkArgs A) {
  const auto gr = GraphOf<SPLIT>::get(A);
  const uint32_t lane = threadIdx.x & 31u;
  const unsigned long long total = A.totals->tiles;
  for (;;) {
    unsigned long long tile = 0;
    if (lane == 0) tile = atomicAdd(A.counter, 1ull);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= total) return;
    const int64_t q = find_segment(A.tile_prefix, A.nq, tile);
    const QPlan& P = A.plans[q];
    const uint32_t chunks = P.chunks, R = P.R;
    const unsigned long long local = tile - P.tile_begin;
    const uint32_t kl = (uint32_t)(local / chunks);
    const uint32_t c = (uint32_t)(local - (unsigned long long)kl * chunks);
    const uint32_t p = c * 32u + lane;
    const uint32_t k = P.k_begin + kl;
    SumDigits sum;
    sum_clear(sum);
    if (p < R) {
      const Probe pr = make_probe(A.n, P.seed, k, A.probe_tag);
      const uint64_t pair = (uint64_t)k * R + p;
      const ZOnTheFly zp{pr};
      const float U = walk_pair<DEBUG>(gr, A.visits, A.walk_tag, zp, P.s, P.t, P.L, P.seed, pair);
      if (DEBUG && A.u_debug && q == 0) A.u_debug[(uint64_t)k * R + p] = U;
      sum_add(sum, U);
    }
    sum_warp_reduce(sum);
    if (lane != 0) continue;
    if (PILOT) {
      double S1, S2;
      sum_round(sum.d, S1, S2);
      A.q[2 * (P.probe_begin + kl)] = S1;
      A.q[2 * (P.probe_begin + kl) + 1] = S2;
    } else {
      ProbeAcc* pa = A.acc + P.acc_begin + kl;
      sum_atomic_add(pa->d, sum);
      __threadfence();
      if (atomicAdd(&pa->done, 1u) + 1u == chunks) {
        __threadfence();
        long long d[kSumDigits];
#pragma unroll
        for (int j = 0; j < kSumDigits; ++j) d[j] = (long long)__ldcg(pa->d + j);
        double S1, S2;
        sum_round(d, S1, S2);
        A.q[P.probe_begin + kl] = u_statistic(S1, S2, R);
      }
    }
  }
}

// Probe-table walk kernel: a block claims one probe k of one query, writes the
// whole vector z^(k) into a shared-memory table (sign bits plus the zero set;
// one Feistel cycle-walk per node), then its warps run the probe's 32-replica
// tiles reading z from the table, add each tile's exact sums into the block's
// digits, and the block writes the probe's Q_R.  Same values as the per-visit
// kernel; cheaper whenever a probe's walks visit more nodes than the Feistel
// domain has (2 R (L+1) > 2^b).
// THREADS: 256 (five blocks per SM for small tables), 512 or 1024 (one or two
// blocks per SM with up to 200 KB of table, still 32 warps).
template <bool DEBUG, bool SPLIT, int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS == 256 ? 5 : (THREADS == 512 ? 2 : 1)) walk_table_kernel(WalkArgs A) {
  const auto gr = GraphOf<SPLIT>::get(A);
  extern __shared__ uint32_t tab[];
  __shared__ unsigned long long sh_probe;
  __shared__ unsigned long long sh_sum[kSumDigits];
  __shared__ uint32_t sh_tile;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = A.n;
  const unsigned long long total = A.totals->table_probes;
  for (;;) {
    if (threadIdx.x == 0) {
      sh_probe = atomicAdd(A.counter, 1ull);
      sh_tile = 0;
    }
    if (threadIdx.x < kSumDigits) sh_sum[threadIdx.x] = 0ull;
    __syncthreads();
    const unsigned long long j = sh_probe;
    if (j >= total) return;
    const int64_t q = find_segment(A.table_prefix, A.nq, j);
    const QPlan& P = A.plans[q];
    const uint32_t kl = (uint32_t)(j - P.table_begin);
    const uint32_t k = P.k_begin + kl;
    build_probe_table(make_probe(n, P.seed, k, A.probe_tag), tab, n);
    __syncthreads();
    const ZTable zp = table_reader(tab, n);
    const uint32_t R = P.R, chunks = P.chunks;
    for (;;) {
      uint32_t c = 0;
      if (lane == 0) c = atomicAdd(&sh_tile, 1u);
      c = __shfl_sync(0xffffffffu, c, 0);
      if (c >= chunks) break;
      const uint32_t p = c * 32u + lane;
      SumDigits sum;
      sum_clear(sum);
      if (p < R) {
        const uint64_t pair = (uint64_t)k * R + p;
        const float U = walk_pair_table<DEBUG>(gr, A.visits, A.walk_tag, zp, P.s, P.t, P.L, P.seed, pair);
        if (DEBUG && A.u_debug && q == 0) A.u_debug[(uint64_t)k * R + p] = U;
        sum_add(sum, U);
      }
      sum_warp_reduce(sum);
      if (lane == 0) {
#pragma unroll
        for (int d = 0; d < kSumDigits; ++d)
          if (sum.d[d] != 0) atomicAdd(sh_sum + d, (unsigned long long)sum.d[d]);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long d[kSumDigits];
#pragma unroll
      for (int i = 0; i < kSumDigits; ++i) d[i] = (long long)sh_sum[i];
      double S1, S2;
      sum_round(d, S1, S2);
      A.q[P.probe_begin + kl] = u_statistic(S1, S2, R);
    }
    __syncthreads();
  }
}

// Exact S1, S2 of caller values through the walk kernels' accumulator (tests):
// lanes add strided values, warps reduce, shared 64-bit atomics combine.
__global__ void debug_exact_sum_kernel(const float* __restrict__ u, int64_t n, double* __restrict__ out) {
  __shared__ unsigned long long acc[kSumDigits];
  if (threadIdx.x < kSumDigits) acc[threadIdx.x] = 0ull;
  __syncthreads();
  const int64_t rounds = (n + blockDim.x - 1) / blockDim.x;
  for (int64_t r = 0; r < rounds; ++r) {
    const int64_t i = r * blockDim.x + threadIdx.x;
    SumDigits sum;
    sum_clear(sum);
    if (i < n) sum_add(sum, u[i]);
    sum_warp_reduce(sum);
    if ((threadIdx.x & 31u) == 0u)
      for (int d = 0; d < kSumDigits; ++d) atomicAdd(acc + d, (unsigned long long)sum.d[d]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long d[kSumDigits];
    for (int j = 0; j < kSumDigits; ++j) d[j] = (long long)acc[j];
    sum_round(d, out[0], out[1]);
  }
}

// Median of the G block means of B contiguous probes (Eq. final-estimator).
__global__ void mom_kernel(const QPlan* __restrict__ plans, const double* __restrict__ qbuf,
                           double* __restrict__ beta, int32_t* __restrict__ status) {
  __shared__ double means[4096];
  const int64_t q = blockIdx.x;
  const QPlan& P = plans[q];
  if (P.status != PW_OK || P.K == 0) {
    if (threadIdx.x == 0) {
      beta[q] = P.status == PW_OK ? 0.0 : __longlong_as_double(0x7ff8000000000000ll);
      status[q] = P.status;
    }
    return;
  }
  for (uint32_t g = threadIdx.x; g < P.G; g += blockDim.x) {
    const double* x = qbuf + P.q_begin + (uint64_t)g * P.B;
    double sum = 0.0;
    for (uint32_t k = 0; k < P.B; ++k) sum = __dadd_rn(sum, x[k]);
    means[g] = __ddiv_rn(sum, (double)P.B);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t G = P.G;
    for (uint32_t i = 1; i < G; ++i) {  // insertion sort
      const double v = means[i];
      uint32_t j = i;
      while (j > 0 && means[j - 1] > v) {
        means[j] = means[j - 1];
        --j;
      }
      means[j] = v;
    }
    const double med = (G & 1u) ? means[G / 2] : __ddiv_rn(__dadd_rn(means[G / 2 - 1], means[G / 2]), 2.0);
    beta[q] = med;
    status[q] = PW_OK;
  }
}

// Sharded query: keep only median-of-means blocks [g0, g1) of query 0; probe
// indices keep their global values (k_begin), so the walks are those of the
// whole query.
__global__ void restrict_blocks_kernel(QPlan* plans, uint32_t g0, uint32_t g1) {
  QPlan& P = plans[0];
  if (P.status != PW_OK || P.K == 0) return;
  P.k_begin = g0 * P.B;
  P.K = (g1 - g0) * P.B;
  P.G = g1 - g0;
}

// Block means of a sharded query (Eq. final-estimator before the median).
__global__ void block_means_kernel(const QPlan* __restrict__ plans, const double* __restrict__ qbuf,
                                   double* __restrict__ means, int32_t* __restrict__ status) {
  const QPlan& P = plans[0];
  for (uint32_t g = threadIdx.x; g < P.G; g += blockDim.x) {
    const double* x = qbuf + P.q_begin + (uint64_t)g * P.B;
    double sum = 0.0;
    for (uint32_t k = 0; k < P.B; ++k) sum = __dadd_rn(sum, x[k]);
    means[g] = __ddiv_rn(sum, (double)P.B);
  }
  if (threadIdx.x == 0) status[0] = P.status;
}

static cudaEvent_t prof_event(pw_graph* g) {
  ProfileState& P = g->prof;
  if (!P.pool.empty()) {
    cudaEvent_t e = P.pool.back();
    P.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void prof_begin(pw_graph* g, cudaStream_t stream, cudaEvent_t* a) {
  *a = nullptr;
  if (!g->prof.enabled) return;
  *a = prof_event(g);
  cudaEventRecord(*a, stream);
}

void prof_end(pw_graph* g, cudaStream_t stream, cudaEvent_t a, int kind) {
  if (!g->prof.enabled || !a) return;
  cudaEvent_t b = prof_event(g);
  cudaEventRecord(b, stream);
  g->prof.spans.push_back({a, b, kind});
}

// Largest graph whose probe table (1 bit per node) fits in shared memory next to the kernel's own state.
static size_t table_bytes(const pw_graph* g) { return sizeof(uint32_t) * (size_t)table_words((uint32_t)g->n); }
static constexpr size_t kMaxTableBytes = 200 * 1024;

// Table-kernel block size by shared memory: 256 threads while five tables fit
// per SM (then registers limit it to five blocks), 512 while two fit, else 1024.
static int default_table_threads(const pw_graph* g) {
  const size_t per_block = table_bytes(g) + 2048;
  const size_t fit = ((size_t)228 << 10) / per_block;
  return fit >= 5 ? 256 : (fit >= 2 ? 512 : 1024);
}

using WalkFn = void (*)(WalkArgs);

// The per-visit kernel of a launch (DEBUG builds exist only at MINB 1).
static WalkFn walk_fn(bool debug, bool pilot, bool split, int minb) {
  if (debug) return split ? walk_kernel<true, false, true, 1> : walk_kernel<true, false, false, 1>;
  if (minb == 3) {
    if (pilot) return split ? walk_kernel<false, true, true, 3> : walk_kernel<false, true, false, 3>;
    return split ? walk_kernel<false, false, true, 3> : walk_kernel<false, false, false, 3>;
  }
  if (pilot) return split ? walk_kernel<false, true, true, 1> : walk_kernel<false, true, false, 1>;
  return split ? walk_kernel<false, false, true, 1> : walk_kernel<false, false, false, 1>;
}

// The table kernel of a launch (DEBUG builds exist only at 256 threads).
static WalkFn table_fn(bool debug, bool split, int threads) {
  if (debug) return split ? walk_table_kernel<true, true, 256> : walk_table_kernel<true, false, 256>;
  if (threads == 1024) return split ? walk_table_kernel<false, true, 1024> : walk_table_kernel<false, false, 1024>;
  if (threads == 512) return split ? walk_table_kernel<false, true, 512> : walk_table_kernel<false, false, 512>;
  return split ? walk_table_kernel<false, true, 256> : walk_table_kernel<false, false, 256>;
}

// Persistent grid: SMs x resident blocks, measured once per kernel and
// shared-memory size on this graph.
static int grid_of(pw_graph* g, WalkFn fn, int threads, size_t smem) {
  const auto key = std::make_pair((const void*)fn, smem);
  auto it = g->grids.find(key);
  if (it != g->grids.end()) return it->second;
  int nb = 0;
  if (smem > 48 * 1024) cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)fn, threads, smem);
  const int grid = g->sm_count * (nb > 0 ? nb : 1);
  g->grids[key] = grid;
  return grid;
}

static pw_status launch_walk(pw_graph* g, cudaStream_t stream, const WalkArgs& a, bool debug, bool pilot) {
  const WalkFn fn = walk_fn(debug, pilot, g->layout == 2, g->visit_minb);
  const cudaError_t e = launch_with_window(g, fn, grid_of(g, fn, kWalkThreads, 0), kWalkThreads, 0, stream, a);
  count_launch();
  PW_CUDA_TRY(e);
  return PW_OK;
}

static int table_threads(const pw_graph* g) {
  return g->table_threads ? g->table_threads : default_table_threads(g);
}

static pw_status launch_table(pw_graph* g, cudaStream_t stream, const WalkArgs& a, bool debug) {
  const size_t smem = table_bytes(g);
  const int threads = debug ? 256 : table_threads(g);
  const WalkFn fn = table_fn(debug, g->layout == 2, threads);
  const cudaError_t e = launch_with_window(g, fn, grid_of(g, fn, threads, smem), threads, smem, stream, a);
  count_launch();
  PW_CUDA_TRY(e);
  return PW_OK;
}

// Device scratch of one batch.  Sizes depend on the query count, the pilot
// shape and the sum of K; nothing depends on R, so a batch never waits for its
// pilot to size memory.
struct BatchBuffers {
  QPlan* plans;
  QPlan* pplans;
  unsigned long long* prefix;    // 6 (nq + 1): main tiles, table probes, probes; then the pilot's three
  Totals* totals;                // [0] main, [1] pilot
  unsigned long long* counters;  // [0] main per-visit tiles, [1] pilot tiles, [2] table probes
  double* pilot_s;               // (S1, S2) per pilot probe
  double* q;                     // Q_R per probe
  ProbeAcc* acc;                 // per-visit probe accumulators
};

static bool has_pilot(const BudgetArgs& ba) { return ba.mode == PW_BUDGET_PILOT || ba.mode == PW_BUDGET_ADAPTIVE; }

struct BatchSizes {
  size_t plans, prefix, totals, counters, pilot_s, q, acc;
};

static BatchSizes batch_sizes(size_t nq, size_t total_K, const BudgetArgs& ba) {
  BatchSizes z;
  z.plans = sizeof(QPlan) * nq;
  z.prefix = sizeof(unsigned long long) * 6 * (nq + 1);
  z.totals = sizeof(Totals) * 3;
  z.counters = 64;
  z.pilot_s = has_pilot(ba) ? sizeof(double) * 2 * nq * (size_t)ba.K0 : 16;
  z.q = sizeof(double) * (total_K ? total_K : 1);
  z.acc = sizeof(ProbeAcc) * (total_K ? total_K : 1);
  return z;
}

// First stage: counters cleared, plans of every query (and their pilots).
static pw_status enqueue_budget(pw_graph* g, int64_t count, const int64_t* d_s, const int64_t* d_t, const double* d_eps,
                                const int32_t* d_L, const uint64_t* d_seeds, const BudgetArgs& ba,
                                const BatchBuffers& B, cudaStream_t stream) {
  PW_CUDA_TRY(cudaMemsetAsync(B.counters, 0, 64, stream));
  const int qthreads = 128;
  const int qblocks = (int)((count + qthreads - 1) / qthreads);
  budget_init_kernel<<<qblocks, qthreads, 0, stream>>>(count, d_s, d_t, d_eps, d_L, d_seeds, ba, g->n, g->d_node,
                                                       B.plans, has_pilot(ba) ? B.pplans : nullptr);
  count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  return PW_OK;
}

// The rest of the pipeline: pilot, walk kernels, median.  No host
// synchronisation: every size it needs was fixed by batch_sizes.
static pw_status enqueue_walks(pw_graph* g, int64_t count, const pw_params* params, const BudgetArgs& ba,
                               const BatchBuffers& B, double* d_beta, int32_t* d_status, cudaStream_t stream,
                               DebugOut* dbg) {
  const size_t nq = (size_t)count;
  const bool pilot = has_pilot(ba);
  const int qthreads = 128;
  const int qblocks = (int)((count + qthreads - 1) / qthreads);
  unsigned long long* prefix = B.prefix;
  unsigned long long* pprefix = B.prefix + 3 * (nq + 1);
  WalkArgs wa;
  memset(&wa, 0, sizeof wa);
  wa.rec = g->d_rec;
  wa.col = g->d_col;
  wa.node = g->d_node;
  wa.nq = count;
  wa.n = (uint32_t)g->n;
  pw_status st;
  if (pilot) {
    ModeArgs pm{1, 0, 0.0, 0.0};
    scan_kernel<<<1, 1024, 0, stream>>>(B.pplans, count, pprefix, B.totals + 1, pm, 0);
    count_launch();
    wa.plans = B.pplans;
    wa.tile_prefix = pprefix;
    wa.totals = B.totals + 1;
    wa.counter = B.counters + 1;
    wa.q = B.pilot_s;
    wa.walk_tag = kTagWalkPilot;
    wa.probe_tag = kTagProbePilot;
    cudaEvent_t ev;
    prof_begin(g, stream, &ev);
    if ((st = launch_walk(g, stream, wa, false, true)) != PW_OK) return st;
    prof_end(g, stream, ev, 1);
    if (g->prof.enabled) g->prof.pilot_transitions += 2ull * nq * (uint64_t)ba.K0 * (uint64_t)ba.R0;
    pilot_budget_kernel<<<qblocks, qthreads, 0, stream>>>(count, B.plans, B.pplans, B.pilot_s, ba, g->d_node);
    count_launch();
    PW_CUDA_TRY(cudaGetLastError());
  }
  const bool sharded = dbg && dbg->g_begin >= 0;
  if (sharded) {
    restrict_blocks_kernel<<<1, 1, 0, stream>>>(B.plans, (uint32_t)dbg->g_begin, (uint32_t)dbg->g_end);
    count_launch();
    PW_CUDA_TRY(cudaGetLastError());
  }
  const bool table_ok = table_bytes(g) <= kMaxTableBytes;
  const int forced = params && params->walk_mode ? params->walk_mode : g->walk_policy;
  ModeArgs M{forced, table_ok ? 1 : 0, g->table_probe_cost, g->table_visit_gain};
  if (params && (params->walk_mode < 0 || params->walk_mode > 2))
    return set_error(PW_ERR_ARG, "walk_mode must be 0, 1 or 2");
  scan_kernel<<<1, 1024, 0, stream>>>(B.plans, count, prefix, B.totals, M, 0);
  count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  if (dbg && dbg->budget_only) return PW_OK;
  const bool debug = dbg && (dbg->visits || dbg->u);
  wa.plans = B.plans;
  wa.tile_prefix = prefix;
  wa.table_prefix = prefix + (nq + 1);
  wa.acc = B.acc;
  wa.q = B.q;
  wa.visits = dbg ? dbg->visits : nullptr;
  wa.u_debug = dbg ? dbg->u : nullptr;
  wa.walk_tag = kTagWalk;
  wa.probe_tag = kTagProbe;
  cudaEvent_t ev_walk;
  prof_begin(g, stream, &ev_walk);
  cudaEvent_t tw[2] = {nullptr, nullptr};
  if (dbg && dbg->time_walk) {
    PW_CUDA_TRY(cudaEventCreate(&tw[0]));
    cudaError_t e = cudaEventCreate(&tw[1]);
    if (e == cudaSuccess) e = cudaEventRecord(tw[0], stream);
    if (e != cudaSuccess) {
      cudaEventDestroy(tw[0]);
      if (tw[1]) cudaEventDestroy(tw[1]);
      return cuda_error(e, "walk timing events");
    }
  }
  // one walk stage: accumulators zeroed, then the table and per-visit kernels
  // (each takes only its own queries' probes, as the scan assigned them)
  auto walk_stage = [&](Totals* totals, unsigned long long* counters) -> pw_status {
    zero_acc_kernel<<<g->sm_count * 4, 256, 0, stream>>>(B.acc, totals);
    count_launch();
    PW_CUDA_TRY(cudaGetLastError());
    wa.totals = totals;
    pw_status s2 = PW_OK;
    if (table_ok) {
      wa.counter = counters + 2;
      s2 = launch_table(g, stream, wa, debug);
    }
    if (s2 == PW_OK) {
      wa.counter = counters;
      s2 = launch_walk(g, stream, wa, debug, false);
    }
    return s2;
  };
  st = walk_stage(B.totals, B.counters);
  if (st == PW_OK && ba.mode == PW_BUDGET_ADAPTIVE) {
    // the stopping rule on the first stage's Q_R, then the second stage's
    // probes with their own offsets and totals (Q slots stay in place)
    adapt_kernel<<<qblocks, qthreads, 0, stream>>>(count, B.plans, B.q, ba, g->d_node);
    count_launch();
    scan_kernel<<<1, 1024, 0, stream>>>(B.plans, count, prefix, B.totals + 2, M, 1);
    count_launch();
    const cudaError_t e = cudaGetLastError();
    st = e == cudaSuccess ? walk_stage(B.totals + 2, B.counters + 4) : cuda_error(e, "adaptive stage");
  }
  if (tw[0]) {
    cudaError_t e = st == PW_OK ? cudaEventRecord(tw[1], stream) : cudaSuccess;
    if (st == PW_OK && e == cudaSuccess) e = cudaEventSynchronize(tw[1]);
    if (st == PW_OK && e == cudaSuccess) e = cudaEventElapsedTime(&dbg->walk_ms, tw[0], tw[1]);
    cudaEventDestroy(tw[0]);
    cudaEventDestroy(tw[1]);
    if (st == PW_OK && e != cudaSuccess) return cuda_error(e, "walk timing events");
  }
  if (st != PW_OK) return st;
  prof_end(g, stream, ev_walk, 0);
  if (g->prof.enabled) {
    g->prof.walk_launches += 1;
    g->prof.queries += nq;
  }
  cudaEvent_t ev_fin;
  prof_begin(g, stream, &ev_fin);
  if (sharded)
    block_means_kernel<<<1, 128, 0, stream>>>(B.plans, B.q, dbg->block_means, d_status);
  else
    mom_kernel<<<(unsigned)count, 128, 0, stream>>>(B.plans, B.q, d_beta, d_status);
  count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  prof_end(g, stream, ev_fin, 2);
  return PW_OK;
}

// Totals of a finished batch for the profile (pinned copy, read by pw_profile).
static pw_status prof_totals(pw_graph* g, const Totals* d_totals, cudaStream_t stream) {
  ProfileState& P = g->prof;
  if (!P.enabled) return PW_OK;
  Totals* h = nullptr;
  if (!P.spare.empty()) {
    h = P.spare.back();
    P.spare.pop_back();
  } else {
    PW_CUDA_TRY(cudaMallocHost(&h, sizeof(Totals)));
  }
  P.pending.push_back(h);
  PW_CUDA_TRY(cudaMemcpyAsync(h, d_totals, sizeof(Totals), cudaMemcpyDeviceToHost, stream));
  return PW_OK;
}

static pw_status batch_buffers(pw_graph* g, size_t nq, size_t total_K, const BudgetArgs& ba, BatchBuffers* B) {
  Workspace& ws = g->ws;
  const BatchSizes z = batch_sizes(nq, total_K, ba);
  pw_status st;
  if ((st = ensure_buffer(ws.plans, z.plans)) != PW_OK) return st;
  if ((st = ensure_buffer(ws.pilot_plans, z.plans)) != PW_OK) return st;
  if ((st = ensure_buffer(ws.tile_prefix, z.prefix)) != PW_OK) return st;
  if ((st = ensure_buffer(ws.totals, z.totals)) != PW_OK) return st;
  if ((st = ensure_buffer(ws.counters, z.counters)) != PW_OK) return st;
  if ((st = ensure_buffer(ws.pilot_s, z.pilot_s)) != PW_OK) return st;
  if ((st = ensure_buffer(ws.q, z.q)) != PW_OK) return st;
  if ((st = ensure_buffer(ws.acc, z.acc)) != PW_OK) return st;
  B->plans = (QPlan*)ws.plans.ptr;
  B->pplans = (QPlan*)ws.pilot_plans.ptr;
  B->prefix = (unsigned long long*)ws.tile_prefix.ptr;
  B->totals = (Totals*)ws.totals.ptr;
  B->counters = (unsigned long long*)ws.counters.ptr;
  B->pilot_s = (double*)ws.pilot_s.ptr;
  B->q = (double*)ws.q.ptr;
  B->acc = (ProbeAcc*)ws.acc.ptr;
  return PW_OK;
}

// Sum of K over the batch, read back from the device (one synchronisation).
static pw_status device_total_K(pw_graph* g, int64_t count, const int64_t* d_s, const int64_t* d_t,
                                const double* d_eps, const int32_t* d_L, const uint64_t* d_seeds, const BudgetArgs& ba,
                                cudaStream_t stream, size_t* total_K) {
  Workspace& ws = g->ws;
  pw_status st;
  if ((st = ensure_buffer(ws.plans, sizeof(QPlan) * (size_t)count)) != PW_OK) return st;
  if ((st = ensure_buffer(ws.counters, 64)) != PW_OK) return st;
  const int qthreads = 128;
  const int qblocks = (int)((count + qthreads - 1) / qthreads);
  budget_init_kernel<<<qblocks, qthreads, 0, stream>>>(count, d_s, d_t, d_eps, d_L, d_seeds, ba, g->n, g->d_node,
                                                       (QPlan*)ws.plans.ptr, nullptr);
  count_launch();
  unsigned long long* out = (unsigned long long*)ws.counters.ptr + 7;
  sum_k_kernel<<<1, 1024, 0, stream>>>((const QPlan*)ws.plans.ptr, count, out);
  count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  PW_CUDA_TRY(cudaMemcpyAsync(&ws.host_totals->pad[0], out, 8, cudaMemcpyDeviceToHost, stream));
  PW_CUDA_TRY(cudaStreamSynchronize(stream));
  *total_K = (size_t)ws.host_totals->pad[0];
  return PW_OK;
}

// Every stage of a batch whose scratch is sized, then a copy of its totals.
static pw_status enqueue_batch(pw_graph* g, int64_t count, const int64_t* d_s, const int64_t* d_t,
                               const double* d_eps, const int32_t* d_L, const uint64_t* d_seeds,
                               const pw_params* params, const BudgetArgs& ba, const BatchBuffers& B, double* d_beta,
                               int32_t* d_status, cudaStream_t stream, DebugOut* dbg) {
  pw_status st;
  if ((st = enqueue_budget(g, count, d_s, d_t, d_eps, d_L, d_seeds, ba, B, stream)) != PW_OK) return st;
  if ((st = enqueue_walks(g, count, params, ba, B, d_beta, d_status, stream, dbg)) != PW_OK) return st;
  PW_CUDA_TRY(cudaMemcpyAsync(g->ws.host_totals, B.totals, sizeof(Totals), cudaMemcpyDeviceToHost, stream));
  st = prof_totals(g, B.totals, stream);
  if (st == PW_OK && ba.mode == PW_BUDGET_ADAPTIVE && !(dbg && dbg->budget_only)) st = prof_totals(g, B.totals + 2, stream);
  return st;
}

pw_status run_batch(pw_graph* g, int64_t count, const int64_t* d_s, const int64_t* d_t, const double* d_eps,
                    const int32_t* d_L, const uint64_t* d_seeds, const pw_params* params, double* d_beta,
                    int32_t* d_status, cudaStream_t stream, DebugOut* dbg, int64_t total_K) {
  BudgetArgs ba;
  pw_status st = resolve_budget(params, g, &ba, nullptr);
  if (st != PW_OK) return st;
  if (count < 0) return set_error(PW_ERR_ARG, "count < 0");
  if (count == 0) return PW_OK;
  Workspace& ws = g->ws;
  PW_CUDA_TRY(cudaStreamWaitEvent(stream, ws.last_use, 0));
  size_t K = 0;
  if (total_K >= 0) {
    K = (size_t)total_K;
  } else if ((st = device_total_K(g, count, d_s, d_t, d_eps, d_L, d_seeds, ba, stream, &K)) != PW_OK) {
    return st;
  }
  BatchBuffers B;
  if ((st = batch_buffers(g, (size_t)count, K, ba, &B)) != PW_OK) return st;
  if (dbg && dbg->u && count != 1) return set_error(PW_ERR_ARG, "replica output needs a single-query batch");
  if ((st = enqueue_batch(g, count, d_s, d_t, d_eps, d_L, d_seeds, params, ba, B, d_beta, d_status, stream, dbg)) !=
      PW_OK)
    return st;
  PW_CUDA_TRY(cudaEventRecord(ws.last_use, stream));
  return PW_OK;
}

// Sum of K over host-array queries, from the same plan as the device
// (invalid queries and s == t contribute 0).
static size_t host_total_K(const pw_graph* g, int64_t count, const int64_t* s, const int64_t* t, const double* eps,
                           const int32_t* L, const BudgetArgs& ba) {
  size_t K = 0;
  for (int64_t i = 0; i < count; ++i) {
    const bool in = s[i] >= 0 && s[i] < g->n && t[i] >= 0 && t[i] < g->n;
    QPlan P;
    plan_query(s[i], t[i], eps[i], L[i], 0, g->n, in ? g->deg[(size_t)s[i]] : 1, in ? g->deg[(size_t)t[i]] : 1, ba,
               &P, nullptr);
    K += q_slots(P);
  }
  return K;
}

template <class T>
static void key_put(std::vector<unsigned char>& k, const T& v) {
  const unsigned char* p = (const unsigned char*)&v;
  k.insert(k.end(), p, p + sizeof(T));
}

// A host-array call through a CUDA graph: the staged inputs at h (in_bytes)
// go in, the results come back to ho (out_bytes).  Returns PW_PENDING
// without running anything when this shape has not been seen on the previous
// call (the caller then runs it eagerly); captures it on its second
// consecutive call; replays it afterwards.
static pw_status graph_batch(pw_graph* g, int64_t count, const char* h, char* ho, size_t in_bytes, size_t out_bytes,
                             const pw_params* params, const BudgetArgs& ba, size_t total_K) {
  Workspace& ws = g->ws;
  GraphCache& gc = g->gcache;
  BatchBuffers B;
  pw_status st = batch_buffers(g, (size_t)count, total_K, ba, &B);  // allocations stay outside the capture
  if (st != PW_OK) return st;
  const bool table_ok = table_bytes(g) <= kMaxTableBytes;
  if (table_ok) {  // occupancy queries stay outside the capture
    const WalkFn tf = table_fn(false, g->layout == 2, table_threads(g));
    grid_of(g, tf, table_threads(g), table_bytes(g));
  }
  for (int pilot = 0; pilot < 2; ++pilot) grid_of(g, walk_fn(false, pilot != 0, g->layout == 2, g->visit_minb), kWalkThreads, 0);
  std::vector<unsigned char> key;
  key_put(key, count);
  key_put(key, total_K);
  key_put(key, ba);
  key_put(key, params ? params->walk_mode : 0);
  key_put(key, g->table_probe_cost);
  key_put(key, g->table_visit_gain);
  key_put(key, g->visit_minb);
  key_put(key, g->walk_policy);
  key_put(key, g->table_threads);
  key_put(key, g->l2_window);
  key_put(key, B);
  key_put(key, ws.queries.ptr);
  key_put(key, ws.results.ptr);
  key_put(key, (const void*)h);
  if (!(gc.exec && key == gc.key)) {
    if (key != gc.seen) {
      gc.seen = key;
      return PW_PENDING;
    }
    const uint64_t before = pw_launch_count(0);
    PW_CUDA_TRY(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
    char* d = (char*)ws.queries.ptr;
    const size_t nq = (size_t)count;
    cudaError_t e = cudaMemcpyAsync(d, h, in_bytes, cudaMemcpyHostToDevice, g->stream);
    st = e == cudaSuccess ? PW_OK : cuda_error(e, "graph input copy");
    if (st == PW_OK)
      st = enqueue_batch(g, count, (const int64_t*)d, (const int64_t*)(d + nq * 8), (const double*)(d + nq * 16),
                         (const int32_t*)(d + nq * 32), (const uint64_t*)(d + nq * 24), params, ba, B,
                         (double*)ws.results.ptr, (int32_t*)((char*)ws.results.ptr + nq * 8), g->stream, nullptr);
    if (st == PW_OK) {
      e = cudaMemcpyAsync(ho, ws.results.ptr, out_bytes, cudaMemcpyDeviceToHost, g->stream);
      if (e != cudaSuccess) st = cuda_error(e, "graph result copy");
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(g->stream, &graph);
    const uint64_t captured = pw_launch_count(0) - before;
    count_launches(-(int64_t)captured);  // nothing ran during the capture
    if (st == PW_OK && ec != cudaSuccess) st = cuda_error(ec, "cudaStreamEndCapture");
    if (st == PW_OK) {
      if (gc.exec) cudaGraphExecDestroy(gc.exec);
      gc.exec = nullptr;
      e = cudaGraphInstantiate(&gc.exec, graph, 0);
      if (e != cudaSuccess) {
        gc.exec = nullptr;
        st = cuda_error(e, "cudaGraphInstantiate");
      }
    }
    if (graph) cudaGraphDestroy(graph);
    if (st != PW_OK) {
      gc.key.clear();
      gc.seen.clear();
      return st;
    }
    gc.key = key;
    gc.launches = captured;
  }
  PW_CUDA_TRY(cudaGraphLaunch(gc.exec, g->stream));
  count_launches((int64_t)gc.launches);
  PW_CUDA_TRY(cudaEventRecord(ws.last_use, g->stream));
  PW_CUDA_TRY(cudaStreamSynchronize(g->stream));
  return PW_OK;
}

// Host-array batch: stage inputs in pinned memory, run, copy results back.
// Nothing between the input copy and the result copy waits for the host, so a
// call whose shape repeats runs as one CUDA graph.
static pw_status host_batch(pw_graph* g, int64_t count, const int64_t* s, const int64_t* t, const double* eps,
                            const int32_t* L, const uint64_t* seeds, const pw_params* params, double* beta,
                            int32_t* status, DebugOut* dbg) {
  if (count < 0) return set_error(PW_ERR_ARG, "count < 0");
  if (count == 0) return PW_OK;
  if (!s || !t || !eps || !L || !beta || !status) return set_error(PW_ERR_ARG, "NULL array");
  Workspace& ws = g->ws;
  const size_t nq = (size_t)count;
  const size_t in_bytes = nq * (8 + 8 + 8 + 8 + 4), out_bytes = nq * (8 + 4);
  BudgetArgs ba;
  pw_status st = resolve_budget(params, g, &ba, nullptr);
  if (st != PW_OK) return st;
  if ((st = ensure_host_staging(ws, in_bytes + out_bytes + 64)) != PW_OK) return st;
  if ((st = ensure_buffer(ws.queries, in_bytes + 64)) != PW_OK) return st;
  if ((st = ensure_buffer(ws.results, out_bytes + 64)) != PW_OK) return st;
  PW_CUDA_TRY(cudaStreamWaitEvent(g->stream, ws.last_use, 0));
  PW_CUDA_TRY(cudaStreamSynchronize(g->stream));
  char* h = (char*)ws.host_staging;
  memcpy(h, s, nq * 8);
  memcpy(h + nq * 8, t, nq * 8);
  memcpy(h + nq * 16, eps, nq * 8);
  if (seeds) {
    memcpy(h + nq * 24, seeds, nq * 8);
  } else {
    for (size_t i = 0; i < nq; ++i)
      ((uint64_t*)(h + nq * 24))[i] = default_seed(ba.global_seed, s[i], t[i], eps[i], L[i]);
  }
  memcpy(h + nq * 32, L, nq * 4);
  const size_t K = host_total_K(g, count, s, t, eps, L, ba);
  char* d = (char*)ws.queries.ptr;
  double* d_beta = (double*)ws.results.ptr;
  int32_t* d_status = (int32_t*)((char*)ws.results.ptr + nq * 8);
  char* ho = h + in_bytes;
  if (!dbg && !g->prof.enabled) {
    st = graph_batch(g, count, h, ho, in_bytes, out_bytes, params, ba, K);
    if (st == PW_OK) {
      memcpy(beta, ho, nq * 8);
      memcpy(status, ho + nq * 8, nq * 4);
    }
    if (st != PW_PENDING) return st;  // PENDING: shape not seen twice yet, run it eagerly
  }
  PW_CUDA_TRY(cudaMemcpyAsync(d, h, in_bytes, cudaMemcpyHostToDevice, g->stream));
  st = run_batch(g, count, (const int64_t*)d, (const int64_t*)(d + nq * 8), (const double*)(d + nq * 16),
                 (const int32_t*)(d + nq * 32), (const uint64_t*)(d + nq * 24), params, d_beta, d_status, g->stream,
                 dbg, (int64_t)K);
  if (st != PW_OK) return st;
  if (dbg && dbg->budget_only) {
    PW_CUDA_TRY(cudaStreamSynchronize(g->stream));
    return PW_OK;
  }
  PW_CUDA_TRY(cudaMemcpyAsync(ho, ws.results.ptr, out_bytes, cudaMemcpyDeviceToHost, g->stream));
  PW_CUDA_TRY(cudaStreamSynchronize(g->stream));
  memcpy(beta, ho, nq * 8);
  memcpy(status, ho + nq * 8, nq * 4);
  return PW_OK;
}

static pw_status copy_plan(pw_graph* g, int64_t q, QPlan* out) {
  PW_CUDA_TRY(cudaMemcpyAsync(out, (QPlan*)g->ws.plans.ptr + q, sizeof(QPlan), cudaMemcpyDeviceToHost, g->stream));
  PW_CUDA_TRY(cudaStreamSynchronize(g->stream));
  return PW_OK;
}

// Walk kernels that ran in the latest batch: 1 per-visit, 2 table, 3 both.
static int last_walk_mode(const pw_graph* g) {
  const Totals* T = g->ws.host_totals;
  if (!T) return 0;
  return (T->tiles > 0 ? 1 : 0) | (T->table_probes > 0 ? 2 : 0);
}

}  // namespace pw

using namespace pw;

extern "C" {

pw_status pw_query_batch(pw_graph* g, int64_t count, const int64_t* s, const int64_t* t, const double* eps,
                         const int32_t* L, const uint64_t* seeds, const pw_params* params, double* beta_hat,
                         int32_t* per_query_status) {
  if (!g) return set_error(PW_ERR_ARG, "graph is NULL");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  return host_batch(g, count, s, t, eps, L, seeds, params, beta_hat, per_query_status, nullptr);
}

pw_status pw_query_batch_device(pw_graph* g, int64_t count, const int64_t* d_s, const int64_t* d_t,
                                const double* d_eps, const int32_t* d_L, const uint64_t* d_seeds,
                                const pw_params* params, double* d_beta_hat, int32_t* d_status, void* stream) {
  if (!g) return set_error(PW_ERR_ARG, "graph is NULL");
  if (count > 0 && (!d_s || !d_t || !d_eps || !d_L || !d_beta_hat || !d_status))
    return set_error(PW_ERR_ARG, "NULL device array");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  return run_batch(g, count, d_s, d_t, d_eps, d_L, d_seeds, params, d_beta_hat, d_status, (cudaStream_t)stream,
                   nullptr, -1);
}

pw_status pw_query(pw_graph* g, int64_t s, int64_t t, double eps, int32_t L, const uint64_t* seed,
                   const pw_params* params, double* beta_hat) {
  if (!g || !beta_hat) return set_error(PW_ERR_ARG, "NULL argument");
  if (s < 0 || s >= g->n || t < 0 || t >= g->n) return set_error(PW_ERR_ARG, "node id out of range");
  if (!(eps > 0.0 && eps < 1.0)) return set_error(PW_ERR_ARG, "eps must lie in (0, 1)");
  if (L < 0) return set_error(PW_ERR_ARG, "L < 0");
  if (s == t) {
    *beta_hat = 0.0;
    return PW_OK;
  }
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  BudgetArgs ba;
  pw_status st = resolve_budget(params, g, &ba, nullptr);
  if (st != PW_OK) return st;
  const uint64_t sd = seed ? *seed : default_seed(ba.global_seed, s, t, eps, L);
  int32_t qst = 0;
  st = host_batch(g, 1, &s, &t, &eps, &L, &sd, params, beta_hat, &qst, nullptr);
  if (st != PW_OK) return st;
  if (qst != PW_OK) return set_error((pw_status)qst, "query rejected (budget beyond 2^32 probes or replicas)");
  return PW_OK;
}

pw_status pw_budget(pw_graph* g, int64_t s, int64_t t, double eps, int32_t L, const uint64_t* seed,
                    const pw_params* params, uint64_t* B, uint64_t* G, uint64_t* K, uint64_t* R) {
  if (!g) return set_error(PW_ERR_ARG, "graph is NULL");
  if (s < 0 || s >= g->n || t < 0 || t >= g->n) return set_error(PW_ERR_ARG, "node id out of range");
  if (!(eps > 0.0 && eps < 1.0)) return set_error(PW_ERR_ARG, "eps must lie in (0, 1)");
  if (L < 0) return set_error(PW_ERR_ARG, "L < 0");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  BudgetArgs ba;
  pw_status st = resolve_budget(params, g, &ba, nullptr);
  if (st != PW_OK) return st;
  const uint64_t sd = seed ? *seed : default_seed(ba.global_seed, s, t, eps, L);
  DebugOut dbg;
  dbg.budget_only = true;
  double beta;
  int32_t qst;
  st = host_batch(g, 1, &s, &t, &eps, &L, &sd, params, &beta, &qst, &dbg);
  if (st != PW_OK) return st;
  QPlan P;
  if ((st = copy_plan(g, 0, &P)) != PW_OK) return st;
  if (P.status != PW_OK) return set_error((pw_status)P.status, "query rejected");
  if (B) *B = P.B;
  if (G) *G = P.G;
  if (K) *K = P.K;
  if (R) *R = P.R;
  return PW_OK;
}

pw_status pw_debug_query(pw_graph* g, int64_t s, int64_t t, double eps, int32_t L, const uint64_t* seed,
                         const pw_params* params, double* beta_hat, uint64_t* budget, double* pilot, double* q,
                         int64_t q_cap, float* u, int64_t u_cap, uint32_t* visits) {
  if (!g || !beta_hat) return set_error(PW_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  BudgetArgs ba;
  pw_status st = resolve_budget(params, g, &ba, nullptr);
  if (st != PW_OK) return st;
  const uint64_t sd = seed ? *seed : default_seed(ba.global_seed, s, t, eps, L);
  // pass 1: the budget alone, to size the replica output
  DebugOut pre;
  pre.budget_only = true;
  int32_t qst = 0;
  st = host_batch(g, 1, &s, &t, &eps, &L, &sd, params, beta_hat, &qst, &pre);
  if (st != PW_OK) return st;
  QPlan P0;
  if ((st = copy_plan(g, 0, &P0)) != PW_OK) return st;
  const uint64_t K0 = q_slots(P0), KR0 = K0 * P0.R;  // ADAPTIVE: the most its second stage may reach
  if ((q && (uint64_t)q_cap < K0) || (u && (uint64_t)u_cap < KR0)) return set_error(PW_ERR_ARG, "q_cap or u_cap too small");
  // pass 2: the whole query, with replica values and visit counts
  DebugOut dbg;
  DeviceBuffer vis;
  if (visits) {
    if ((st = ensure_buffer(vis, sizeof(uint32_t) * (size_t)g->n)) != PW_OK) return st;
    PW_CUDA_TRY(cudaMemsetAsync(vis.ptr, 0, sizeof(uint32_t) * (size_t)g->n, g->stream));
    dbg.visits = (uint32_t*)vis.ptr;
  }
  if (u && KR0) {
    if ((st = ensure_buffer(g->ws.u_debug, sizeof(float) * (size_t)KR0)) != PW_OK) return st;
    dbg.u = (float*)g->ws.u_debug.ptr;
  }
  st = host_batch(g, 1, &s, &t, &eps, &L, &sd, params, beta_hat, &qst, &dbg);
  if (st == PW_OK && qst != PW_OK) st = set_error((pw_status)qst, "query rejected");
  QPlan P;
  memset(&P, 0, sizeof P);
  if (st == PW_OK) st = copy_plan(g, 0, &P);
  if (st == PW_OK) {
    const uint64_t K = (uint64_t)P.G * P.B, KR = K * P.R;  // after an ADAPTIVE second stage too
    if (budget) {
      budget[0] = P.B;
      budget[1] = P.G;
      budget[2] = K;
      budget[3] = P.R;
    }
    if (pilot) {
      pilot[0] = P.sigma2;
      pilot[1] = P.qbar;
      pilot[2] = P.theta;
    }
    if (q && K) cudaMemcpyAsync(q, (double*)g->ws.q.ptr + P.q_begin, sizeof(double) * K, cudaMemcpyDeviceToHost,
                                g->stream);
    if (u && KR) cudaMemcpyAsync(u, g->ws.u_debug.ptr, sizeof(float) * KR, cudaMemcpyDeviceToHost, g->stream);
    if (visits) cudaMemcpyAsync(visits, vis.ptr, sizeof(uint32_t) * (size_t)g->n, cudaMemcpyDeviceToHost, g->stream);
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) st = cuda_error(e, "debug copy-out");
  }
  free_buffer(vis);
  return st;
}

pw_status pw_query_blocks(pw_graph* g, int64_t s, int64_t t, double eps, int32_t L, const uint64_t* seed,
                          const pw_params* params, int64_t g_begin, int64_t g_end, double* block_means) {
  if (!g || !block_means) return set_error(PW_ERR_ARG, "NULL argument");
  if (s < 0 || s >= g->n || t < 0 || t >= g->n || s == t) return set_error(PW_ERR_ARG, "need 0 <= s != t < n");
  if (!(eps > 0.0 && eps < 1.0) || L < 0) return set_error(PW_ERR_ARG, "eps must lie in (0, 1) and L >= 0");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  BudgetArgs ba;
  pw_status st = resolve_budget(params, g, &ba, nullptr);
  if (st != PW_OK) return st;
  if (g_begin < 0 || g_end <= g_begin || g_end > (int64_t)ba.G) return set_error(PW_ERR_ARG, "block range outside [0, G)");
  if (ba.mode == PW_BUDGET_ADAPTIVE) return set_error(PW_ERR_ARG, "pw_query_blocks needs a budget fixed in advance");
  const uint64_t sd = seed ? *seed : default_seed(ba.global_seed, s, t, eps, L);
  DebugOut dbg;
  DeviceBuffer means;
  if ((st = ensure_buffer(means, sizeof(double) * (size_t)(g_end - g_begin))) != PW_OK) return st;
  dbg.g_begin = g_begin;
  dbg.g_end = g_end;
  dbg.block_means = (double*)means.ptr;
  double beta;
  int32_t qst = 0;
  st = host_batch(g, 1, &s, &t, &eps, &L, &sd, params, &beta, &qst, &dbg);
  if (st == PW_OK && qst != PW_OK) st = set_error((pw_status)qst, "query rejected");
  if (st == PW_OK) {
    cudaError_t e = cudaMemcpy(block_means, means.ptr, sizeof(double) * (size_t)(g_end - g_begin),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = cuda_error(e, "block means copy-out");
  }
  free_buffer(means);
  return st;
}

pw_status pw_query_stabilized(pw_graph* g, int64_t count, const int64_t* s, const int64_t* t, const double* eps,
                              int32_t L_max, const uint64_t* seeds, const pw_params* params, double* beta_hat,
                              int32_t* L_stop, int32_t* per_query_status) {
  if (!g) return set_error(PW_ERR_ARG, "graph is NULL");
  if (count < 0 || L_max < 2) return set_error(PW_ERR_ARG, "count < 0 or L_max < 2");
  if (count == 0) return PW_OK;
  if (!s || !t || !eps || !beta_hat || !L_stop || !per_query_status) return set_error(PW_ERR_ARG, "NULL array");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  BudgetArgs ba;
  pw_status st = resolve_budget(params, g, &ba, nullptr);
  if (st != PW_OK) return st;
  const size_t nq = (size_t)count;
  std::vector<uint64_t> qseed(nq);
  for (size_t i = 0; i < nq; ++i)
    qseed[i] = seeds ? seeds[i] : default_seed(ba.global_seed, s[i], t[i], eps[i], L_max);
  std::vector<double> prev(nq, 0.0);
  std::vector<int64_t> act;  // queries still doubling
  for (size_t i = 0; i < nq; ++i) {
    per_query_status[i] = PW_OK;
    L_stop[i] = 0;
    beta_hat[i] = 0.0;
    if (s[i] == t[i]) {
      L_stop[i] = 1;
    } else {
      act.push_back((int64_t)i);
    }
  }
  std::vector<int64_t> bs, bt;
  std::vector<double> be, bb;
  std::vector<int32_t> bL, bst;
  std::vector<uint64_t> bseed;
  for (int32_t L = 1; !act.empty(); L = L >= L_max ? L_max : (2 * L > L_max ? L_max : 2 * L)) {
    const size_t na = act.size();
    bs.resize(na); bt.resize(na); be.resize(na); bL.assign(na, L); bseed.resize(na); bb.resize(na); bst.resize(na);
    for (size_t j = 0; j < na; ++j) {
      const size_t i = (size_t)act[j];
      bs[j] = s[i];
      bt[j] = t[i];
      be[j] = eps[i];
      bseed[j] = level_seed(qseed[i], L);
    }
    st = host_batch(g, (int64_t)na, bs.data(), bt.data(), be.data(), bL.data(), bseed.data(), params, bb.data(),
                    bst.data(), nullptr);
    if (st != PW_OK) return st;
    std::vector<int64_t> next;
    for (size_t j = 0; j < na; ++j) {
      const size_t i = (size_t)act[j];
      if (bst[j] != PW_OK) {
        per_query_status[i] = bst[j];
        beta_hat[i] = bb[j];
        L_stop[i] = L;
        continue;
      }
      // Section 4.3: accept 2L once |beta(2L) - beta(L)| <= (eps/2) |beta(2L)|
      const bool stable = L > 1 && fabs(bb[j] - prev[i]) <= eps[i] / 2.0 * fabs(bb[j]);
      if (stable || L >= L_max) {
        beta_hat[i] = bb[j];
        L_stop[i] = L;
      } else {
        prev[i] = bb[j];
        next.push_back((int64_t)i);
      }
    }
    act.swap(next);
    if (L >= L_max) break;
  }
  return PW_OK;
}

pw_status pw_profile(pw_graph* g, int32_t enable, int32_t reset, pw_profile_stats* out) {
  if (!g) return set_error(PW_ERR_ARG, "graph is NULL");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  ProfileState& P = g->prof;
  if (!P.pending.empty()) PW_CUDA_TRY(cudaEventSynchronize(g->ws.last_use));
  for (Totals* h : P.pending) {
    P.transitions += 2ull * h->steps;
    P.spare.push_back(h);
  }
  P.pending.clear();
  for (auto& sp : P.spans) {
    PW_CUDA_TRY(cudaEventSynchronize(sp.b));
    float ms = 0.f;
    PW_CUDA_TRY(cudaEventElapsedTime(&ms, sp.a, sp.b));
    (sp.kind == 0 ? P.walk_ms : sp.kind == 1 ? P.pilot_ms : sp.kind == 2 ? P.finish_ms : P.series_ms) += ms;
    P.pool.push_back(sp.a);
    P.pool.push_back(sp.b);
  }
  P.spans.clear();
  if (out) {
    out->walk_ms = P.walk_ms;
    out->pilot_ms = P.pilot_ms;
    out->finish_ms = P.finish_ms;
    out->walk_launches = P.walk_launches;
    out->transitions = P.transitions;
    out->pilot_transitions = P.pilot_transitions;
    out->queries = P.queries;
    PW_CUDA_TRY(cudaEventSynchronize(g->ws.last_use));
    out->walk_mode = last_walk_mode(g);
    out->layout = g->layout;
    out->series_ms = P.series_ms;
    out->series_steps = P.series_steps;
  }
  if (reset) {
    P.walk_ms = P.pilot_ms = P.finish_ms = P.series_ms = 0;
    P.walk_launches = P.transitions = P.pilot_transitions = P.queries = P.series_steps = 0;
  }
  P.enabled = enable != 0;
  return PW_OK;
}

// Walk-kernel autotuner: time the sample in each walk kernel and its variants,
// keep the fastest variant of each, and fit the graph's cost model (per-visit:
// visits * visit_ns; table: probes * probe_ns + visits * table_visit_ns).  The
// runs use a FIXED budget (B = 4 probes per block, the caller's G, R = 1024 or
// 256 replicas), so the two table runs have the same probes and visits in the
// ratio 4: their timings separate the table build from the table walks.  (A
// PILOT budget would not do: its R follows the pilot, which depends on L.)
pw_status pw_autotune(pw_graph* g, int64_t count, const int64_t* s, const int64_t* t, const double* eps,
                      const int32_t* L, const uint64_t* seeds, const pw_params* params, pw_tune_result* out) {
  if (!g || !out) return set_error(PW_ERR_ARG, "NULL argument");
  if (count <= 0) return set_error(PW_ERR_ARG, "pw_autotune needs a non-empty sample");
  if (!s || !t || !eps || !L) return set_error(PW_ERR_ARG, "NULL array");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  memset(out, 0, sizeof *out);
  BudgetArgs ba;
  pw_status st = resolve_budget(params, g, &ba, nullptr);
  if (st != PW_OK) return st;
  pw_params p;
  if (params)
    p = *params;
  else
    memset(&p, 0, sizeof p);
  const pw_params caller = p;
  if ((st = set_l2_window(g, 0)) != PW_OK) return st;  // variants are timed without a window
  p.budget_mode = PW_BUDGET_FIXED;
  p.B = 16;
  p.G = ba.G;
  const uint64_t R_hi = 1024, R_lo = 256;
  const size_t nq = (size_t)count;
  std::vector<double> beta(nq);
  std::vector<int32_t> status(nq);
  // probes and visits of each timed run, from its totals
  struct Run {
    DebugOut d;
    double n_probes = 0, n_visits = 0;
  };
  // one warm-up and one timed run of the sample in walk kernel `mode` with R replicas
  auto timed = [&](int mode, uint64_t R, Run* r) -> pw_status {
    p.walk_mode = mode;
    p.R = R;
    for (int rep = 0; rep < 2; ++rep) {
      r->d = DebugOut();
      r->d.time_walk = true;
      const pw_status st2 = host_batch(g, count, s, t, eps, L, seeds, &p, beta.data(), status.data(), &r->d);
      if (st2 != PW_OK) return st2;
    }
    r->n_probes = (double)g->ws.host_totals->probes;
    r->n_visits = (double)g->ws.host_totals->visits;
    for (size_t i = 0; i < nq; ++i)
      if (status[i] != PW_OK) return set_error((pw_status)status[i], "pw_autotune: a sample query failed");
    return PW_OK;
  };
  Run dv, dt, dq;
  // per-visit kernel: registers left to the compiler or capped for 3 blocks/SM
  int best_minb = 1;
  for (int minb : {1, 3}) {
    g->visit_minb = minb;
    Run r;
    if ((st = timed(1, R_hi, &r)) != PW_OK) return st;
    if (minb == 1 || r.d.walk_ms < dv.d.walk_ms) {
      dv = r;
      best_minb = minb;
    }
  }
  g->visit_minb = best_minb;
  out->visit_occupancy = best_minb;
  out->sample_ms[0] = dv.d.walk_ms;
  out->visit_ns = dv.n_visits > 0 ? 1e6 * dv.d.walk_ms / dv.n_visits : 0.0;
  out->sample_mode = 1;
  // L2 windows, timed on the caller's budget with everything else as kept
  auto tune_window = [&]() -> pw_status {
    p = caller;
    p.walk_mode = 0;
    int best_w = 0;
    for (int w = 0; w < 3; ++w) {
      if (w == 2 && g->layout != 2) continue;
      if (set_l2_window(g, w) != PW_OK) continue;  // not available on this device
      DebugOut d;
      for (int rep = 0; rep < 2; ++rep) {
        d = DebugOut();
        d.time_walk = true;
        const pw_status st2 = host_batch(g, count, s, t, eps, L, seeds, &p, beta.data(), status.data(), &d);
        if (st2 != PW_OK) {
          set_l2_window(g, 0);
          return st2;
        }
      }
      out->window_ms[w] = d.walk_ms;
      // a window takes persisting L2 from the whole context: kept only when
      // it beats no window by 2 % or more
      if (w > 0 && d.walk_ms < 0.98 * out->window_ms[0] && d.walk_ms < out->window_ms[best_w]) best_w = w;
    }
    out->l2_window = best_w;
    return set_l2_window(g, best_w);
  };
  if (table_bytes(g) > kMaxTableBytes) {
    g->table_visit_gain = 0.0;  // the table cannot be built: always per-visit
    g->tuned = 1;
    return tune_window();
  }
  out->table_available = 1;
  // table kernel: block size
  int best_threads = 256;
  for (int threads : {256, 512, 1024}) {
    g->table_threads = threads;
    Run r;
    if ((st = timed(2, R_hi, &r)) != PW_OK) return st;
    if (threads == 256 || r.d.walk_ms < dt.d.walk_ms) {
      dt = r;
      best_threads = threads;
    }
  }
  g->table_threads = best_threads;
  out->table_threads = best_threads;
  if ((st = timed(2, R_lo, &dq)) != PW_OK) return st;
  out->sample_ms[1] = dt.d.walk_ms;
  out->sample_ms[2] = dq.d.walk_ms;
  // solve  T = P c + V w  for the two table runs (times in ns)
  const double T2 = 1e6 * dt.d.walk_ms, T3 = 1e6 * dq.d.walk_ms;
  const double P2 = dt.n_probes, P3 = dq.n_probes, V2 = dt.n_visits, V3 = dq.n_visits;
  const double det = P2 * V3 - P3 * V2;
  double c = 0.0, w = 0.0;
  if (det != 0.0) {
    c = (T2 * V3 - T3 * V2) / det;
    w = (P2 * T3 - P3 * T2) / det;
  }
  if (det == 0.0 || c < 0.0 || w < 0.0) {  // degenerate sample: attribute the larger share alone
    if (det != 0.0 && c < 0.0) {
      c = 0.0;
      w = V2 > 0.0 ? T2 / V2 : 0.0;
    } else {
      w = 0.0;
      c = P2 > 0.0 ? T2 / P2 : 0.0;
    }
  }
  out->table_probe_ns = c;
  out->table_visit_ns = w;
  g->table_probe_cost = c;
  g->table_visit_gain = out->visit_ns - w;
  g->tuned = 1;
  const double Vs = dv.n_visits, Ps = dv.n_probes;
  out->sample_mode = Ps * g->table_probe_cost < Vs * g->table_visit_gain ? 2 : 1;
  // policy check on the caller's own budget (PILOT: R from the pilot): the
  // fitted per-query model against every query per-visit and every query on
  // the table, each timed once more; the fastest is kept
  p = caller;
  double best_ms = 0.0;
  int best_policy = 0;
  for (int policy : {0, 1, 2}) {
    g->walk_policy = policy;
    DebugOut d;
    for (int rep = 0; rep < 2; ++rep) {
      d = DebugOut();
      d.time_walk = true;
      p.walk_mode = 0;
      if ((st = host_batch(g, count, s, t, eps, L, seeds, &p, beta.data(), status.data(), &d)) != PW_OK) return st;
    }
    out->policy_ms[policy] = d.walk_ms;
    if (policy == 0 || d.walk_ms < best_ms) {
      best_ms = d.walk_ms;
      best_policy = policy;
    }
  }
  // A model that mixes the kernels runs two walk launches per batch, each
  // with its own tail; a single-kernel policy within 1 % of it is kept instead.
  if (best_policy == 0) {
    const int single = out->policy_ms[1] <= out->policy_ms[2] ? 1 : 2;
    if (out->policy_ms[single] <= 1.01 * out->policy_ms[0]) best_policy = single;
  }
  g->walk_policy = best_policy;
  out->policy = best_policy;
  return tune_window();
}

pw_status pw_debug_exact_sum(pw_graph* g, const float* u, int64_t n, double* S1, double* S2) {
  if (!g || (!u && n > 0) || !S1 || !S2 || n < 0) return set_error(PW_ERR_ARG, "NULL argument or n < 0");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  DeviceBuffer b;
  pw_status st = ensure_buffer(b, sizeof(float) * (size_t)n + 64);
  if (st != PW_OK) return st;
  float* du = (float*)((char*)b.ptr + 64);
  double* dout = (double*)b.ptr;
  cudaError_t e = n ? cudaMemcpyAsync(du, u, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, g->stream) : cudaSuccess;
  if (e == cudaSuccess) {
    debug_exact_sum_kernel<<<1, 256, 0, g->stream>>>(du, n, dout);
    count_launch();
    e = cudaGetLastError();
  }
  double out[2] = {0.0, 0.0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof out, cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  free_buffer(b);
  if (e != cudaSuccess) return cuda_error(e, "pw_debug_exact_sum");
  *S1 = out[0];
  *S2 = out[1];
  return PW_OK;
}

pw_status pw_debug_batch_probe_q(pw_graph* g, int64_t count, const int64_t* s, const int64_t* t,
                                 const double* eps, const int32_t* L, const uint64_t* seeds,
                                 const pw_params* params, double* beta_hat, int32_t* per_query_status,
                                 uint64_t* KR, int64_t n_sel, const int64_t* sel_query, const int64_t* sel_probe,
                                 double* q_sel) {
  if (!g) return set_error(PW_ERR_ARG, "graph is NULL");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  pw_status st = host_batch(g, count, s, t, eps, L, seeds, params, beta_hat, per_query_status, nullptr);
  if (st != PW_OK || count == 0) return st;
  std::vector<QPlan> plans((size_t)count);
  PW_CUDA_TRY(cudaMemcpyAsync(plans.data(), g->ws.plans.ptr, sizeof(QPlan) * (size_t)count, cudaMemcpyDeviceToHost,
                              g->stream));
  PW_CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (KR)
    for (int64_t i = 0; i < count; ++i) {
      KR[2 * i] = (uint64_t)plans[(size_t)i].G * plans[(size_t)i].B;
      KR[2 * i + 1] = plans[(size_t)i].R;
    }
  for (int64_t i = 0; i < n_sel; ++i) {
    const int64_t qi = sel_query[i], k = sel_probe[i];
    if (qi < 0 || qi >= count || k < 0 || (uint64_t)k >= (uint64_t)plans[(size_t)qi].G * plans[(size_t)qi].B)
      return set_error(PW_ERR_ARG, "selection out of range");
    PW_CUDA_TRY(cudaMemcpyAsync(q_sel + i, (double*)g->ws.q.ptr + plans[(size_t)qi].q_begin + k, sizeof(double),
                                cudaMemcpyDeviceToHost, g->stream));
  }
  PW_CUDA_TRY(cudaStreamSynchronize(g->stream));
  return PW_OK;
}

}  // extern "C"

namespace pw {

// ---------------------------------------------------------------------------
// Batch entry point that allocates nothing.
//
// Some callers cannot allocate device memory while they run queries: a
// real-time service that forbids allocator calls (cudaMalloc can block and
// synchronise the device) in its request path, or code that runs where the
// CUDA allocator is off limits.  pw_query_batch_noalloc serves them: its
// scratch (query plans, offsets, counters, pilot sums, Q_R values and probe
// accumulators) is carved out of the file-scope array below, so the call
// itself makes no cudaMalloc, cudaFree or allocating library call.  The array
// holds kNoAllocScratchBytes on every GPU that loads the library, until the
// process exits.  Every call shares it: calls that overlap on the GPU
// (different streams, or another thread) race on its contents; the counters
// and accumulators that must start at zero are cleared by each call.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;
static __device__ __align__(256) unsigned char pw_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_lock;
static void* g_noalloc_addr[128] = {nullptr};

// Device address of the scratch array on `device` (which must be current).
// In host code the array's name is only a host-side stand-in, so the real
// address comes from cudaGetSymbolAddress, once per device.
static pw_status noalloc_scratch(int device, unsigned char** out) {
  if (device < 0 || device >= 128) return set_error(PW_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> guard(g_noalloc_lock);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, pw_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(pw_noalloc_scratch)");
    g_noalloc_addr[device] = p;
  }
  *out = (unsigned char*)g_noalloc_addr[device];
  return PW_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace pw

extern "C" pw_status pw_query_batch_noalloc(pw_graph* g, int64_t count, const int64_t* d_s, const int64_t* d_t,
                                            const double* d_eps, const int32_t* d_L, const uint64_t* d_seeds,
                                            const pw_params* params, double* d_beta_hat, int32_t* d_status,
                                            void* stream_ptr) {
  using namespace pw;
  if (!g) return set_error(PW_ERR_ARG, "graph is NULL");
  if (count < 0) return set_error(PW_ERR_ARG, "count < 0");
  if (count == 0) return PW_OK;
  if (!d_s || !d_t || !d_eps || !d_L || !d_beta_hat || !d_status) return set_error(PW_ERR_ARG, "NULL device array");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  BudgetArgs ba;
  pw_status st = resolve_budget(params, g, &ba, nullptr);
  if (st != PW_OK) return st;
  unsigned char* base = nullptr;
  if ((st = noalloc_scratch(g->device, &base)) != PW_OK) return st;
  cudaStream_t stream = (cudaStream_t)stream_ptr;
  const size_t nq = (size_t)count;
  // plans and counters first: the sum of K over the batch sizes the rest
  size_t off = 0;
  const size_t o_plans = off;
  off = align256(off + sizeof(QPlan) * nq);
  const size_t o_counters = off;
  off = align256(off + 64);
  if (off > kNoAllocScratchBytes)
    return set_error(PW_ERR_NOMEM, "pw_query_batch_noalloc: batch needs more than the 64 MiB static scratch");
  BatchBuffers B;
  B.plans = (QPlan*)(base + o_plans);
  B.counters = (unsigned long long*)(base + o_counters);
  PW_CUDA_TRY(cudaStreamWaitEvent(stream, g->ws.last_use, 0));
  const int qthreads = 128;
  const int qblocks = (int)((count + qthreads - 1) / qthreads);
  budget_init_kernel<<<qblocks, qthreads, 0, stream>>>(count, d_s, d_t, d_eps, d_L, d_seeds, ba, g->n, g->d_node,
                                                       B.plans, nullptr);
  count_launch();
  sum_k_kernel<<<1, 1024, 0, stream>>>(B.plans, count, B.counters + 7);
  count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  PW_CUDA_TRY(cudaMemcpyAsync(&g->ws.host_totals->pad[0], B.counters + 7, 8, cudaMemcpyDeviceToHost, stream));
  PW_CUDA_TRY(cudaStreamSynchronize(stream));
  const BatchSizes z = batch_sizes(nq, (size_t)g->ws.host_totals->pad[0], ba);
  const size_t o_pplans = off;
  off = align256(off + z.plans);
  const size_t o_prefix = off;
  off = align256(off + z.prefix);
  const size_t o_totals = off;
  off = align256(off + z.totals);
  const size_t o_pilot = off;
  off = align256(off + z.pilot_s);
  const size_t o_q = off;
  off = align256(off + z.q);
  const size_t o_acc = off;
  off = align256(off + z.acc);
  if (off > kNoAllocScratchBytes)
    return set_error(PW_ERR_NOMEM, "pw_query_batch_noalloc: the probes of this batch need more than the 64 MiB "
                                   "static scratch (104 bytes per probe); split the batch");
  B.pplans = (QPlan*)(base + o_pplans);
  B.prefix = (unsigned long long*)(base + o_prefix);
  B.totals = (Totals*)(base + o_totals);
  B.pilot_s = (double*)(base + o_pilot);
  B.q = (double*)(base + o_q);
  B.acc = (ProbeAcc*)(base + o_acc);
  if ((st = enqueue_budget(g, count, d_s, d_t, d_eps, d_L, d_seeds, ba, B, stream)) != PW_OK) return st;
  if ((st = enqueue_walks(g, count, params, ba, B, d_beta_hat, d_status, stream, nullptr)) != PW_OK) return st;
  PW_CUDA_TRY(cudaMemcpyAsync(g->ws.host_totals, B.totals, sizeof(Totals), cudaMemcpyDeviceToHost, stream));
  PW_CUDA_TRY(cudaEventRecord(g->ws.last_use, stream));
  return PW_OK;
}
