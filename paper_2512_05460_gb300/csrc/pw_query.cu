// Query pipeline of Algorithm 1 on the device:
//   budget (line 1) -> [pilot walks + pilot budget] -> tile/U/probe offsets ->
//   persistent walk kernel (lines 2-11) -> per-probe U-statistic (lines 12-14)
//   -> median of block means (lines 16-20).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pw_budget.cuh"
#include "pw_device.cuh"
#include "pw_internal.h"
#include "pw_walk.cuh"

namespace pw {

constexpr int kWalkThreads = 256;

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

// PILOT: R >= 4 sigma^2 / theta (Lemma 3.7) from the pilot replicas, in the
// oracle's summation order (per probe over replicas, then over probes).
__global__ void pilot_budget_kernel(int64_t nq, QPlan* __restrict__ plans, const QPlan* __restrict__ pilot,
                                    const float* __restrict__ pilot_u, BudgetArgs A, const int4* __restrict__ node) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const QPlan PP = pilot[q];
  if (PP.K == 0) return;
  QPlan& P = plans[q];
  double sum_var = 0.0, sum_q = 0.0;
  for (uint32_t k = 0; k < PP.K; ++k) {
    const float* u = pilot_u + PP.u_begin + (uint64_t)k * PP.R;
    double S1 = 0.0, S2 = 0.0;
    for (uint32_t p = 0; p < PP.R; ++p) accumulate_s(S1, S2, u[p]);
    pilot_accumulate(sum_var, sum_q, S1, S2, PP.R);
  }
  pilot_finish(P, sum_var, sum_q, PP.K, node[P.s].z, node[P.t].z, A);
}

// Exclusive offsets of tiles (K*chunks), U slots (K*R) and probes (K); one
// block.  prefix[0..nq] are tile offsets, prefix[nq+1..2nq+1] probe offsets.
__global__ void scan_kernel(QPlan* __restrict__ plans, int64_t nq, unsigned long long* __restrict__ prefix,
                            Totals* __restrict__ totals) {
  __shared__ unsigned long long sh[3][1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t per = (nq + nt - 1) / nt;
  const int64_t b0 = per * tid, b = b0 < nq ? b0 : nq, e = b + per < nq ? b + per : nq;
  unsigned long long st = 0, su = 0, sp = 0, ss = 0;
  for (int64_t q = b; q < e; ++q) {
    const QPlan& P = plans[q];
    st += (unsigned long long)P.K * P.chunks;
    su += (unsigned long long)P.K * P.R;
    sp += P.K;
    ss += (unsigned long long)P.K * P.R * (unsigned long long)(P.L > 0 ? P.L : 0);
  }
  sh[0][tid] = st;
  sh[1][tid] = su;
  sh[2][tid] = sp;
  __shared__ unsigned long long steps_sh[1024];
  steps_sh[tid] = ss;
  __syncthreads();
  if (tid == 0) {
    unsigned long long a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (int i = 0; i < nt; ++i) {
      const unsigned long long x0 = sh[0][i], x1 = sh[1][i], x2 = sh[2][i];
      sh[0][i] = a0;
      sh[1][i] = a1;
      sh[2][i] = a2;
      a0 += x0;
      a1 += x1;
      a2 += x2;
      a3 += steps_sh[i];
    }
    totals->tiles = a0;
    totals->u_slots = a1;
    totals->probes = a2;
    totals->steps = a3;
    prefix[nq] = a0;
    prefix[2 * nq + 1] = a2;
  }
  __syncthreads();
  st = sh[0][tid];
  su = sh[1][tid];
  sp = sh[2][tid];
  for (int64_t q = b; q < e; ++q) {
    QPlan& P = plans[q];
    P.tile_begin = st;
    P.u_begin = su;
    P.probe_begin = sp;
    prefix[q] = st;
    prefix[nq + 1 + q] = sp;
    st += (unsigned long long)P.K * P.chunks;
    su += (unsigned long long)P.K * P.R;
    sp += P.K;
  }
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
  const int4* rec;
  const int4* node;
  const QPlan* plans;
  const unsigned long long* tile_prefix;
  const Totals* totals;
  unsigned long long* tile_counter;
  float* u;
  uint32_t* visits;
  int64_t nq;
  uint32_t n;
  uint32_t walk_tag, probe_tag;
};

// Persistent walk kernel: each warp pops tiles (query, probe k, 32 replicas)
// from a device counter until the work runs out; lane l runs replica 32c + l.
template <bool DEBUG>
__global__ void __launch_bounds__(kWalkThreads) walk_kernel(WalkArgs A) {
  const uint32_t lane = threadIdx.x & 31u;
  const unsigned long long total = A.totals->tiles;
  for (;;) {
    unsigned long long tile = 0;
    if (lane == 0) tile = atomicAdd(A.tile_counter, 1ull);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= total) return;
    const int64_t q = find_segment(A.tile_prefix, A.nq, tile);
    const QPlan& P = A.plans[q];
    const uint32_t chunks = P.chunks, R = P.R;
    const unsigned long long local = tile - P.tile_begin;
    const uint32_t kl = (uint32_t)(local / chunks);
    const uint32_t c = (uint32_t)(local - (unsigned long long)kl * chunks);
    const uint32_t p = c * 32u + lane;
    if (p >= R) continue;
    const uint32_t k = P.k_begin + kl;
    const Probe pr = make_probe(A.n, P.seed, k, A.probe_tag);
    const uint64_t pair = (uint64_t)k * R + p;
    const ZOnTheFly zp{pr};
    const float U = walk_pair<DEBUG>(A.rec, A.node, A.visits, A.walk_tag, zp, P.s, P.t, P.L, P.seed, pair);
    A.u[P.u_begin + (uint64_t)kl * R + p] = U;
  }
}

// Probe-major kernel: a block claims one probe k of one query, writes the
// whole vector z^(k) into a shared-memory table (sign bits plus the zero set;
// one Feistel cycle-walk per node), then its warps run the
// probe's 32-replica tiles reading z from the table.  Same values as the
// on-the-fly kernel; cheaper whenever a probe's walks visit more nodes than
// the graph has (2 R (L+1) > n).
template <bool DEBUG>
__global__ void __launch_bounds__(kWalkThreads, 5) walk_table_kernel(WalkArgs A,
                                                                  const unsigned long long* __restrict__ probe_prefix,
                                                                  unsigned long long* __restrict__ probe_counter) {
  extern __shared__ uint32_t tab[];
  __shared__ unsigned long long sh_probe;
  __shared__ uint32_t sh_tile;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = A.n;
  const unsigned long long total = A.totals->probes;
  for (;;) {
    if (threadIdx.x == 0) {
      sh_probe = atomicAdd(probe_counter, 1ull);
      sh_tile = 0;
    }
    __syncthreads();
    const unsigned long long j = sh_probe;
    if (j >= total) return;
    const int64_t q = find_segment(probe_prefix, A.nq, j);
    const QPlan& P = A.plans[q];
    const uint32_t kl = (uint32_t)(j - P.probe_begin);
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
      if (p < R) {
        const uint64_t pair = (uint64_t)k * R + p;
        const float U = walk_pair_table<DEBUG>(A.rec, A.node, A.visits, A.walk_tag, zp, P.s, P.t, P.L, P.seed, pair);
        A.u[P.u_begin + (uint64_t)kl * R + p] = U;
      }
    }
    __syncthreads();
  }
}

// Q_R per probe (Eq. Q-Ustat): S1, S2 in FP64 over replicas in order.
__global__ void probe_finish_kernel(const QPlan* __restrict__ plans, int64_t nq,
                                    const unsigned long long* __restrict__ probe_prefix,
                                    const Totals* __restrict__ totals, const float* __restrict__ u,
                                    double* __restrict__ qbuf) {
  const unsigned long long total = totals->probes;
  for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < total;
       j += (unsigned long long)gridDim.x * blockDim.x) {
    const int64_t q = find_segment(probe_prefix, nq, j);
    const QPlan& P = plans[q];
    const unsigned long long k = j - P.probe_begin;
    const float* x = u + P.u_begin + k * P.R;
    double S1 = 0.0, S2 = 0.0;
    for (uint32_t p = 0; p < P.R; ++p) accumulate_s(S1, S2, x[p]);
    qbuf[j] = u_statistic(S1, S2, P.R);
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
    const double* x = qbuf + P.probe_begin + (uint64_t)g * P.B;
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
    const double* x = qbuf + P.probe_begin + (uint64_t)g * P.B;
    double sum = 0.0;
    for (uint32_t k = 0; k < P.B; ++k) sum = __dadd_rn(sum, x[k]);
    means[g] = __ddiv_rn(sum, (double)P.B);
  }
  if (threadIdx.x == 0) status[0] = P.status;
}

static int walk_grid(pw_graph* g, bool debug) {
  static int occ[2] = {0, 0};
  int& o = occ[debug ? 1 : 0];
  if (o == 0) {
    int nb = 0;
    if (debug)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, walk_kernel<true>, kWalkThreads, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, walk_kernel<false>, kWalkThreads, 0);
    o = nb > 0 ? nb : 1;
  }
  return g->sm_count * o;
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

static int table_grid(pw_graph* g, bool debug, size_t smem) {
  int nb = 0;
  if (debug) {
    cudaFuncSetAttribute(walk_table_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, walk_table_kernel<true>, kWalkThreads, smem);
  } else {
    cudaFuncSetAttribute(walk_table_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, walk_table_kernel<false>, kWalkThreads, smem);
  }
  return g->sm_count * (nb > 0 ? nb : 1);
}

// Walk kernel of a batch: the caller's walk_mode, else the graph's cost model
// (probe table when probes * table_probe_cost < visits * table_visit_gain,
// 2 R (L+1) visits per probe); the table needs its bits in shared memory.
static int pick_walk_mode(const pw_graph* g, const pw_params* params, const Totals& T) {
  int mode = params ? params->walk_mode : 0;
  if (mode == 0) {
    const double visits = 2.0 * ((double)T.steps + (double)T.u_slots);
    mode = (table_bytes(g) <= kMaxTableBytes && (double)T.probes * g->table_probe_cost < visits * g->table_visit_gain)
               ? 2
               : 1;
  }
  if (mode == 2 && table_bytes(g) > kMaxTableBytes) mode = 1;
  return mode;
}

static pw_status launch_walk_table(pw_graph* g, cudaStream_t stream, bool debug, const WalkArgs& a,
                                   const unsigned long long* probe_prefix, unsigned long long* probe_counter) {
  const size_t smem = table_bytes(g);
  const int grid = table_grid(g, debug, smem);
  if (debug)
    walk_table_kernel<true><<<grid, kWalkThreads, smem, stream>>>(a, probe_prefix, probe_counter);
  else
    walk_table_kernel<false><<<grid, kWalkThreads, smem, stream>>>(a, probe_prefix, probe_counter);
  count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  return PW_OK;
}

static pw_status launch_walk(pw_graph* g, cudaStream_t stream, bool debug, const WalkArgs& a) {
  const int grid = walk_grid(g, debug);
  if (debug)
    walk_kernel<true><<<grid, kWalkThreads, 0, stream>>>(a);
  else
    walk_kernel<false><<<grid, kWalkThreads, 0, stream>>>(a);
  count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  return PW_OK;
}

pw_status run_batch(pw_graph* g, int64_t count, const int64_t* d_s, const int64_t* d_t, const double* d_eps,
                    const int32_t* d_L, const uint64_t* d_seeds, const pw_params* params, double* d_beta,
                    int32_t* d_status, cudaStream_t stream, DebugOut* dbg) {
  BudgetArgs ba;
  pw_status st = resolve_budget(params, g, &ba, nullptr);
  if (st != PW_OK) return st;
  if (count < 0) return set_error(PW_ERR_ARG, "count < 0");
  if (count == 0) return PW_OK;
  Workspace& ws = g->ws;
  PW_CUDA_TRY(cudaStreamWaitEvent(stream, ws.last_use, 0));
  const bool pilot = ba.mode == PW_BUDGET_PILOT;
  const size_t nq = (size_t)count;
  if ((st = ensure_buffer(ws.plans, sizeof(QPlan) * nq)) != PW_OK) return st;
  if ((st = ensure_buffer(ws.pilot_plans, sizeof(QPlan) * nq)) != PW_OK) return st;
  if ((st = ensure_buffer(ws.tile_prefix, sizeof(unsigned long long) * 4 * (nq + 1))) != PW_OK) return st;
  if ((st = ensure_buffer(ws.totals, sizeof(Totals) * 2)) != PW_OK) return st;
  if ((st = ensure_buffer(ws.counters, 64)) != PW_OK) return st;
  QPlan* plans = (QPlan*)ws.plans.ptr;
  QPlan* pplans = (QPlan*)ws.pilot_plans.ptr;
  unsigned long long* prefix = (unsigned long long*)ws.tile_prefix.ptr;
  unsigned long long* pprefix = prefix + 2 * (nq + 1);
  Totals* totals = (Totals*)ws.totals.ptr;
  unsigned long long* counters = (unsigned long long*)ws.counters.ptr;
  PW_CUDA_TRY(cudaMemsetAsync(counters, 0, 64, stream));
  const int qthreads = 128;
  const int qblocks = (int)((count + qthreads - 1) / qthreads);
  budget_init_kernel<<<qblocks, qthreads, 0, stream>>>(count, d_s, d_t, d_eps, d_L, d_seeds, ba, g->n, g->d_node,
                                                       plans, pilot ? pplans : nullptr);
  count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  WalkArgs wa;
  wa.rec = g->d_rec;
  wa.node = g->d_node;
  wa.nq = count;
  wa.n = (uint32_t)g->n;
  wa.visits = nullptr;
  if (pilot) {
    const size_t pslots = nq * (size_t)ba.K0 * (size_t)ba.R0;
    if ((st = ensure_buffer(ws.pilot_u, sizeof(float) * pslots)) != PW_OK) return st;
    scan_kernel<<<1, 1024, 0, stream>>>(pplans, count, pprefix, totals + 1);
    count_launch();
    wa.plans = pplans;
    wa.tile_prefix = pprefix;
    wa.totals = totals + 1;
    wa.tile_counter = counters + 1;
    wa.u = (float*)ws.pilot_u.ptr;
    wa.walk_tag = kTagWalkPilot;
    wa.probe_tag = kTagProbePilot;
    cudaEvent_t ev;
    prof_begin(g, stream, &ev);
    if ((st = launch_walk(g, stream, false, wa)) != PW_OK) return st;
    prof_end(g, stream, ev, 1);
    if (g->prof.enabled) g->prof.pilot_transitions += 2ull * nq * (uint64_t)ba.K0 * (uint64_t)ba.R0;
    pilot_budget_kernel<<<qblocks, qthreads, 0, stream>>>(count, plans, pplans, (const float*)ws.pilot_u.ptr, ba,
                                                          g->d_node);
    count_launch();
    PW_CUDA_TRY(cudaGetLastError());
  }
  const bool sharded = dbg && dbg->g_begin >= 0;
  if (sharded) {
    restrict_blocks_kernel<<<1, 1, 0, stream>>>(plans, (uint32_t)dbg->g_begin, (uint32_t)dbg->g_end);
    count_launch();
    PW_CUDA_TRY(cudaGetLastError());
  }
  scan_kernel<<<1, 1024, 0, stream>>>(plans, count, prefix, totals);
  count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  PW_CUDA_TRY(cudaMemcpyAsync(ws.host_totals, totals, sizeof(Totals), cudaMemcpyDeviceToHost, stream));
  PW_CUDA_TRY(cudaStreamSynchronize(stream));
  const Totals T = *ws.host_totals;
  if (dbg && dbg->budget_only) {
    PW_CUDA_TRY(cudaEventRecord(ws.last_use, stream));
    return PW_OK;
  }
  if ((st = ensure_buffer(ws.u, sizeof(float) * (size_t)T.u_slots)) != PW_OK) return st;
  if ((st = ensure_buffer(ws.q, sizeof(double) * (size_t)T.probes)) != PW_OK) return st;
  const bool debug = dbg && dbg->visits;
  wa.plans = plans;
  wa.tile_prefix = prefix;
  wa.totals = totals;
  wa.tile_counter = counters;
  wa.u = (float*)ws.u.ptr;
  wa.visits = debug ? dbg->visits : nullptr;
  wa.walk_tag = kTagWalk;
  wa.probe_tag = kTagProbe;
  const int mode = pick_walk_mode(g, params, T);
  g->last_walk_mode = mode;
  cudaEvent_t ev_walk;
  prof_begin(g, stream, &ev_walk);
  cudaEvent_t tw[2] = {nullptr, nullptr};
  if (dbg && dbg->time_walk) {
    dbg->n_probes = T.probes;
    dbg->n_visits = 2ull * (T.steps + T.u_slots);
    PW_CUDA_TRY(cudaEventCreate(&tw[0]));
    cudaError_t e = cudaEventCreate(&tw[1]);
    if (e == cudaSuccess) e = cudaEventRecord(tw[0], stream);
    if (e != cudaSuccess) {
      cudaEventDestroy(tw[0]);
      if (tw[1]) cudaEventDestroy(tw[1]);
      return cuda_error(e, "walk timing events");
    }
  }
  if (T.tiles > 0) {
    if (mode == 2)
      st = launch_walk_table(g, stream, debug, wa, prefix + nq + 1, counters + 2);
    else
      st = launch_walk(g, stream, debug, wa);
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
    g->prof.walk_launches += T.tiles > 0 ? 1 : 0;
    g->prof.transitions += 2ull * T.steps;
    g->prof.queries += nq;
  }
  cudaEvent_t ev_fin;
  prof_begin(g, stream, &ev_fin);
  if (T.probes > 0) {
    const int fthreads = 128;
    const unsigned long long want = (T.probes + fthreads - 1) / fthreads;
    const int fblocks = (int)std::min<unsigned long long>(want, (unsigned long long)g->sm_count * 64);
    probe_finish_kernel<<<fblocks, fthreads, 0, stream>>>(plans, count, prefix + nq + 1, totals,
                                                          (const float*)ws.u.ptr, (double*)ws.q.ptr);
    count_launch();
    PW_CUDA_TRY(cudaGetLastError());
  }
  if (sharded)
    block_means_kernel<<<1, 128, 0, stream>>>(plans, (const double*)ws.q.ptr, dbg->block_means, d_status);
  else
    mom_kernel<<<(unsigned)count, 128, 0, stream>>>(plans, (const double*)ws.q.ptr, d_beta, d_status);
  count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  prof_end(g, stream, ev_fin, 2);
  PW_CUDA_TRY(cudaEventRecord(ws.last_use, stream));
  return PW_OK;
}

// Host-array batch: stage inputs in pinned memory, run, copy results back.
static pw_status host_batch(pw_graph* g, int64_t count, const int64_t* s, const int64_t* t, const double* eps,
                            const int32_t* L, const uint64_t* seeds, const pw_params* params, double* beta,
                            int32_t* status, DebugOut* dbg) {
  if (count < 0) return set_error(PW_ERR_ARG, "count < 0");
  if (count == 0) return PW_OK;
  if (!s || !t || !eps || !L || !beta || !status) return set_error(PW_ERR_ARG, "NULL array");
  Workspace& ws = g->ws;
  const size_t nq = (size_t)count;
  const size_t in_bytes = nq * (8 + 8 + 8 + 8 + 4), out_bytes = nq * (8 + 4);
  pw_status st;
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
    BudgetArgs ba;
    if ((st = resolve_budget(params, g, &ba, nullptr)) != PW_OK) return st;
    for (size_t i = 0; i < nq; ++i)
      ((uint64_t*)(h + nq * 24))[i] = default_seed(ba.global_seed, s[i], t[i], eps[i], L[i]);
  }
  memcpy(h + nq * 32, L, nq * 4);
  char* d = (char*)ws.queries.ptr;
  PW_CUDA_TRY(cudaMemcpyAsync(d, h, in_bytes, cudaMemcpyHostToDevice, g->stream));
  double* d_beta = (double*)ws.results.ptr;
  int32_t* d_status = (int32_t*)((char*)ws.results.ptr + nq * 8);
  st = run_batch(g, count, (const int64_t*)d, (const int64_t*)(d + nq * 8), (const double*)(d + nq * 16),
                 (const int32_t*)(d + nq * 32), (const uint64_t*)(d + nq * 24), params, d_beta, d_status, g->stream,
                 dbg);
  if (st != PW_OK) return st;
  if (dbg && dbg->budget_only) return PW_OK;
  char* ho = h + in_bytes;
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
                   nullptr);
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
  DebugOut dbg;
  DeviceBuffer vis;
  if (visits) {
    if ((st = ensure_buffer(vis, sizeof(uint32_t) * (size_t)g->n)) != PW_OK) return st;
    PW_CUDA_TRY(cudaMemsetAsync(vis.ptr, 0, sizeof(uint32_t) * (size_t)g->n, g->stream));
    dbg.visits = (uint32_t*)vis.ptr;
  }
  int32_t qst = 0;
  st = host_batch(g, 1, &s, &t, &eps, &L, &sd, params, beta_hat, &qst, &dbg);
  if (st == PW_OK && qst != PW_OK) st = set_error((pw_status)qst, "query rejected");
  QPlan P;
  memset(&P, 0, sizeof P);
  if (st == PW_OK) st = copy_plan(g, 0, &P);
  if (st == PW_OK) {
    if (budget) {
      budget[0] = P.B;
      budget[1] = P.G;
      budget[2] = P.K;
      budget[3] = P.R;
    }
    if (pilot) {
      pilot[0] = P.sigma2;
      pilot[1] = P.qbar;
      pilot[2] = P.theta;
    }
    const uint64_t K = P.K, KR = (uint64_t)P.K * P.R;
    if ((q && (uint64_t)q_cap < K) || (u && (uint64_t)u_cap < KR)) {
      st = set_error(PW_ERR_ARG, "q_cap or u_cap too small");
    } else {
      if (q && K) cudaMemcpyAsync(q, (double*)g->ws.q.ptr + P.probe_begin, sizeof(double) * K, cudaMemcpyDeviceToHost,
                                  g->stream);
      if (u && KR) cudaMemcpyAsync(u, (float*)g->ws.u.ptr + P.u_begin, sizeof(float) * KR, cudaMemcpyDeviceToHost,
                                   g->stream);
      if (visits)
        cudaMemcpyAsync(visits, vis.ptr, sizeof(uint32_t) * (size_t)g->n, cudaMemcpyDeviceToHost, g->stream);
      cudaError_t e = cudaStreamSynchronize(g->stream);
      if (e != cudaSuccess) st = cuda_error(e, "debug copy-out");
    }
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
    out->walk_mode = g->last_walk_mode;
    out->reserved = 0;
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

// Walk-kernel autotuner: time the sample in each walk kernel and fit the
// graph's cost model (per-visit: visits * visit_ns; table: probes * probe_ns +
// visits * table_visit_ns).  The two table runs differ only in L, which moves
// the visits but not the probes (K depends on eps alone), so the pair of
// timings separates the table build from the table walks.
pw_status pw_autotune(pw_graph* g, int64_t count, const int64_t* s, const int64_t* t, const double* eps,
                      const int32_t* L, const uint64_t* seeds, const pw_params* params, pw_tune_result* out) {
  if (!g || !out) return set_error(PW_ERR_ARG, "NULL argument");
  if (count <= 0) return set_error(PW_ERR_ARG, "pw_autotune needs a non-empty sample");
  if (!s || !t || !eps || !L) return set_error(PW_ERR_ARG, "NULL array");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  memset(out, 0, sizeof *out);
  pw_params p;
  if (params)
    p = *params;
  else
    memset(&p, 0, sizeof p);
  const size_t nq = (size_t)count;
  std::vector<double> beta(nq);
  std::vector<int32_t> status(nq);
  std::vector<int32_t> L4(nq);
  for (size_t i = 0; i < nq; ++i) L4[i] = L[i] >= 4 ? L[i] / 4 : 4 * L[i];
  // one warm-up and one timed run of the sample in walk kernel `mode`
  auto timed = [&](int mode, const int32_t* Ls, DebugOut* d) -> pw_status {
    p.walk_mode = mode;
    for (int rep = 0; rep < 2; ++rep) {
      *d = DebugOut();
      d->time_walk = true;
      const pw_status st = host_batch(g, count, s, t, eps, Ls, seeds, &p, beta.data(), status.data(), d);
      if (st != PW_OK) return st;
    }
    for (size_t i = 0; i < nq; ++i)
      if (status[i] != PW_OK) return set_error((pw_status)status[i], "pw_autotune: a sample query failed");
    return PW_OK;
  };
  DebugOut dv, dt, dq;
  pw_status st = timed(1, L, &dv);
  if (st != PW_OK) return st;
  out->sample_ms[0] = dv.walk_ms;
  out->visit_ns = dv.n_visits ? 1e6 * dv.walk_ms / (double)dv.n_visits : 0.0;
  out->sample_mode = 1;
  if (table_bytes(g) > kMaxTableBytes) {
    g->table_visit_gain = 0.0;  // the table cannot be built: always per-visit
    g->tuned = 1;
    return PW_OK;
  }
  out->table_available = 1;
  if ((st = timed(2, L, &dt)) != PW_OK) return st;
  if ((st = timed(2, L4.data(), &dq)) != PW_OK) return st;
  out->sample_ms[1] = dt.walk_ms;
  out->sample_ms[2] = dq.walk_ms;
  // solve  T = P c + V w  for the two table runs (times in ns)
  const double T2 = 1e6 * dt.walk_ms, T3 = 1e6 * dq.walk_ms;
  const double P2 = (double)dt.n_probes, P3 = (double)dq.n_probes, V2 = (double)dt.n_visits, V3 = (double)dq.n_visits;
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
  const double Vs = (double)dv.n_visits, Ps = (double)dv.n_probes;
  out->sample_mode = Ps * g->table_probe_cost < Vs * g->table_visit_gain ? 2 : 1;
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
      KR[2 * i] = plans[(size_t)i].K;
      KR[2 * i + 1] = plans[(size_t)i].R;
    }
  for (int64_t i = 0; i < n_sel; ++i) {
    const int64_t qi = sel_query[i], k = sel_probe[i];
    if (qi < 0 || qi >= count || k < 0 || (uint64_t)k >= plans[(size_t)qi].K)
      return set_error(PW_ERR_ARG, "selection out of range");
    PW_CUDA_TRY(cudaMemcpyAsync(q_sel + i, (double*)g->ws.q.ptr + plans[(size_t)qi].probe_begin + k, sizeof(double),
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
// scratch (query plans, offsets, counters, the U_p and Q_R buffers) is carved
// out of the file-scope array below, so the call itself makes no cudaMalloc,
// cudaFree or allocating library call.  The array holds kNoAllocScratchBytes
// on every GPU that loads the library, until the process exits.  Every call
// shares it: calls that overlap on the GPU (different streams, or another
// thread) race on its contents; the counters that must start at zero are
// cleared by each call.
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
  const bool pilot = ba.mode == PW_BUDGET_PILOT;
  const size_t nq = (size_t)count;
  // fixed part of the layout: plans, pilot plans, offsets, totals, counters, pilot U
  size_t off = 0;
  const size_t o_plans = off;
  off = align256(off + sizeof(QPlan) * nq);
  const size_t o_pplans = off;
  off = align256(off + sizeof(QPlan) * nq);
  const size_t o_prefix = off;
  off = align256(off + sizeof(unsigned long long) * 4 * (nq + 1));
  const size_t o_totals = off;
  off = align256(off + sizeof(Totals) * 2);
  const size_t o_counters = off;
  off = align256(off + 64);
  const size_t o_pilot_u = off;
  off = align256(off + (pilot ? sizeof(float) * nq * (size_t)ba.K0 * (size_t)ba.R0 : 0));
  if (off > kNoAllocScratchBytes)
    return set_error(PW_ERR_NOMEM, "pw_query_batch_noalloc: batch needs more than the 64 MiB static scratch");
  QPlan* plans = (QPlan*)(base + o_plans);
  QPlan* pplans = (QPlan*)(base + o_pplans);
  unsigned long long* prefix = (unsigned long long*)(base + o_prefix);
  unsigned long long* pprefix = prefix + 2 * (nq + 1);
  Totals* totals = (Totals*)(base + o_totals);
  unsigned long long* counters = (unsigned long long*)(base + o_counters);
  float* pilot_u = (float*)(base + o_pilot_u);
  PW_CUDA_TRY(cudaStreamWaitEvent(stream, g->ws.last_use, 0));
  PW_CUDA_TRY(cudaMemsetAsync(counters, 0, 64, stream));
  const int qthreads = 128;
  const int qblocks = (int)((count + qthreads - 1) / qthreads);
  budget_init_kernel<<<qblocks, qthreads, 0, stream>>>(count, d_s, d_t, d_eps, d_L, d_seeds, ba, g->n, g->d_node,
                                                       plans, pilot ? pplans : nullptr);
  count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  WalkArgs wa;
  wa.rec = g->d_rec;
  wa.node = g->d_node;
  wa.nq = count;
  wa.n = (uint32_t)g->n;
  wa.visits = nullptr;
  if (pilot) {
    scan_kernel<<<1, 1024, 0, stream>>>(pplans, count, pprefix, totals + 1);
    count_launch();
    wa.plans = pplans;
    wa.tile_prefix = pprefix;
    wa.totals = totals + 1;
    wa.tile_counter = counters + 1;
    wa.u = pilot_u;
    wa.walk_tag = kTagWalkPilot;
    wa.probe_tag = kTagProbePilot;
    if ((st = launch_walk(g, stream, false, wa)) != PW_OK) return st;
    pilot_budget_kernel<<<qblocks, qthreads, 0, stream>>>(count, plans, pplans, pilot_u, ba, g->d_node);
    count_launch();
    PW_CUDA_TRY(cudaGetLastError());
  }
  scan_kernel<<<1, 1024, 0, stream>>>(plans, count, prefix, totals);
  count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  PW_CUDA_TRY(cudaMemcpyAsync(g->ws.host_totals, totals, sizeof(Totals), cudaMemcpyDeviceToHost, stream));
  PW_CUDA_TRY(cudaStreamSynchronize(stream));
  const Totals T = *g->ws.host_totals;
  const size_t o_u = off;
  off = align256(off + sizeof(float) * (size_t)T.u_slots);
  const size_t o_q = off;
  off = align256(off + sizeof(double) * (size_t)T.probes);
  if (off > kNoAllocScratchBytes)
    return set_error(PW_ERR_NOMEM, "pw_query_batch_noalloc: the walks of this batch need more than the 64 MiB "
                                   "static scratch (U_p and Q_R buffers); split the batch");
  float* u = (float*)(base + o_u);
  double* qbuf = (double*)(base + o_q);
  const int mode = pick_walk_mode(g, params, T);
  g->last_walk_mode = mode;
  wa.plans = plans;
  wa.tile_prefix = prefix;
  wa.totals = totals;
  wa.tile_counter = counters;
  wa.u = u;
  wa.walk_tag = kTagWalk;
  wa.probe_tag = kTagProbe;
  if (T.tiles > 0) {
    st = mode == 2 ? launch_walk_table(g, stream, false, wa, prefix + nq + 1, counters + 2)
                   : launch_walk(g, stream, false, wa);
    if (st != PW_OK) return st;
  }
  if (T.probes > 0) {
    const int fthreads = 128;
    const unsigned long long want = (T.probes + fthreads - 1) / fthreads;
    const int fblocks = (int)std::min<unsigned long long>(want, (unsigned long long)g->sm_count * 64);
    probe_finish_kernel<<<fblocks, fthreads, 0, stream>>>(plans, count, prefix + nq + 1, totals, u, qbuf);
    count_launch();
    PW_CUDA_TRY(cudaGetLastError());
  }
  mom_kernel<<<(unsigned)count, 128, 0, stream>>>(plans, qbuf, d_beta_hat, d_status);
  count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  PW_CUDA_TRY(cudaEventRecord(g->ws.last_use, stream));
  return PW_OK;
}
