// Continuous-batching server: one persistent kernel fed by a device work queue.
//
// Work unit = one probe job (query slot, stage, probes k .. k + count - 1): a
// block runs all R replicas of its probes (its warps take 32-replica tiles),
// adds each tile's exact replica sums into the block's digits of that probe
// (pw_exact.cuh), and writes Q_R of each probe (Eq. Q-Ustat) or, in the pilot
// stage, the probe's (S1, S2).  The block that completes the last pilot
// probe of a query computes R (Lemma 3.7 condition) and publishes the query's
// main stage; the block that completes the last main probe takes the median of
// the block means (Eq. final-estimator) and writes the result to host-mapped
// memory.  New queries enter through a ring written by the host (copy engine,
// no kernel launch); main stages through a ring written by the device.
//
// The host scheduler thread admits queued requests while their accumulator
// memory (8 bytes per probe + 16 per pilot probe) fits, relaunches the kernel
// when it has exited after an idle period, and collects completions.  Every
// device wait is bounded (iteration cap and %globaltimer deadline); a kernel
// with nothing to do exits instead of spinning.
#include <math.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "pw_budget.cuh"
#include "pw_device.cuh"
#include "pw_exact.cuh"
#include "pw_internal.h"
#include "pw_walk.cuh"

namespace pw {

constexpr uint32_t kStagePilot = 0, kStageMain = 1;
constexpr int kServerThreads = 256;
constexpr uint32_t kServerGmax = 2048;  // block means of the final job live in shared memory
constexpr size_t kServerMeansBytes = sizeof(double) * kServerGmax;
constexpr uint32_t kJobProbes = 8;      // at most 8 probes per job

struct SlotDev {
  QPlan plan;          // main plan; R written by the pilot transition in PILOT mode
  uint64_t ticket;
  uint32_t K[2];       // probes per stage
  uint32_t R0;         // pilot replicas per probe
  uint32_t use_table;  // main-stage walks read a per-probe table of z
  uint32_t next[2];    // claim cursors
  uint32_t done[2];    // completed probes
  double* q;           // K values of Q_R (main stage)
  double* ps;          // K0 pairs (S1, S2) of the pilot
};

struct Completion {
  unsigned long long ticket;
  double beta;
  int32_t status;
  int32_t pad;
};

struct ServerArgs {
  const int4* rec;     // fused records (layout 1)
  const int32_t* col;  // col_idx (layout 2)
  const int4* node;
  uint32_t n;
  uint32_t table_words;  // 0: graph too large for a shared-memory table
  SlotDev* slots;
  unsigned long long* heads;  // [2]: host ring, device ring
  unsigned long long* dtail;  // producer position of the device ring
  uint32_t* ring_slot;        // [2][cap]
  uint32_t* ring_stage;       // [2][cap]
  unsigned long long* ring_seq;  // [2][cap]: entry i is valid when seq == its position
  uint32_t cap;
  Completion* comp;  // host-mapped
  const uint32_t* stop;
  unsigned long long* last_claim;  // %globaltimer of the latest job claim by any block
  uint32_t* exit_flag;             // set once the whole grid has been idle for idle_ns
  unsigned long long idle_ns;
  const double* model;  // device: walk-mode cost model {table cost per probe, saving per visit}
  BudgetArgs A;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <class T>
__device__ __forceinline__ T ld_volatile(const T* p) {
  return *(const volatile T*)p;
}

// Slot memory is reused by successive queries: read it through L2, not L1.
__device__ __forceinline__ QPlan load_plan(const QPlan* p) {
  QPlan P;
  const unsigned long long* src = (const unsigned long long*)p;
  unsigned long long* dst = (unsigned long long*)&P;
#pragma unroll
  for (int i = 0; i < (int)(sizeof(QPlan) / 8); ++i) dst[i] = __ldcg(src + i);
  return P;
}

// Claim the next probe job; false when the stop flag or the grid-wide exit
// flag is set.  The exit flag is raised when no block has claimed a job for
// idle_ns, so the grid leaves together and the host relaunches all of it when
// work returns (blocks never leave one by one while others keep working).
// Device-ring (main stage) work is taken first.
// Probes per job: one when the main stage reads a per-probe table (a block
// builds one table at a time), else enough probes for about 8 tiles of 32
// replicas, so every warp of the block has work when R is small.
__device__ __forceinline__ uint32_t probes_per_job(const SlotDev* S, uint32_t stage) {
  const uint32_t R = stage == kStagePilot ? __ldcg(&S->R0) : __ldcg(&S->plan.R);
  if (stage == kStageMain && __ldcg(&S->use_table)) return 1u;
  const uint32_t chunks = (R + 31u) / 32u;
  return chunks >= 8u ? 1u : 8u / chunks;
}

__device__ bool find_job(const ServerArgs& A, uint32_t& slot, uint32_t& stage, uint32_t& k, uint32_t& count) {
  for (uint32_t it = 0; it < (1u << 28); ++it) {
    if (ld_volatile(A.exit_flag) || ld_volatile(A.stop)) return false;
    bool retry = false;
    for (int r = 1; r >= 0 && !retry; --r) {
      const unsigned long long h = ld_volatile(A.heads + r);
      const uint32_t idx = (uint32_t)(h % A.cap) + (uint32_t)r * A.cap;
      if (ld_volatile(A.ring_seq + idx) != h) continue;
      const uint32_t sl = ld_volatile(A.ring_slot + idx);
      const uint32_t sg = ld_volatile(A.ring_stage + idx);
      SlotDev* S = A.slots + sl;
      const uint32_t K = __ldcg(&S->K[sg]);
      const uint32_t want = probes_per_job(S, sg);
      const uint32_t kk = atomicAdd(&S->next[sg], want);
      if (kk < K) {
        slot = sl;
        stage = sg;
        k = kk;
        count = (K - kk < want) ? K - kk : want;
        atomicMax(A.last_claim, global_ns());
        return true;
      }
      atomicCAS(A.heads + r, h, h + 1);  // this entry is exhausted
      retry = true;
    }
    if (retry) continue;
    const unsigned long long now = global_ns(), last = ld_volatile(A.last_claim);
    if (now > last && now - last > A.idle_ns) {
      atomicExch(A.exit_flag, 1u);
      return false;
    }
    __nanosleep(256);
  }
  atomicExch(A.exit_flag, 1u);
  return false;
}

// One per-visit replica (probe entries by Feistel at each visit), compiled as a
// separate function.  Inlined into the job loop below, the same code ran about
// 20x slower per walk step on a 4M-node grid (identical results); behind a call
// boundary it runs at walk_kernel's speed.
template <class GR>
__device__ __noinline__ float server_walk_visit(const GR gr, uint32_t n, uint32_t walk_tag, uint32_t probe_tag,
                                                int32_t s, int32_t t, int32_t L, uint64_t seed, uint32_t k,
                                                uint64_t pair) {
  const Probe pr = make_probe(n, seed, k, probe_tag);
  const ZOnTheFly zp{pr};
  return walk_pair<false>(gr, nullptr, walk_tag, zp, s, t, L, seed, pair);
}

// TABLE: the graph's probe table fits in shared memory, so main-stage jobs may
// use it (4 blocks/SM); without it only per-visit jobs exist and MINB is the
// occupancy the registers are capped for: 2 blocks/SM (the registers the
// per-visit path asks for) or 3 (fewer registers, some spilled), whichever
// pw_server_tune finds faster on the graph.
// The graph access of the server: fused records, or col_idx plus node records.
template <class GR>
__device__ __forceinline__ GR server_graph(const ServerArgs& A);
template <>
__device__ __forceinline__ FusedRecords server_graph<FusedRecords>(const ServerArgs& A) {
  return FusedRecords{A.rec, A.node};
}
template <>
__device__ __forceinline__ SplitRecords server_graph<SplitRecords>(const ServerArgs& A) {
  return SplitRecords{A.col, A.node};
}

template <bool TABLE, class GR, int MINB>
__global__ void __launch_bounds__(kServerThreads, MINB) server_kernel(ServerArgs A) {
  const GR gr = server_graph<GR>(A);
  extern __shared__ uint32_t smem[];
  uint32_t* tab = smem;
  double* means = (double*)(smem + A.table_words);  // table_words is a multiple of 4
  __shared__ unsigned long long j_sum[kJobProbes][kSumDigits];
  __shared__ uint32_t j_slot, j_stage, j_k, j_count, j_valid, j_last, j_tile;
  const uint32_t lane = threadIdx.x & 31u;
  if (threadIdx.x == 0) atomicMax(A.last_claim, global_ns());  // a fresh launch starts its idle clock
  for (;;) {
    if (threadIdx.x == 0) {
      uint32_t sl = 0, sg = 0, kk = 0, cnt = 0;
      j_valid = find_job(A, sl, sg, kk, cnt) ? 1u : 0u;
      j_slot = sl;
      j_stage = sg;
      j_k = kk;
      j_count = cnt;
      j_tile = 0;
      j_last = 0;
    }
    if (threadIdx.x < kJobProbes * kSumDigits) (&j_sum[0][0])[threadIdx.x] = 0ull;
    __syncthreads();
    if (!j_valid) return;
    const uint32_t slot = j_slot, stage = j_stage, k0 = j_k, nprobe = j_count;
    SlotDev* S = A.slots + slot;
    const QPlan P = load_plan(&S->plan);
    const bool pilot = stage == kStagePilot;
    const uint32_t R = pilot ? __ldcg(&S->R0) : P.R;
    const uint32_t walk_tag = pilot ? kTagWalkPilot : kTagWalk;
    const uint32_t probe_tag = pilot ? kTagProbePilot : kTagProbe;
    const bool table = TABLE && !pilot && __ldcg(&S->use_table) != 0u;  // then nprobe == 1
    const uint32_t chunks = (R + 31u) / 32u;
    if (TABLE && table) build_probe_table(make_probe(A.n, P.seed, k0, probe_tag), tab, A.n);
    __syncthreads();
    // tiles of 32 replicas over the job's probes; each tile's exact sums go
    // into the digits of its probe j (any order gives the same digits)
    for (;;) {
      uint32_t c = 0;
      if (lane == 0) c = atomicAdd(&j_tile, 1u);
      c = __shfl_sync(0xffffffffu, c, 0);
      if (c >= chunks * nprobe) break;
      const uint32_t j = c / chunks, p = (c - j * chunks) * 32u + lane;
      const uint32_t k = k0 + j;
      SumDigits sum;
      sum_clear(sum);
      if (p < R) {
        const uint64_t pair = (uint64_t)k * R + p;
        float U;
        if (TABLE && table) {
          const ZTable zp = table_reader(tab, A.n);
          U = walk_pair_table<false>(gr, nullptr, walk_tag, zp, P.s, P.t, P.L, P.seed, pair);
        } else {
          U = server_walk_visit<GR>(gr, A.n, walk_tag, probe_tag, P.s, P.t, P.L, P.seed, k, pair);
        }
        sum_add(sum, U);
      }
      sum_warp_reduce(sum);
      if (lane == 0) {
#pragma unroll
        for (int d = 0; d < kSumDigits; ++d)
          if (sum.d[d] != 0) atomicAdd(&j_sum[j][d], (unsigned long long)sum.d[d]);
      }
    }
    __syncthreads();
    if (threadIdx.x < nprobe) {  // one thread per probe: S1, S2 rounded from the exact digits
      const uint32_t j = threadIdx.x, k = k0 + j;
      long long dj[kSumDigits];
#pragma unroll
      for (int d = 0; d < kSumDigits; ++d) dj[d] = (long long)j_sum[j][d];
      double S1, S2;
      sum_round(dj, S1, S2);
      if (pilot) {
        __stcg(S->ps + 2 * k, S1);
        __stcg(S->ps + 2 * k + 1, S2);
      } else {
        __stcg(S->q + k, u_statistic(S1, S2, R));
      }
      __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t old = atomicAdd(&S->done[stage], nprobe);
      j_last = (old + nprobe == __ldcg(&S->K[stage])) ? 1u : 0u;
      if (j_last) __threadfence();
    }
    __syncthreads();
    if (j_last) {
      if (pilot) {
        if (threadIdx.x == 0) {
          const uint32_t K0 = __ldcg(&S->K[kStagePilot]);
          double sum_var = 0.0, sum_q = 0.0;
          for (uint32_t kk = 0; kk < K0; ++kk)
            pilot_accumulate(sum_var, sum_q, __ldcg(S->ps + 2 * kk), __ldcg(S->ps + 2 * kk + 1), R);
          QPlan M = P;
          pilot_finish(M, sum_var, sum_q, K0, __ldg(&A.node[P.s].z), __ldg(&A.node[P.t].z), A.A);
          __stcg(&S->plan.R, M.R);
          __stcg(&S->plan.chunks, M.chunks);
          __stcg(&S->plan.sigma2, M.sigma2);
          __stcg(&S->plan.qbar, M.qbar);
          __stcg(&S->plan.theta, M.theta);
          // table when building z^(k) is cheaper than evaluating it at every
          // visit, by the graph's walk-mode cost model
          const double visits = 2.0 * (double)M.R * (double)(P.L + 1);
          const double probe_cost = __ldcg(A.model), visit_gain = __ldcg(A.model + 1);
          __stcg(&S->use_table, (A.table_words > 0 && probe_cost < visit_gain * visits) ? 1u : 0u);
          __threadfence();
          const unsigned long long pos = atomicAdd(A.dtail, 1ull);
          const uint32_t idx = (uint32_t)(pos % A.cap) + A.cap;
          A.ring_slot[idx] = slot;
          A.ring_stage[idx] = kStageMain;
          __threadfence();
          *(volatile unsigned long long*)(A.ring_seq + idx) = pos;
        }
      } else {
        const uint32_t G = P.G, B = P.B;
        for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) {
          double sum = 0.0;
          for (uint32_t kk = 0; kk < B; ++kk) sum = __dadd_rn(sum, __ldcg(S->q + (uint64_t)g * B + kk));
          means[g] = __ddiv_rn(sum, (double)B);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          for (uint32_t i = 1; i < G; ++i) {
            const double v = means[i];
            uint32_t j = i;
            while (j > 0 && means[j - 1] > v) {
              means[j] = means[j - 1];
              --j;
            }
            means[j] = v;
          }
          const double med = (G & 1u) ? means[G / 2] : __ddiv_rn(__dadd_rn(means[G / 2 - 1], means[G / 2]), 2.0);
          Completion* c = A.comp + slot;
          c->beta = med;
          c->status = PW_OK;
          __threadfence_system();
          *(volatile unsigned long long*)&c->ticket = __ldcg(&S->ticket);
          __threadfence_system();
        }
      }
    }
    __syncthreads();
  }
}

using ServerFn = void (*)(ServerArgs);
// minb: 2 or 3 blocks/SM for the per-visit-only kernel (the table kernel is 4)
static ServerFn server_fn(bool table, int layout, int minb) {
  if (layout == 2) {
    if (table) return server_kernel<true, SplitRecords, 4>;
    return minb == 3 ? server_kernel<false, SplitRecords, 3> : server_kernel<false, SplitRecords, 2>;
  }
  if (table) return server_kernel<true, FusedRecords, 4>;
  return minb == 3 ? server_kernel<false, FusedRecords, 3> : server_kernel<false, FusedRecords, 2>;
}

struct Request {
  uint64_t ticket;
  int64_t s, t;
  double eps;
  int32_t L;
  uint64_t seed;
  double t_submit_ms;
};

struct Result {
  double beta;
  int32_t status;
  double latency_ms;  // submit to completion seen by the scheduler
};

static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace pw

struct pw_server {
  pw_graph* g = nullptr;
  pw::BudgetArgs ba{};
  uint32_t S = 0, cap = 0;
  pw::SlotDev* d_slots = nullptr;
  pw::SlotDev* h_slot_stage = nullptr;  // pinned staging, one per slot
  unsigned long long* d_ctl = nullptr;  // heads[2], dtail, pad
  uint32_t* d_ring_slot = nullptr;
  uint32_t* d_ring_stage = nullptr;
  unsigned long long* d_ring_seq = nullptr;
  uint32_t* h_ring_stage_buf = nullptr;          // pinned: cap x {slot, stage}
  unsigned long long* h_ring_seq_buf = nullptr;  // pinned: cap
  pw::Completion* h_comp = nullptr;  // mapped pinned
  pw::Completion* d_comp = nullptr;
  uint32_t* d_stop = nullptr;
  uint32_t* h_stop = nullptr;  // pinned
  char* d_pool = nullptr;
  size_t pool_bytes = 0;
  std::map<size_t, size_t> free_ranges;
  std::vector<uint64_t> slot_ticket;
  std::vector<std::pair<size_t, size_t>> slot_range;
  std::vector<uint32_t> free_slots;
  uint64_t host_tail = 0;
  cudaStream_t kstream = nullptr, cstream = nullptr;
  size_t smem = 0;
  int minb = 2;      // occupancy variant of the per-visit-only kernel (server_fn)
  int grid = 0;      // blocks of the persistent kernel: SMs x resident blocks of that variant
  int grids[2] = {0, 0};  // per-visit-only kernel: grid at minb 2, 3
  double table_probe_cost = 0.0, table_visit_gain = 0.0;  // walk-mode cost model (host copy of d_model)
  double* d_model = nullptr;
  bool kernel_live = false;
  uint32_t active = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<pw::Request> pending;
  std::unordered_map<uint64_t, pw::Result> results;    // finished, not yet delivered
  std::unordered_set<uint64_t> unfinished;              // submitted, no result yet
  std::vector<double> slot_submit_ms;
  uint64_t next_ticket = 1, submitted = 0, completed = 0;
  bool stopping = false;
  pw_status fatal = PW_OK;
  std::string fatal_msg;
};

namespace pw {

static bool pool_alloc(pw_server* sv, size_t bytes, size_t* off) {
  bytes = (bytes + 255) & ~(size_t)255;
  for (auto it = sv->free_ranges.begin(); it != sv->free_ranges.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes, roff = it->first + bytes;
      sv->free_ranges.erase(it);
      if (rest) sv->free_ranges[roff] = rest;
      return true;
    }
  }
  return false;
}

static void pool_free(pw_server* sv, size_t off, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  auto it = sv->free_ranges.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != sv->free_ranges.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    sv->free_ranges.erase(nx);
  }
  if (it != sv->free_ranges.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      sv->free_ranges.erase(it);
    }
  }
}

static ServerArgs server_args(pw_server* sv) {
  ServerArgs a;
  a.rec = sv->g->d_rec;
  a.col = sv->g->d_col;
  a.node = sv->g->d_node;
  a.n = (uint32_t)sv->g->n;
  a.table_words = (uint32_t)((sv->smem - kServerMeansBytes) / sizeof(uint32_t));
  a.slots = sv->d_slots;
  a.heads = sv->d_ctl;
  a.dtail = sv->d_ctl + 2;
  a.last_claim = sv->d_ctl + 3;
  a.exit_flag = (uint32_t*)(sv->d_ctl + 4);
  a.ring_slot = sv->d_ring_slot;
  a.ring_stage = sv->d_ring_stage;
  a.ring_seq = sv->d_ring_seq;
  a.cap = sv->cap;
  a.comp = sv->d_comp;
  a.stop = sv->d_stop;
  a.idle_ns = 5ull * 1000 * 1000;
  a.model = sv->d_model;
  a.A = sv->ba;
  return a;
}

// Admit one request: plan on the host, reserve accumulator memory, write the
// slot and a host-ring entry with the copy engine.  Returns false when no slot
// or memory is free (the request stays queued).
static bool admit(pw_server* sv, const Request& rq) {
  pw_graph* g = sv->g;
  const bool ok_ids = rq.s >= 0 && rq.s < g->n && rq.t >= 0 && rq.t < g->n;
  QPlan P, PP;
  plan_query(rq.s, rq.t, rq.eps, rq.L, rq.seed, g->n, ok_ids ? g->deg[(size_t)rq.s] : 1,
             ok_ids ? g->deg[(size_t)rq.t] : 1, sv->ba, &P, &PP);
  if (P.status == PW_OK && P.G > kServerGmax) P.status = PW_ERR_ARG;
  if (P.status != PW_OK || P.K == 0) {  // invalid, or s == t: answered on the host
    sv->results[rq.ticket] = {P.status == PW_OK ? 0.0 : NAN, P.status, now_ms() - rq.t_submit_ms};
    sv->unfinished.erase(rq.ticket);
    sv->completed++;
    return true;
  }
  if (sv->free_slots.empty()) return false;
  const bool pilot = sv->ba.mode == PW_BUDGET_PILOT;
  const size_t bytes = sizeof(double) * (size_t)P.K + (pilot ? 2 * sizeof(double) * (size_t)PP.K : 0) + 256;
  if (((bytes + 255) & ~(size_t)255) > sv->pool_bytes) {  // could never be admitted: fail it now
    sv->results[rq.ticket] = {NAN, PW_ERR_NOMEM, now_ms() - rq.t_submit_ms};
    sv->unfinished.erase(rq.ticket);
    sv->completed++;
    return true;
  }
  size_t off = 0;
  if (!pool_alloc(sv, bytes, &off)) return false;
  const uint32_t slot = sv->free_slots.back();
  sv->free_slots.pop_back();
  sv->slot_ticket[slot] = rq.ticket;
  sv->slot_range[slot] = {off, bytes};
  sv->slot_submit_ms[slot] = rq.t_submit_ms;
  SlotDev& h = sv->h_slot_stage[slot];
  memset(&h, 0, sizeof h);
  h.plan = P;
  h.ticket = rq.ticket;
  h.K[kStagePilot] = pilot ? PP.K : 0;
  h.K[kStageMain] = P.K;
  h.R0 = pilot ? PP.R : 0;
  h.q = (double*)(sv->d_pool + off);
  h.ps = (double*)(sv->d_pool + off + sizeof(double) * (size_t)P.K);
  if (!pilot) {
    const double visits = 2.0 * (double)P.R * (double)(P.L + 1);
    const uint32_t words = (uint32_t)((sv->smem - kServerMeansBytes) / sizeof(uint32_t));
    h.use_table = (words > 0 && sv->table_probe_cost < sv->table_visit_gain * visits) ? 1u : 0u;
  }
  sv->h_comp[slot].ticket = 0;
  cudaMemcpyAsync(sv->d_slots + slot, &h, sizeof(SlotDev), cudaMemcpyHostToDevice, sv->cstream);
  const uint64_t pos = sv->host_tail++;
  const uint32_t idx = (uint32_t)(pos % sv->cap);
  sv->h_ring_stage_buf[2 * idx] = slot;
  sv->h_ring_stage_buf[2 * idx + 1] = pilot ? kStagePilot : kStageMain;
  sv->h_ring_seq_buf[idx] = pos;
  cudaMemcpyAsync(sv->d_ring_slot + idx, &sv->h_ring_stage_buf[2 * idx], sizeof(uint32_t), cudaMemcpyHostToDevice,
                  sv->cstream);
  cudaMemcpyAsync(sv->d_ring_stage + idx, &sv->h_ring_stage_buf[2 * idx + 1], sizeof(uint32_t),
                  cudaMemcpyHostToDevice, sv->cstream);
  cudaMemcpyAsync(sv->d_ring_seq + idx, &sv->h_ring_seq_buf[idx], sizeof(unsigned long long), cudaMemcpyHostToDevice,
                  sv->cstream);
  sv->active++;
  return true;
}

static void collect(pw_server* sv) {
  for (uint32_t s = 0; s < sv->S; ++s) {
    const uint64_t want = sv->slot_ticket[s];
    if (!want) continue;
    const volatile pw::Completion* c = sv->h_comp + s;
    if (c->ticket != want) continue;
    std::atomic_thread_fence(std::memory_order_acquire);
    sv->results[want] = {c->beta, c->status, now_ms() - sv->slot_submit_ms[s]};
    sv->unfinished.erase(want);
    sv->completed++;
    pool_free(sv, sv->slot_range[s].first, sv->slot_range[s].second);
    sv->slot_ticket[s] = 0;
    sv->free_slots.push_back(s);
    sv->active--;
  }
}

static void worker_loop(pw_server* sv) {
  cudaSetDevice(sv->g->device);
  const ServerArgs args = server_args(sv);
  for (;;) {
    bool idle = true;
    int minb = 2, grid = 0;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      minb = sv->minb;
      grid = sv->grid;
      const uint32_t before = sv->active;
      collect(sv);
      if (sv->active != before) idle = false;
      while (!sv->pending.empty() && !sv->stopping) {
        if (!admit(sv, sv->pending.front())) break;
        sv->pending.pop_front();
        idle = false;
      }
      if (sv->stopping && sv->active == 0) break;
      if (!idle) sv->cv.notify_all();
    }
    if (sv->active > 0) {
      if (sv->kernel_live && cudaStreamQuery(sv->kstream) == cudaSuccess) sv->kernel_live = false;
      if (!sv->kernel_live) {
        // the host-ring copies of newly admitted work are ordered before the launch
        cudaEvent_t ev;
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        cudaEventRecord(ev, sv->cstream);
        cudaStreamWaitEvent(sv->kstream, ev, 0);
        cudaEventDestroy(ev);
        cudaMemsetAsync(sv->d_ctl + 4, 0, sizeof(unsigned long long), sv->kstream);  // exit flag
        const ServerFn fn = server_fn(args.table_words > 0, sv->g->layout, minb);
        const cudaError_t e = launch_with_window(sv->g, fn, grid, kServerThreads, sv->smem, sv->kstream, args);
        count_launch();
        if (e != cudaSuccess) {
          std::lock_guard<std::mutex> lk(sv->mu);
          sv->fatal = cuda_error(e, "server_kernel launch");
          sv->fatal_msg = pw_last_error();
          sv->stopping = true;
        }
        sv->kernel_live = true;
      }
    } else if (sv->kernel_live && cudaStreamQuery(sv->kstream) == cudaSuccess) {
      sv->kernel_live = false;
    }
    if (idle) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->cv.notify_all();
}

}  // namespace pw

using namespace pw;

extern "C" {

pw_status pw_server_create(pw_graph* g, const pw_params* params, size_t accum_bytes, pw_server** out) {
  if (!g || !out) return set_error(PW_ERR_ARG, "NULL argument");
  *out = nullptr;
  BudgetArgs ba;
  pw_status st = resolve_budget(params, g, &ba, nullptr);
  if (st != PW_OK) return st;
  if (ba.G > kServerGmax) return set_error(PW_ERR_ARG, "server supports G <= 2048");
  if (ba.mode == PW_BUDGET_ADAPTIVE) return set_error(PW_ERR_ARG, "servers run budgets fixed at admission (not ADAPTIVE)");
  if (accum_bytes < ((size_t)1 << 20)) accum_bytes = (size_t)1 << 20;
  PW_CUDA_TRY(cudaSetDevice(g->device));
  pw_server* sv = new pw_server();
  sv->g = g;
  sv->ba = ba;
  // The default walk-mode model (n Feistel passes per table against 2.5 per
  // visit), not the graph's autotuned costs: those are fitted on the batch
  // kernels, whose per-visit path is faster than the server's (the server's
  // runs inside the table-capable kernel at its register cap).
  // pw_server_tune picks the server's own policy by timing it.
  sv->table_probe_cost = (double)g->n;
  sv->table_visit_gain = 2.5;
  sv->S = 4096;
  sv->cap = 4096;
  sv->pool_bytes = accum_bytes;
  auto fail = [&](pw_status s2) {
    pw_server_destroy(sv);
    return s2;
  };
  cudaError_t e = cudaSuccess;
  const size_t ring = (size_t)2 * sv->cap;
  if ((e = cudaMalloc(&sv->d_slots, sizeof(SlotDev) * sv->S)) != cudaSuccess ||
      (e = cudaMalloc(&sv->d_ctl, sizeof(unsigned long long) * 8)) != cudaSuccess ||
      (e = cudaMalloc(&sv->d_ring_slot, sizeof(uint32_t) * ring)) != cudaSuccess ||
      (e = cudaMalloc(&sv->d_ring_stage, sizeof(uint32_t) * ring)) != cudaSuccess ||
      (e = cudaMalloc(&sv->d_ring_seq, sizeof(unsigned long long) * ring)) != cudaSuccess ||
      (e = cudaMalloc(&sv->d_stop, sizeof(uint32_t))) != cudaSuccess ||
      (e = cudaMalloc(&sv->d_model, 2 * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&sv->d_pool, accum_bytes)) != cudaSuccess ||
      (e = cudaMallocHost(&sv->h_slot_stage, sizeof(SlotDev) * sv->S)) != cudaSuccess ||
      (e = cudaMallocHost(&sv->h_ring_stage_buf, sizeof(uint32_t) * 2 * sv->cap)) != cudaSuccess ||
      (e = cudaMallocHost(&sv->h_ring_seq_buf, sizeof(unsigned long long) * sv->cap)) != cudaSuccess ||
      (e = cudaMallocHost(&sv->h_stop, sizeof(uint32_t))) != cudaSuccess ||
      (e = cudaHostAlloc(&sv->h_comp, sizeof(Completion) * sv->S, cudaHostAllocMapped)) != cudaSuccess ||
      (e = cudaHostGetDevicePointer(&sv->d_comp, sv->h_comp, 0)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&sv->kstream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&sv->cstream, cudaStreamNonBlocking)) != cudaSuccess)
    return fail(cuda_error(e, "server allocation"));
  memset(sv->h_comp, 0, sizeof(Completion) * sv->S);
  const double model[2] = {sv->table_probe_cost, sv->table_visit_gain};
  if ((e = cudaMemcpy(sv->d_model, model, sizeof model, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(sv->d_slots, 0, sizeof(SlotDev) * sv->S)) != cudaSuccess ||
      (e = cudaMemset(sv->d_ctl, 0, sizeof(unsigned long long) * 8)) != cudaSuccess ||
      (e = cudaMemset(sv->d_ring_seq, 0xFF, sizeof(unsigned long long) * ring)) != cudaSuccess ||
      (e = cudaMemset(sv->d_stop, 0, sizeof(uint32_t))) != cudaSuccess)
    return fail(cuda_error(e, "server initialisation"));
  sv->free_ranges[0] = accum_bytes;
  sv->slot_ticket.assign(sv->S, 0);
  sv->slot_range.assign(sv->S, {0, 0});
  sv->slot_submit_ms.assign(sv->S, 0.0);
  for (uint32_t s = 0; s < sv->S; ++s) sv->free_slots.push_back(sv->S - 1 - s);
  // shared memory: probe table (if it fits next to the block means) + block means
  const size_t ubytes = kServerMeansBytes;
  // rounded to 16 bytes so the FP64 block means that follow stay aligned
  const size_t tbytes = (sizeof(uint32_t) * (size_t)table_words((uint32_t)g->n) + 15) & ~(size_t)15;
  sv->smem = ubytes + ((tbytes + ubytes <= 200 * 1024) ? tbytes : 0);
  const bool with_table = sv->smem > ubytes;
  for (int v = 0; v < (with_table ? 1 : 2); ++v) {
    const ServerFn fn = server_fn(with_table, g->layout, 2 + v);
    if ((e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sv->smem)) !=
        cudaSuccess)
      return fail(cuda_error(e, "server smem attribute"));
    int nb = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)fn, kServerThreads, sv->smem)) !=
        cudaSuccess)
      return fail(cuda_error(e, "server occupancy"));
    sv->grids[v] = g->sm_count * (nb > 0 ? nb : 1);
  }
  sv->minb = 2;
  sv->grid = sv->grids[0];
  cudaDeviceSynchronize();
  sv->worker = std::thread(worker_loop, sv);
  *out = sv;
  return PW_OK;
}

pw_status pw_server_submit(pw_server* sv, int64_t s, int64_t t, double eps, int32_t L, const uint64_t* seed,
                           uint64_t* ticket) {
  if (!sv || !ticket) return set_error(PW_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->fatal != PW_OK) return set_error(sv->fatal, sv->fatal_msg);
  if (sv->stopping) return set_error(PW_ERR_CANCELLED, "server is shutting down");
  if (sv->pending.size() >= (size_t)1 << 24) return set_error(PW_ERR_FULL, "server queue full");
  Request rq;
  rq.ticket = sv->next_ticket++;
  rq.s = s;
  rq.t = t;
  rq.eps = eps;
  rq.L = L;
  rq.seed = seed ? *seed : default_seed(sv->ba.global_seed, s, t, eps, L);
  rq.t_submit_ms = now_ms();
  sv->pending.push_back(rq);
  sv->unfinished.insert(rq.ticket);
  sv->submitted++;
  *ticket = rq.ticket;
  return PW_OK;
}

pw_status pw_server_poll(pw_server* sv, uint64_t ticket, double* beta_hat) {
  if (!sv || !beta_hat) return set_error(PW_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->results.find(ticket);
  if (it == sv->results.end()) {
    if (!sv->unfinished.count(ticket)) return set_error(PW_ERR_ARG, "unknown or already delivered ticket");
    if (sv->fatal != PW_OK) return set_error(sv->fatal, sv->fatal_msg);
    return PW_PENDING;
  }
  *beta_hat = it->second.beta;
  const int32_t st = it->second.status;
  sv->results.erase(it);
  if (st != PW_OK) return set_error((pw_status)st, "query rejected");
  return PW_OK;
}

pw_status pw_server_collect(pw_server* sv, int64_t cap, uint64_t* tickets, double* beta_hat, int32_t* status,
                            double* latency_ms, int64_t* count) {
  if (!sv || !count || (cap > 0 && (!tickets || !beta_hat || !status))) return set_error(PW_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  int64_t n = 0;
  for (auto it = sv->results.begin(); it != sv->results.end() && n < cap;) {
    tickets[n] = it->first;
    beta_hat[n] = it->second.beta;
    status[n] = it->second.status;
    if (latency_ms) latency_ms[n] = it->second.latency_ms;
    ++n;
    it = sv->results.erase(it);
  }
  *count = n;
  return PW_OK;
}

pw_status pw_server_drain(pw_server* sv, int64_t timeout_ms) {
  if (!sv) return set_error(PW_ERR_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(sv->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  while (sv->completed < sv->submitted && sv->fatal == PW_OK) {
    if (sv->cv.wait_until(lk, deadline) == std::cv_status::timeout && sv->completed < sv->submitted)
      return set_error(PW_ERR_TIMEOUT, "server drain timed out");
  }
  if (sv->fatal != PW_OK) return set_error(sv->fatal, sv->fatal_msg);
  return PW_OK;
}

pw_status pw_server_tune(pw_server* sv, int64_t count, const int64_t* s, const int64_t* t, const double* eps,
                         const int32_t* L, const uint64_t* seeds, pw_server_tune_result* out) {
  if (!sv || !out || !s || !t || !eps || !L || count <= 0) return set_error(PW_ERR_ARG, "NULL argument or empty sample");
  memset(out, 0, sizeof *out);
  pw_graph* g = sv->g;
  const bool table = sv->smem > kServerMeansBytes;
  std::vector<uint64_t> tk((size_t)count);
  std::vector<double> ref, got((size_t)count);
  // the sample as a burst, once to warm up and once timed: queries/s; the
  // estimates must equal those of the first case timed, bit for bit
  auto burst = [&](double* qps) -> pw_status {
    double secs = 0.0;
    for (int rep = 0; rep < 2; ++rep) {
      const double t0 = now_ms();
      for (int64_t i = 0; i < count; ++i) {
        const pw_status st = pw_server_submit(sv, s[i], t[i], eps[i], L[i], seeds ? seeds + i : nullptr, &tk[(size_t)i]);
        if (st != PW_OK) return st;
      }
      pw_status st = pw_server_drain(sv, 3600 * 1000);
      if (st != PW_OK) return st;
      secs = (now_ms() - t0) / 1000.0;
      for (int64_t i = 0; i < count; ++i) {
        st = pw_server_poll(sv, tk[(size_t)i], &got[(size_t)i]);
        if (st != PW_OK) return set_error(st, "pw_server_tune: a sample query failed");
      }
    }
    if (ref.empty()) ref = got;
    if (memcmp(ref.data(), got.data(), sizeof(double) * (size_t)count) != 0)
      return set_error(PW_ERR_INTERNAL, "pw_server_tune: two server variants gave different estimates");
    *qps = (double)count / secs;
    return PW_OK;
  };
  PW_CUDA_TRY(cudaSetDevice(g->device));
  if (!table) {
    // Without a table every policy runs the same per-visit jobs; what can be
    // chosen is the kernel's occupancy.  The running kernel (idle, about to
    // exit) finishes before the variant changes, so each burst is served by
    // the variant it times.
    int best = 0;
    for (int v = 0; v < 2; ++v) {
      PW_CUDA_TRY(cudaStreamSynchronize(sv->kstream));
      {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->minb = 2 + v;
        sv->grid = sv->grids[v];
      }
      const pw_status st = burst(&out->occupancy_qps[v]);
      if (st != PW_OK) return st;
      if (out->occupancy_qps[v] > out->occupancy_qps[best]) best = v;
    }
    PW_CUDA_TRY(cudaStreamSynchronize(sv->kstream));
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->minb = 2 + best;
      sv->grid = sv->grids[best];
    }
    out->queries_per_s[0] = out->occupancy_qps[best];
    out->policy = 0;
    out->occupancy = 2 + best;
    return PW_OK;
  }
  // candidate policies {table cost per probe, saving per visit}: the default
  // model, the graph's batch-fitted model, every query per-visit, every query
  // on the table
  const double cand[4][2] = {{(double)g->n, 2.5}, {g->table_probe_cost, g->table_visit_gain}, {1.0, 0.0}, {0.0, 1.0}};
  const bool valid[4] = {true, g->tuned != 0, true, true};
  int best = 0;
  for (int c = 0; c < 4; ++c) {
    if (!valid[c]) continue;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->table_probe_cost = cand[c][0];
      sv->table_visit_gain = cand[c][1];
    }
    PW_CUDA_TRY(cudaMemcpy(sv->d_model, cand[c], 2 * sizeof(double), cudaMemcpyHostToDevice));
    const pw_status st = burst(&out->queries_per_s[c]);
    if (st != PW_OK) return st;
    if (out->queries_per_s[c] > out->queries_per_s[best]) best = c;
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->table_probe_cost = cand[best][0];
    sv->table_visit_gain = cand[best][1];
  }
  PW_CUDA_TRY(cudaMemcpy(sv->d_model, cand[best], 2 * sizeof(double), cudaMemcpyHostToDevice));
  out->policy = best;
  out->occupancy = 4;
  return PW_OK;
}

pw_status pw_server_destroy(pw_server* sv) {
  if (!sv) return PW_OK;
  cudaSetDevice(sv->g->device);
  if (sv->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stopping = true;
      for (const Request& rq : sv->pending) {
        sv->results[rq.ticket] = {NAN, PW_ERR_CANCELLED, now_ms() - rq.t_submit_ms};
        sv->unfinished.erase(rq.ticket);
        sv->completed++;
      }
      sv->pending.clear();
    }
    sv->worker.join();
  }
  if (sv->d_stop && sv->h_stop && sv->kstream && sv->cstream) {
    *sv->h_stop = 1;
    cudaMemcpyAsync(sv->d_stop, sv->h_stop, sizeof(uint32_t), cudaMemcpyHostToDevice, sv->cstream);
    cudaStreamSynchronize(sv->cstream);
    cudaStreamSynchronize(sv->kstream);
  }
  cudaFree(sv->d_slots);
  cudaFree(sv->d_ctl);
  cudaFree(sv->d_ring_slot);
  cudaFree(sv->d_ring_stage);
  cudaFree(sv->d_ring_seq);
  cudaFree(sv->d_stop);
  cudaFree(sv->d_model);
  cudaFree(sv->d_pool);
  if (sv->h_slot_stage) cudaFreeHost(sv->h_slot_stage);
  if (sv->h_ring_stage_buf) cudaFreeHost(sv->h_ring_stage_buf);
  if (sv->h_ring_seq_buf) cudaFreeHost(sv->h_ring_seq_buf);
  if (sv->h_stop) cudaFreeHost(sv->h_stop);
  if (sv->h_comp) cudaFreeHost(sv->h_comp);
  if (sv->kstream) cudaStreamDestroy(sv->kstream);
  if (sv->cstream) cudaStreamDestroy(sv->cstream);
  delete sv;
  return PW_OK;
}

}  // extern "C"
