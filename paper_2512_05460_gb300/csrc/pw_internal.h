// Internal types shared by the translation units of libprobewalk.so.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "probewalk.h"

namespace pw {

// Per-query plan, one per query of a batch, resident in device memory.
struct QPlan {
  uint64_t seed;
  uint64_t tile_begin;   // first per-visit walk tile of this query (a tile is 32 replicas of one probe)
  uint64_t acc_begin;    // first per-visit probe accumulator
  uint64_t probe_begin;  // first Q slot (K slots)
  uint64_t table_begin;  // first entry of this query in the table kernel's probe list
  uint64_t q_begin;      // first Q slot of the query (the median reads G B values from here)
  int32_t s, t;
  int32_t L;
  int32_t status;        // pw_status of this query
  uint32_t K, R, B, G;
  uint32_t chunks;       // ceil(R / 32)
  uint32_t k_begin;      // first probe index (a range of blocks of a sharded query; else 0)
  uint32_t mode;         // walk kernel of the query's probes: 1 per-visit evaluation, 2 probe table
  uint32_t Bmax;         // ADAPTIVE: the most probes per block (PILOT's B; Q slots reserved: G Bmax); else 0
  double eps;
  double sigma2, qbar, theta;  // pilot diagnostics
};

// Totals written by the scan kernel.
struct Totals {
  unsigned long long tiles;         // per-visit tiles
  unsigned long long visit_probes;  // probes run by the per-visit kernel
  unsigned long long table_probes;  // probes run by the table kernel
  unsigned long long probes;        // all probes (Q slots)
  unsigned long long steps;         // sum of K * R * L (walk pairs times length)
  unsigned long long visits;        // sum of 2 K R (L + 1)
  unsigned long long pad[2];
};

struct ProfileState {
  bool enabled = false;
  struct Span {
    cudaEvent_t a, b;
    int kind;  // 0 main walk, 1 pilot walk, 2 finish, 3 series pass
  };
  std::vector<Span> spans;
  std::vector<cudaEvent_t> pool;
  std::vector<Totals*> pending, spare;  // pinned copies of profiled batches' totals
  double walk_ms = 0, pilot_ms = 0, finish_ms = 0, series_ms = 0;
  uint64_t walk_launches = 0, transitions = 0, pilot_transitions = 0, queries = 0, series_steps = 0;
};

// Budget inputs shared by all queries of a call (resolved defaults).
struct BudgetArgs {
  int32_t mode;
  int32_t K0, R0;
  uint32_t G;       // ceil(8 ln(1/delta)), evaluated on the host
  double c_B, c_R;
  uint64_t B_fixed, R_fixed;
  uint64_t R_max;
  uint64_t global_seed;
  int32_t d_min;
  double z;    // ADAPTIVE stopping rule's normal quantile
  double cap;  // ADAPTIVE: the most probes per block as a multiple of PILOT's B
};

struct DeviceBuffer {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// A host-array call captured as a CUDA graph: input copy, every launch of the
// pipeline, result copy.  Replayed while the call's shape (`key`: query count,
// probe total, budget, cost model, buffer addresses) repeats; a shape seen on
// two consecutive calls is captured.
struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned char> key, seen;
  uint64_t launches = 0;  // kernel launches in one replay
};

struct Workspace {
  DeviceBuffer plans, pilot_plans, tile_prefix, pilot_s, acc, q, totals, counters, queries, results, u_debug;
  Totals* host_totals = nullptr;  // pinned: totals of the latest batch (valid once last_use has completed)
  void* host_staging = nullptr;   // pinned
  size_t host_staging_bytes = 0;
  cudaEvent_t last_use = nullptr;
};

}  // namespace pw

struct pw_graph {
  int device = 0;
  int64_t n = 0, nnz = 0;
  int32_t d_min = 0, d_max = 0, bipartite = 0;
  std::vector<int32_t> deg;  // host copy of the degrees (host-side query planning)
  int sm_count = 0;
  // Walk-mode cost model: a query's probes run in the probe-table kernel when
  //   K * table_probe_cost < 2 K R (L + 1) * table_visit_gain.
  // Defaults (set at load): n and 2.5, in units of one Feistel pass per node
  // (table) against about 2.5 passes per visit (per-visit evaluation);
  // pw_autotune replaces them by nanoseconds measured on this graph.
  double table_probe_cost = 0.0, table_visit_gain = 2.5;
  int tuned = 0;
  int4* d_rec = nullptr;     // nnz neighbour records (fused layout only)
  int32_t* d_col = nullptr;  // nnz neighbour ids (always)
  int4* d_node = nullptr;    // n node records
  int layout = 1;            // walk access: 1 fused records, 2 col_idx + node records
  cudaStream_t stream = nullptr;
  std::map<std::pair<const void*, size_t>, int> grids;  // persistent grid per walk kernel and shared memory
  // Kernel variants (pw_autotune): per-visit kernel with compiler-chosen
  // registers (1) or registers capped for 3 blocks per SM (3); table-kernel
  // block size (0: by shared memory, else 256, 512 or 1024 threads).
  int visit_minb = 1;
  int table_threads = 0;
  int walk_policy = 0;  // walk_mode 0 means: 0 the cost model per query, 1 all per-visit, 2 all table
  // L2 access-policy window of the walk and server launches
  // (pw_graph_set_l2_window): 0 none, 1 the uniformly gathered array, 2 the
  // node records.  l2_prev_limit: the context's persisting set-aside before
  // this graph raised it (restored when the window is dropped).
  int l2_window = 0;
  cudaAccessPolicyWindow l2_apw{};
  size_t l2_prev_limit = 0;
  bool l2_limit_set = false;
  std::mutex lock;
  pw::GraphCache gcache;
  pw::Workspace ws;
  pw::ProfileState prof;
};

namespace pw {

// Launches fn on the graph's walk data: with the graph's L2 access-policy
// window as a launch attribute when one is set (the stream's own attributes
// are left alone), else a plain launch.
template <class... K, class... A>
inline cudaError_t launch_with_window(const pw_graph* g, void (*fn)(K...), int grid, int threads, size_t smem,
                                      cudaStream_t stream, A&&... args) {
  if (!g->l2_window) {
    fn<<<grid, threads, smem, stream>>>(args...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
  attr[0].val.accessPolicyWindow = g->l2_apw;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, static_cast<A&&>(args)...);
}

pw_status set_error(pw_status st, const std::string& msg);
// pw_graph_set_l2_window without the argument checks and the lock.
pw_status set_l2_window(pw_graph* g, int which);
// CUDA-event spans on a graph's stream, summed by pw_profile (no-ops unless enabled).
void prof_begin(pw_graph* g, cudaStream_t stream, cudaEvent_t* a);
void prof_end(pw_graph* g, cudaStream_t stream, cudaEvent_t a, int kind);
pw_status cuda_error(cudaError_t err, const char* what);
void count_launch();
void count_launches(int64_t delta);  // adjusts the launch count (graph replays, captures)
pw_status ensure_buffer(DeviceBuffer& b, size_t bytes);
void free_buffer(DeviceBuffer& b);
pw_status ensure_host_staging(Workspace& ws, size_t bytes);
void free_workspace(Workspace& ws);

// Resolve defaults; returns PW_ERR_ARG on invalid FIXED values.
pw_status resolve_budget(const pw_params* params, const pw_graph* g, BudgetArgs* out, double* delta_out);

// Run a batch whose query arrays are already on the device.  Writes beta and
// status (device).  If debug_u / debug_q / debug_visits are non-null the
// corresponding debug outputs are produced (device pointers sized by caller).
struct DebugOut {
  uint32_t* visits = nullptr;  // device, n counters of visits by the main walks
  float* u = nullptr;          // device, K R replica values of query 0 (single-query batches only)
  bool budget_only = false;    // stop after the budget (and pilot) stage
  int64_t g_begin = -1;        // >= 0: run only median-of-means blocks [g_begin, g_end) of query 0
  int64_t g_end = -1;
  double* block_means = nullptr;  // device, g_end - g_begin block means (instead of the median)
  bool time_walk = false;         // record the main walk kernels' duration (walk_ms, after the batch)
  float walk_ms = 0.f;
};
// Run a batch whose query arrays are on the device.  total_K: the sum of K over
// the queries when the caller knows it (host-array calls), else -1, and the
// batch reads it back from the device once (one synchronisation of `stream`).
pw_status run_batch(pw_graph* g, int64_t count, const int64_t* d_s, const int64_t* d_t, const double* d_eps,
                    const int32_t* d_L, const uint64_t* d_seeds, const pw_params* params, double* d_beta,
                    int32_t* d_status, cudaStream_t stream, DebugOut* dbg, int64_t total_K);

}  // namespace pw

#define PW_CUDA_TRY(expr)                                            \
  do {                                                               \
    cudaError_t _e = (expr);                                         \
    if (_e != cudaSuccess) return pw::cuda_error(_e, #expr);         \
  } while (0)
