// Graph loading (validation, neighbour-record layout, upload) and the small
// debug kernels (Philox, probe vector, single trajectory).
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "pw_device.cuh"
#include "pw_internal.h"

namespace pw {

// node[v] = {v, row_start(v), deg(v), bits(1/deg(v))}; in the fused layout
// also rec[e] = node[col[e]] for every CSR entry e (rec may be NULL).
__global__ void build_records_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                     int64_t n, int64_t nnz, int4* __restrict__ rec, int4* __restrict__ node) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t first = rec ? 0 : nnz;
  for (int64_t e = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz + n; e += stride) {
    const int32_t u = e < nnz ? col[e] : (int32_t)(e - nnz);
    const int32_t start = row_ptr[u];
    const int32_t d = row_ptr[u + 1] - start;
    const float inv = __fdiv_rn(1.0f, (float)d);
    const int4 r = make_int4(u, start, d, (int)__float_as_uint(inv));
    if (e < nnz)
      rec[e] = r;
    else
      node[e - nnz] = r;
  }
}

__global__ void debug_philox_kernel(uint4 ctr, uint2 key, uint4* out) {
  const Philox4 o = philox4x32_10(ctr.x, ctr.y, ctr.z, ctr.w, key.x, key.y);
  *out = make_uint4(o.x, o.y, o.z, o.w);
}

__global__ void debug_probe_kernel(uint32_t n, uint64_t seed, uint32_t k, uint32_t tag, int8_t* z, int32_t* r) {
  const Probe P = make_probe(n, seed, k, tag);
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    z[v] = (int8_t)probe_z(P, v);
  if (blockIdx.x == 0 && threadIdx.x == 0) *r = (int32_t)(n - P.n_active);
}

// One trajectory with the walk kernel's step rule: step i draws word (i & 3) of
// the Philox block (walk lo, walk hi, i >> 2, tag) and moves to neighbour
// floor(word * d / 2^32).
__global__ void debug_walk_kernel(const int32_t* __restrict__ col, const int4* __restrict__ node, int32_t start,
                                  int32_t L, uint64_t seed, uint64_t walk_id, uint32_t tag, int64_t* traj) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int4 cur = node[start];
  traj[0] = cur.x;
  for (int32_t i = 1; i <= L; ++i) {
    const Philox4 o = philox_seeded(seed, (uint32_t)walk_id, (uint32_t)(walk_id >> 32), (uint32_t)i >> 2, tag);
    const uint32_t w[4] = {o.x, o.y, o.z, o.w};
    const uint32_t j = __umulhi(w[i & 3], (uint32_t)cur.z);
    cur = node[col[(uint32_t)cur.y + j]];
    traj[i] = cur.x;
  }
}

// Sector-throughput ceiling of the walk's memory side: dependent random
// gathers with the walk's access per step (the next index depends on the
// loaded value, as in a walk), 8 independent chains per thread, no other work.
// Fused layout: one 16-B record uniform over the record array.  Split layout:
// a 4-B col_idx entry uniform over col_idx, then the node record it names.
template <bool SPLIT>
__global__ void __launch_bounds__(256) gather_peak_kernel(const int4* __restrict__ rec, const int32_t* __restrict__ col,
                                                         const int4* __restrict__ node, uint32_t nnz, uint32_t iters,
                                                         uint32_t* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (tid * 8u + (uint32_t)j) * 0x9E3779B1u + 0x7F4A7C15u;
  uint32_t acc = 0;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t e = __umulhi(x[j], nnz);
      const int4 r = SPLIT ? __ldg(node + __ldg(col + e)) : __ldg(rec + e);
      x[j] = x[j] * 1664525u + 1013904223u + (uint32_t)r.y;
      acc += (uint32_t)r.x;
    }
  }
  if (acc == 0x12345678u) sink[0] = acc;
}

static pw_status validate_csr(int64_t n, const int64_t* rp, const int32_t* col, int64_t nnz, uint32_t flags,
                              int32_t* d_min, int32_t* d_max, int32_t* bipartite) {
  if (rp[0] != 0 || rp[n] != nnz) return set_error(PW_ERR_GRAPH, "row_ptr must start at 0 and end at nnz");
  for (int64_t v = 0; v < n; ++v)
    if (rp[v + 1] < rp[v] || rp[v + 1] > nnz)
      return set_error(PW_ERR_GRAPH, "row_ptr is not monotone within [0, nnz] at node " + std::to_string(v));
  // per-row checks and symmetry, in parallel; the first offending node is reported
  int64_t bad_row = INT64_MAX, bad_sym = INT64_MAX;
  int32_t dmn = INT32_MAX, dmx = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(min : dmn, bad_row, bad_sym) reduction(max : dmx)
  for (int64_t v = 0; v < n; ++v) {
    const int64_t a = rp[v], b = rp[v + 1];
    const int64_t d = b - a;
    dmn = (int32_t)std::min<int64_t>(dmn, d);
    dmx = (int32_t)std::max<int64_t>(dmx, d);
    bool ok = d > 0;
    for (int64_t e = a; e < b && ok; ++e) {
      const int32_t u = col[e];
      if (u < 0 || u >= n || u == v || (e > a && col[e - 1] >= u)) ok = false;
    }
    if (!ok) {
      bad_row = std::min<int64_t>(bad_row, v);
      continue;
    }
    for (int64_t e = a; e < b; ++e) {
      const int32_t u = col[e];
      if (!std::binary_search(col + rp[u], col + rp[u + 1], (int32_t)v)) {
        bad_sym = std::min<int64_t>(bad_sym, v);
        break;
      }
    }
  }
  if (bad_row != INT64_MAX) {
    const int64_t v = bad_row, a = rp[v], b = rp[v + 1];
    if (b == a) return set_error(PW_ERR_GRAPH, "isolated node " + std::to_string(v));
    for (int64_t e = a; e < b; ++e) {
      const int32_t u = col[e];
      if (u < 0 || u >= n) return set_error(PW_ERR_GRAPH, "neighbour id out of range in row " + std::to_string(v));
      if (u == v) return set_error(PW_ERR_GRAPH, "self-loop at node " + std::to_string(v));
    }
    return set_error(PW_ERR_GRAPH, "row " + std::to_string(v) + " is not strictly increasing");
  }
  if (bad_sym != INT64_MAX) return set_error(PW_ERR_GRAPH, "an edge of node " + std::to_string(bad_sym) + " has no reverse");
  *d_min = dmn;
  *d_max = dmx;
  *bipartite = 0;
  if (!(flags & 1u)) {
    // breadth-first search from node 0: connectivity and 2-colouring
    std::vector<int8_t> colour((size_t)n, -1);
    std::vector<int32_t> queue;
    queue.reserve((size_t)n);
    colour[0] = 0;
    queue.push_back(0);
    bool two = true;
    for (size_t head = 0; head < queue.size(); ++head) {
      const int32_t v = queue[head];
      for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
        const int32_t u = col[e];
        if (colour[u] < 0) {
          colour[u] = (int8_t)(1 - colour[v]);
          queue.push_back(u);
        } else if (colour[u] == colour[v]) {
          two = false;
        }
      }
    }
    if ((int64_t)queue.size() != n) return set_error(PW_ERR_GRAPH, "graph is not connected");
    *bipartite = two ? 1 : 0;
  }
  return PW_OK;
}

static pw_status upload(pw_graph* g, const int64_t* rp64, const int32_t* col) {
  PW_CUDA_TRY(cudaSetDevice(g->device));
  PW_CUDA_TRY(cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device));
  PW_CUDA_TRY(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
  std::vector<int32_t> rp32((size_t)g->n + 1);
  for (int64_t i = 0; i <= g->n; ++i) rp32[(size_t)i] = (int32_t)rp64[i];
  g->deg.resize((size_t)g->n);
  for (int64_t i = 0; i < g->n; ++i) g->deg[(size_t)i] = rp32[(size_t)i + 1] - rp32[(size_t)i];
  int32_t *d_rp = nullptr, *d_col = nullptr;
  PW_CUDA_TRY(cudaMalloc(&d_rp, sizeof(int32_t) * (size_t)(g->n + 1)));
  PW_CUDA_TRY(cudaMalloc(&d_col, sizeof(int32_t) * (size_t)g->nnz));
  g->d_col = d_col;
  if (g->layout == 1) PW_CUDA_TRY(cudaMalloc(&g->d_rec, sizeof(int4) * (size_t)g->nnz));
  PW_CUDA_TRY(cudaMalloc(&g->d_node, sizeof(int4) * (size_t)g->n));
  PW_CUDA_TRY(cudaMemcpyAsync(d_rp, rp32.data(), sizeof(int32_t) * (size_t)(g->n + 1), cudaMemcpyHostToDevice,
                              g->stream));
  PW_CUDA_TRY(cudaMemcpyAsync(d_col, col, sizeof(int32_t) * (size_t)g->nnz, cudaMemcpyHostToDevice, g->stream));
  const int threads = 256;
  const int64_t work = g->nnz + g->n;
  const int blocks = (int)std::min<int64_t>((work + threads - 1) / threads, (int64_t)g->sm_count * 32);
  build_records_kernel<<<blocks, threads, 0, g->stream>>>(d_rp, d_col, g->n, g->nnz, g->d_rec, g->d_node);
  count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  PW_CUDA_TRY(cudaStreamSynchronize(g->stream));
  cudaFree(d_rp);
  PW_CUDA_TRY(cudaMallocHost(&g->ws.host_totals, sizeof(Totals)));
  PW_CUDA_TRY(cudaEventCreateWithFlags(&g->ws.last_use, cudaEventDisableTiming));
  return PW_OK;
}

// The L2 access-policy window of the walk launches (see pw_graph_set_l2_window).
// Caller holds g->lock or owns g alone.
pw_status set_l2_window(pw_graph* g, int which) {
  PW_CUDA_TRY(cudaSetDevice(g->device));
  if (g->l2_window) cudaCtxResetPersistingL2Cache();  // the old window's lines become normal
  g->l2_window = 0;
  g->l2_apw = cudaAccessPolicyWindow{};
  if (which == 0) {
    if (g->l2_limit_set) {
      g->l2_limit_set = false;
      PW_CUDA_TRY(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, g->l2_prev_limit));
    }
    return PW_OK;
  }
  int max_persist = 0, max_window = 0;
  PW_CUDA_TRY(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, g->device));
  PW_CUDA_TRY(cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, g->device));
  if (max_persist <= 0 || max_window <= 0) return set_error(PW_ERR_CUDA, "the device has no persisting L2");
  void* base = nullptr;
  size_t bytes = 0;
  if (which == 1 && g->layout == 2) {
    base = g->d_col;
    bytes = sizeof(int32_t) * (size_t)g->nnz;
  } else if (which == 1) {
    base = g->d_rec;
    bytes = sizeof(int4) * (size_t)g->nnz;
  } else {
    base = g->d_node;
    bytes = sizeof(int4) * (size_t)g->n;
  }
  const size_t num = bytes < (size_t)max_window ? bytes : (size_t)max_window;
  const size_t want = num < (size_t)max_persist ? num : (size_t)max_persist;
  if (!g->l2_limit_set) PW_CUDA_TRY(cudaDeviceGetLimit(&g->l2_prev_limit, cudaLimitPersistingL2CacheSize));
  PW_CUDA_TRY(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want));
  g->l2_limit_set = true;
  size_t got = 0;
  PW_CUDA_TRY(cudaDeviceGetLimit(&got, cudaLimitPersistingL2CacheSize));  // as granted
  if (got == 0) return set_error(PW_ERR_CUDA, "no persisting L2 set-aside granted");
  // a hit ratio that fits the window's persisting lines in the set-aside
  g->l2_apw.base_ptr = base;
  g->l2_apw.num_bytes = num;
  g->l2_apw.hitRatio = got >= num ? 1.0f : (float)((double)got / (double)num);
  g->l2_apw.hitProp = cudaAccessPropertyPersisting;
  g->l2_apw.missProp = cudaAccessPropertyStreaming;
  g->l2_window = which;
  return PW_OK;
}

static void destroy(pw_graph* g) {
  if (!g) return;
  cudaSetDevice(g->device);
  if (g->stream) cudaStreamSynchronize(g->stream);
  if (g->l2_window || g->l2_limit_set) set_l2_window(g, 0);
  free_workspace(g->ws);
  for (auto& sp : g->prof.spans) {
    cudaEventDestroy(sp.a);
    cudaEventDestroy(sp.b);
  }
  for (cudaEvent_t e : g->prof.pool) cudaEventDestroy(e);
  if (g->gcache.exec) cudaGraphExecDestroy(g->gcache.exec);
  for (pw::Totals* h : g->prof.pending) cudaFreeHost(h);
  for (pw::Totals* h : g->prof.spare) cudaFreeHost(h);
  if (g->d_rec) cudaFree(g->d_rec);
  if (g->d_col) cudaFree(g->d_col);
  if (g->d_node) cudaFree(g->d_node);
  if (g->stream) cudaStreamDestroy(g->stream);
  delete g;
}

static pw_status load_common(int64_t n, const int64_t* rp, const int32_t* col, int64_t nnz, int32_t device,
                             uint32_t flags, pw_graph** out) {
  if (!out) return set_error(PW_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!rp || !col) return set_error(PW_ERR_ARG, "row_ptr/col_idx is NULL");
  if (n < 2 || n >= (int64_t)1 << 31) return set_error(PW_ERR_ARG, "n must lie in [2, 2^31)");
  if (nnz < 1 || nnz >= (int64_t)1 << 31) return set_error(PW_ERR_ARG, "nnz must lie in [1, 2^31)");
  int32_t dmn = 0, dmx = 0, bip = 0;
  pw_status st = validate_csr(n, rp, col, nnz, flags, &dmn, &dmx, &bip);
  if (st != PW_OK) return st;
  pw_graph* g = new (std::nothrow) pw_graph();
  if (!g) return set_error(PW_ERR_NOMEM, "host allocation failed");
  g->device = device;
  g->n = n;
  g->nnz = nnz;
  g->table_probe_cost = (double)n;
  g->d_min = dmn;
  g->d_max = dmx;
  g->bipartite = bip;
  // walk layout (flags bit 1 / bit 2 force one): fused 16-byte records while
  // they fill at most half of the L2 (64 MiB); col_idx plus node records when
  // those two arrays stay near the L2's size (160 MiB: most of a step's two
  // gathers hit L2); fused again beyond that, where the split layout's two
  // gathers would both go to DRAM (R-MAT 2^24: 16.6 vs 14.3 queries/s)
  const double fused_bytes = 16.0 * (double)nnz, split_bytes = 4.0 * (double)nnz + 16.0 * (double)n;
  if (flags & 2u)
    g->layout = 1;
  else if (flags & 4u)
    g->layout = 2;
  else
    g->layout = (fused_bytes > (double)((size_t)64 << 20) && split_bytes <= (double)((size_t)160 << 20)) ? 2 : 1;
  st = upload(g, rp, col);
  if (st != PW_OK) {
    destroy(g);
    return st;
  }
  *out = g;
  return PW_OK;
}

}  // namespace pw

extern "C" {

pw_status pw_graph_load(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, int64_t nnz, int32_t device,
                        uint32_t flags, pw_graph** out) {
  return pw::load_common(n, row_ptr, col_idx, nnz, device, flags, out);
}

pw_status pw_graph_load32(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t nnz, int32_t device,
                          uint32_t flags, pw_graph** out) {
  if (!row_ptr || n < 2) return pw::set_error(PW_ERR_ARG, "row_ptr is NULL or n < 2");
  std::vector<int64_t> rp((size_t)n + 1);
  for (int32_t i = 0; i <= n; ++i) rp[(size_t)i] = row_ptr[i];
  return pw::load_common(n, rp.data(), col_idx, nnz, device, flags, out);
}

void pw_graph_free(pw_graph* g) { pw::destroy(g); }

pw_status pw_graph_set_l2_window(pw_graph* g, int32_t which) {
  if (!g) return pw::set_error(PW_ERR_ARG, "graph is NULL");
  if (which < 0 || which > 2) return pw::set_error(PW_ERR_ARG, "which must be 0, 1 or 2");
  if (which == 2 && g->layout != 2) return pw::set_error(PW_ERR_ARG, "a node-record window needs the split layout");
  std::lock_guard<std::mutex> guard(g->lock);
  return pw::set_l2_window(g, which);
}

pw_status pw_graph_info(const pw_graph* g, int64_t* n, int64_t* nnz, int32_t* d_min, int32_t* d_max,
                        int32_t* bipartite) {
  if (!g) return pw::set_error(PW_ERR_ARG, "graph is NULL");
  if (n) *n = g->n;
  if (nnz) *nnz = g->nnz;
  if (d_min) *d_min = g->d_min;
  if (d_max) *d_max = g->d_max;
  if (bipartite) *bipartite = g->bipartite;
  return PW_OK;
}

pw_status pw_debug_philox(pw_graph* g, const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  if (!g || !ctr || !key || !out) return pw::set_error(PW_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  pw::DeviceBuffer& b = g->ws.results;
  pw_status st = pw::ensure_buffer(b, 64);
  if (st != PW_OK) return st;
  pw::debug_philox_kernel<<<1, 1, 0, g->stream>>>(make_uint4(ctr[0], ctr[1], ctr[2], ctr[3]),
                                                   make_uint2(key[0], key[1]), (uint4*)b.ptr);
  pw::count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  PW_CUDA_TRY(cudaMemcpyAsync(out, b.ptr, 16, cudaMemcpyDeviceToHost, g->stream));
  PW_CUDA_TRY(cudaStreamSynchronize(g->stream));
  return PW_OK;
}

pw_status pw_debug_probe(pw_graph* g, uint64_t seed, uint32_t k, uint32_t tag, int8_t* z, int32_t* r) {
  if (!g || !z) return pw::set_error(PW_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  pw::DeviceBuffer& b = g->ws.results;
  pw_status st = pw::ensure_buffer(b, (size_t)g->n + 64);
  if (st != PW_OK) return st;
  int32_t* d_r = (int32_t*)((char*)b.ptr + ((size_t)g->n + 15) / 16 * 16);
  const int blocks = (int)std::min<int64_t>((g->n + 255) / 256, (int64_t)g->sm_count * 8);
  pw::debug_probe_kernel<<<blocks, 256, 0, g->stream>>>((uint32_t)g->n, seed, k, tag, (int8_t*)b.ptr, d_r);
  pw::count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  PW_CUDA_TRY(cudaMemcpyAsync(z, b.ptr, (size_t)g->n, cudaMemcpyDeviceToHost, g->stream));
  int32_t rr = 0;
  PW_CUDA_TRY(cudaMemcpyAsync(&rr, d_r, sizeof rr, cudaMemcpyDeviceToHost, g->stream));
  PW_CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (r) *r = rr;
  return PW_OK;
}

pw_status pw_debug_gather_peak(pw_graph* g, int32_t iters, double* sectors_per_s) {
  if (!g || !sectors_per_s || iters < 1) return pw::set_error(PW_ERR_ARG, "NULL argument or iters < 1");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  pw::DeviceBuffer& b = g->ws.results;
  pw_status st = pw::ensure_buffer(b, 64);
  if (st != PW_OK) return st;
  int nb = 0;
  const bool split = g->layout == 2;
  PW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &nb, split ? pw::gather_peak_kernel<true> : pw::gather_peak_kernel<false>, 256, 0));
  const int blocks = g->sm_count * (nb > 0 ? nb : 1);
  cudaEvent_t e0, e1;
  PW_CUDA_TRY(cudaEventCreate(&e0));
  PW_CUDA_TRY(cudaEventCreate(&e1));
  double best = 0.0;
  for (int rep = 0; rep < 3; ++rep) {
    PW_CUDA_TRY(cudaEventRecord(e0, g->stream));
    if (split)
      pw::gather_peak_kernel<true><<<blocks, 256, 0, g->stream>>>(g->d_rec, g->d_col, g->d_node, (uint32_t)g->nnz,
                                                                  (uint32_t)iters, (uint32_t*)b.ptr);
    else
      pw::gather_peak_kernel<false><<<blocks, 256, 0, g->stream>>>(g->d_rec, g->d_col, g->d_node, (uint32_t)g->nnz,
                                                                   (uint32_t)iters, (uint32_t*)b.ptr);
    pw::count_launch();
    PW_CUDA_TRY(cudaGetLastError());
    PW_CUDA_TRY(cudaEventRecord(e1, g->stream));
    PW_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    PW_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    const double rate = (double)blocks * 256.0 * 8.0 * (double)iters / (ms * 1e-3);
    if (rate > best) best = rate;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *sectors_per_s = best;
  return PW_OK;
}

pw_status pw_debug_walk(pw_graph* g, int64_t start, int32_t L, uint64_t seed, uint64_t walk_id, uint32_t tag,
                        int64_t* trajectory) {
  if (!g || !trajectory) return pw::set_error(PW_ERR_ARG, "NULL argument");
  if (start < 0 || start >= g->n || L < 0) return pw::set_error(PW_ERR_ARG, "start or L out of range");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  pw::DeviceBuffer& b = g->ws.results;
  pw_status st = pw::ensure_buffer(b, sizeof(int64_t) * ((size_t)L + 1));
  if (st != PW_OK) return st;
  pw::debug_walk_kernel<<<1, 32, 0, g->stream>>>(g->d_col, g->d_node, (int32_t)start, L, seed, walk_id, tag,
                                                 (int64_t*)b.ptr);
  pw::count_launch();
  PW_CUDA_TRY(cudaGetLastError());
  PW_CUDA_TRY(cudaMemcpyAsync(trajectory, b.ptr, sizeof(int64_t) * ((size_t)L + 1), cudaMemcpyDeviceToHost,
                              g->stream));
  PW_CUDA_TRY(cudaStreamSynchronize(g->stream));
  return PW_OK;
}

}  // extern "C"
