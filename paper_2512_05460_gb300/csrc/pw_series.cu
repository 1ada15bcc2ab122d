// Truncated series of Lemma 2.3 on the GPU: h^(L) = sum_{i=0}^{L} P^i D^{-1} b_st
// and beta^(L) = ||h||^2 - (1^T h)^2 / n (Eq. tr-beta-exp-Liu), for batches of
// queries (the deterministic quantity the paper's PUSH computes).
//
// Arithmetic: GB300 issues FP64 at about 2 lane operations per SM per clock,
// against 128 for FP32, and an FP64 step was bound by that pipe.  x, y and h
// are therefore held as double-float pairs (hi + lo, two FP32 values with
// |lo| <= ulp(hi)/2, a 48-bit significand), added and multiplied with exact
// error-free transformations (TwoSum, and TwoProd by fused multiply-add), each
// a handful of FP32 operations; the final reduction to beta is FP64.
//
// 32 queries per pass, one warp lane per query column.  x, y and h are n x 32
// row-major (a node's 32 pairs are one 256-byte row), so gathering x over a
// node's neighbours reads whole lines.  Iteration i adds x_i to h and forms
// x_{i+1} = P x_i with (P x)_v = (sum_{u in N(v)} x_u) * (1/d_v), neighbours
// read from col_idx (4 bytes per entry).  Rows of at most 1024
// entries take one warp each and add in CSR order; longer rows (the hubs of
// power-law graphs) are cut into 1024-entry segments whose partial sums are
// added in segment order, so one hub does not hold up a whole step.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pw_device.cuh"
#include "pw_internal.h"

namespace pw {

constexpr int kSeriesCols = 32;
constexpr int32_t kSeriesSegEdges = 1024;  // rows with more entries are split into segments of this size

// ---- double-float arithmetic (value = hi + lo) -----------------------------
// TwoSum (Knuth): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Sum of two pairs; both parts by TwoSum, then renormalised (relative error
// about 2^-46 of the result).
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float s1, e1, s2, e2;
  two_sum(a.x, b.x, s1, e1);
  two_sum(a.y, b.y, s2, e2);
  e1 = __fadd_rn(e1, s2);
  float h = __fadd_rn(s1, e1);
  e1 = __fsub_rn(e1, __fsub_rn(h, s1));
  e1 = __fadd_rn(e1, e2);
  const float hi = __fadd_rn(h, e1);
  return make_float2(hi, __fsub_rn(e1, __fsub_rn(hi, h)));
}

// Product of two pairs; TwoProd of the high parts by fused multiply-add.
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float hi = __fadd_rn(p, e);
  return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, p)));
}

__device__ __forceinline__ float2 df_from_double(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

__global__ void series_init_kernel(float2* __restrict__ x, float2* __restrict__ h, uint32_t n) {
  const size_t total = (size_t)n * kSeriesCols;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    x[i] = make_float2(0.f, 0.f);
    h[i] = make_float2(0.f, 0.f);
  }
}

// Per-pass control block, written by the host before each pass (so one
// captured graph serves every pass of the same L).
struct SeriesCtl {
  int2 st[kSeriesCols];  // (s, t) of each column
  int32_t ncols;
  int32_t pad;
};

__global__ void series_seed_kernel(float2* __restrict__ x, const SeriesCtl* __restrict__ ctl,
                                   const int4* __restrict__ node) {
  const int c = threadIdx.x;
  if (c >= ctl->ncols) return;
  const int s = ctl->st[c].x, t = ctl->st[c].y;
  if (s == t) return;
  x[(size_t)s * kSeriesCols + c] = df_from_double(1.0 / (double)node[s].z);
  x[(size_t)t * kSeriesCols + c] = df_from_double(-1.0 / (double)node[t].z);
}

// 1/d_v as a pair, once per call.
__global__ void series_inv_degree_kernel(const int4* __restrict__ node, float2* __restrict__ inv, uint32_t n) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    inv[v] = df_from_double(1.0 / (double)__ldg(&node[v].z));
}

// Sum of x_u (column = lane) over the neighbour entries [e0, e1) of one row,
// added in CSR order.  A warp loads 32 neighbour ids with one coalesced load
// and keeps 8 row loads in flight before adding them in order.
__device__ __forceinline__ float2 series_row_sum(const float2* __restrict__ x, const int32_t* __restrict__ col,
                                                 int32_t e0, int32_t e1, uint32_t lane) {
  float2 acc = make_float2(0.f, 0.f);
  for (int32_t b = e0; b < e1; b += 32) {
    const int cnt = e1 - b < 32 ? e1 - b : 32;
    const int u_l = (int)lane < cnt ? __ldg(&col[b + (int)lane]) : 0;
    int j = 0;
    for (; j + 8 <= cnt; j += 8) {
      float2 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int u = __shfl_sync(0xffffffffu, u_l, j + q);
        v[q] = __ldg(x + (size_t)u * kSeriesCols + lane);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) acc = df_add(acc, v[q]);
    }
    for (; j < cnt; ++j) {
      const int u = __shfl_sync(0xffffffffu, u_l, j);
      acc = df_add(acc, __ldg(x + (size_t)u * kSeriesCols + lane));
    }
  }
  return acc;
}

// Rows of degree <= kSeriesSegEdges, one warp per row (grid-stride, the next
// row's record fetched while this one is summed):
// h_v += x_v; y_v = (sum over neighbours of x_u) * (1/d_v).  Heavier rows
// are left to the segment kernels below.
__global__ void __launch_bounds__(256) series_light_kernel(const float2* __restrict__ x, float2* __restrict__ y,
                                                           float2* __restrict__ h, const int32_t* __restrict__ col,
                                                           const int4* __restrict__ node,
                                                           const float2* __restrict__ inv, uint32_t n, int last) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int4 nv = v < n ? __ldg(node + v) : make_int4(0, 0, 0, 0);
  for (; v < n; v += warps) {
    const uint32_t vn = v + warps;
    const int4 nv_next = vn < n ? __ldg(node + vn) : make_int4(0, 0, 0, 0);  // in flight during this row
    if (nv.z <= kSeriesSegEdges) {
      const size_t row = (size_t)v * kSeriesCols + lane;
      h[row] = df_add(h[row], x[row]);
      if (!last) y[row] = df_mul(series_row_sum(x, col, nv.y, nv.y + nv.z, lane), __ldg(inv + v));
    }
    nv = nv_next;
  }
}

// One warp per segment of a heavy row: the partial sum of its entries.
__global__ void __launch_bounds__(256) series_segment_kernel(const float2* __restrict__ x,
                                                             float2* __restrict__ partial,
                                                             const int32_t* __restrict__ col,
                                                             const int4* __restrict__ segs, int32_t nseg) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < (uint32_t)nseg; i += warps) {
    const int4 sg = __ldg(segs + i);  // {row, e_begin, e_end, partial slot}
    partial[(size_t)sg.w * kSeriesCols + lane] = series_row_sum(x, col, sg.y, sg.z, lane);
  }
}

// One warp per heavy row: h_v += x_v; y_v = (partials in segment order) * (1/d_v).
__global__ void __launch_bounds__(256) series_heavy_finish_kernel(const float2* __restrict__ x,
                                                                  float2* __restrict__ y, float2* __restrict__ h,
                                                                  const float2* __restrict__ partial,
                                                                  const int4* __restrict__ rows, int32_t nrows,
                                                                  const float2* __restrict__ inv, int last) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < (uint32_t)nrows; i += warps) {
    const int4 hr = __ldg(rows + i);  // {row, first partial slot, partial count, -}
    const size_t row = (size_t)hr.x * kSeriesCols + lane;
    h[row] = df_add(h[row], x[row]);
    if (last) continue;
    float2 acc = make_float2(0.f, 0.f);
    for (int32_t p = 0; p < hr.z; ++p) acc = df_add(acc, partial[(size_t)(hr.y + p) * kSeriesCols + lane]);
    y[row] = df_mul(acc, __ldg(inv + hr.x));
  }
}

// Per column: sum of h^2 and of h over nodes in FP64 (fixed order: per-thread
// strided partial sums, then a shared-memory tree), then beta = sq - tot^2 / n.
__global__ void series_reduce_kernel(const float2* __restrict__ h, uint32_t n, const SeriesCtl* __restrict__ ctl,
                                     double* __restrict__ out) {
  __shared__ double ssq[256], stot[256];
  const int c = blockIdx.x;
  if (c >= ctl->ncols) return;
  double sq = 0.0, tot = 0.0;
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
    const float2 p = h[(size_t)v * kSeriesCols + c];
    const double x = (double)p.x + (double)p.y;
    sq += x * x;
    tot += x;
  }
  ssq[threadIdx.x] = sq;
  stot[threadIdx.x] = tot;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      ssq[threadIdx.x] += ssq[threadIdx.x + w];
      stot[threadIdx.x] += stot[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = ssq[0] - stot[0] * stot[0] / (double)n;
}

}  // namespace pw

using namespace pw;

extern "C" pw_status pw_series_batch(pw_graph* g, int64_t count, const int64_t* s, const int64_t* t, const int32_t* L,
                                     double* beta_L) {
  if (!g) return set_error(PW_ERR_ARG, "graph is NULL");
  if (count < 0) return set_error(PW_ERR_ARG, "count < 0");
  if (count == 0) return PW_OK;
  if (!s || !t || !L || !beta_L) return set_error(PW_ERR_ARG, "NULL array");
  for (int64_t i = 0; i < count; ++i)
    if (s[i] < 0 || s[i] >= g->n || t[i] < 0 || t[i] >= g->n || L[i] < 0)
      return set_error(PW_ERR_ARG, "query " + std::to_string(i) + ": node id out of range or L < 0");
  std::lock_guard<std::mutex> guard(g->lock);
  PW_CUDA_TRY(cudaSetDevice(g->device));
  const size_t n = (size_t)g->n;
  const size_t bytes = sizeof(float2) * n * kSeriesCols;
  // rows of more than kSeriesSegEdges entries: segments {row, e_begin, e_end,
  // partial slot} and rows {row, first slot, slot count}, in CSR order
  std::vector<int4> segs, heavy;
  {
    int64_t start = 0;
    int32_t slot = 0;
    for (int64_t v = 0; v < g->n; ++v) {
      const int32_t d = g->deg[(size_t)v];
      if (d > kSeriesSegEdges) {
        const int32_t first = slot;
        for (int64_t e = start; e < start + d; e += kSeriesSegEdges) {
          const int64_t e1 = std::min<int64_t>(e + kSeriesSegEdges, start + d);
          segs.push_back(make_int4((int)v, (int)e, (int)e1, slot++));
        }
        heavy.push_back(make_int4((int)v, first, slot - first, 0));
      }
      start += d;
    }
  }
  DeviceBuffer xb, yb, hb, sb, ob, segb, rowb, partb, invb;
  pw_status st;
  auto release = [&]() {
    free_buffer(xb);
    free_buffer(yb);
    free_buffer(hb);
    free_buffer(sb);
    free_buffer(ob);
    free_buffer(segb);
    free_buffer(rowb);
    free_buffer(partb);
    free_buffer(invb);
  };
  if ((st = ensure_buffer(xb, bytes)) != PW_OK || (st = ensure_buffer(yb, bytes)) != PW_OK ||
      (st = ensure_buffer(hb, bytes)) != PW_OK || (st = ensure_buffer(sb, sizeof(SeriesCtl))) != PW_OK ||
      (st = ensure_buffer(ob, sizeof(double) * kSeriesCols)) != PW_OK ||
      (st = ensure_buffer(invb, sizeof(float2) * n)) != PW_OK ||
      (!segs.empty() && ((st = ensure_buffer(segb, sizeof(int4) * segs.size())) != PW_OK ||
                         (st = ensure_buffer(rowb, sizeof(int4) * heavy.size())) != PW_OK ||
                         (st = ensure_buffer(partb, sizeof(float2) * kSeriesCols * segs.size())) != PW_OK))) {
    release();
    return st;
  }
  cudaStream_t stream = g->stream;
  const int threads = 256;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, series_light_kernel, threads, 0) != cudaSuccess || occ < 1)
    occ = 1;
  const int grid = g->sm_count * occ;
  const int32_t nseg = (int32_t)segs.size(), nheavy = (int32_t)heavy.size();
  const int seg_grid = (int)std::min<int64_t>((int64_t)grid, ((int64_t)nseg * 32 + threads - 1) / threads);
  const int heavy_grid = (int)std::min<int64_t>((int64_t)grid, ((int64_t)nheavy * 32 + threads - 1) / threads);
  cudaError_t e = cudaSuccess;
  const float2* inv = (const float2*)invb.ptr;
  series_inv_degree_kernel<<<grid, threads, 0, stream>>>(g->d_node, (float2*)invb.ptr, (uint32_t)n);
  count_launch();
  if (nseg > 0) {
    e = cudaMemcpyAsync(segb.ptr, segs.data(), sizeof(int4) * segs.size(), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rowb.ptr, heavy.data(), sizeof(int4) * heavy.size(), cudaMemcpyHostToDevice, stream);
  }
  // One pass (init, seed, L + 1 steps, reduce) enqueued on the stream; returns
  // the number of kernels.  A pass of L + 1 steps is one to three launches
  // per step, so it is captured once per distinct L as a CUDA graph and the
  // graph is replayed for every 32-query group of that L.
  const SeriesCtl* ctl_d = (const SeriesCtl*)sb.ptr;
  auto enqueue_pass = [&](int32_t Lc) -> int {
    int kernels = 0;
    float2* x = (float2*)xb.ptr;
    float2* y = (float2*)yb.ptr;
    float2* h = (float2*)hb.ptr;
    series_init_kernel<<<grid, threads, 0, stream>>>(x, h, (uint32_t)n);
    series_seed_kernel<<<1, kSeriesCols, 0, stream>>>(x, ctl_d, g->d_node);
    kernels += 2;
    for (int32_t i = 0; i <= Lc; ++i) {
      const int last = i == Lc;
      series_light_kernel<<<grid, threads, 0, stream>>>(x, y, h, g->d_col, g->d_node, inv, (uint32_t)n, last);
      ++kernels;
      if (nheavy > 0) {
        if (!last) {
          series_segment_kernel<<<seg_grid, threads, 0, stream>>>(x, (float2*)partb.ptr, g->d_col,
                                                                  (const int4*)segb.ptr, nseg);
          ++kernels;
        }
        series_heavy_finish_kernel<<<heavy_grid, threads, 0, stream>>>(x, y, h, (const float2*)partb.ptr,
                                                                       (const int4*)rowb.ptr, nheavy, inv, last);
        ++kernels;
      }
      std::swap(x, y);
    }
    series_reduce_kernel<<<kSeriesCols, 256, 0, stream>>>(h, (uint32_t)n, ctl_d, (double*)ob.ptr);
    return kernels + 1;
  };
  cudaGraphExec_t exec = nullptr;
  int32_t exec_L = -1;
  int exec_kernels = 0;
  // queries with the same L share a pass: group by L in input order
  std::vector<int64_t> order((size_t)count);
  for (int64_t i = 0; i < count; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return L[a] < L[b]; });
  for (size_t pos = 0; pos < order.size() && e == cudaSuccess;) {
    const int32_t Lc = L[order[pos]];
    SeriesCtl ctl;
    memset(&ctl, 0, sizeof ctl);
    std::vector<int64_t> idx;
    while (pos < order.size() && ctl.ncols < kSeriesCols && L[order[pos]] == Lc) {
      const int64_t i = order[pos++];
      ctl.st[ctl.ncols++] = make_int2((int)s[i], (int)t[i]);
      idx.push_back(i);
    }
    e = cudaMemcpyAsync(sb.ptr, &ctl, sizeof ctl, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) break;
    if (exec_L != Lc) {
      if (exec) cudaGraphExecDestroy(exec);
      exec = nullptr;
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) break;
      exec_kernels = enqueue_pass(Lc);
      const cudaError_t e_launch = cudaGetLastError();
      e = cudaStreamEndCapture(stream, &graph);  // always ends the capture
      if (e == cudaSuccess) e = e_launch;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) break;
      exec_L = Lc;
    }
    cudaEvent_t ev = nullptr;
    prof_begin(g, stream, &ev);
    e = cudaGraphLaunch(exec, stream);
    for (int k = 0; k < exec_kernels; ++k) count_launch();
    prof_end(g, stream, ev, 3);
    if (e != cudaSuccess) break;
    if (g->prof.enabled) g->prof.series_steps += (uint64_t)Lc + 1;
    std::vector<double> res((size_t)ctl.ncols);
    e = cudaMemcpyAsync(res.data(), ob.ptr, sizeof(double) * ctl.ncols, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    for (int c = 0; c < ctl.ncols && e == cudaSuccess; ++c) {
      const int64_t i = idx[(size_t)c];
      beta_L[i] = s[i] == t[i] ? 0.0 : res[(size_t)c];
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  release();
  if (e != cudaSuccess) return cuda_error(e, "series");
  PW_CUDA_TRY(cudaGetLastError());
  return PW_OK;
}
