// Truncated series of Lemma 2.3 on the GPU: h^(L) = sum_{i=0}^{L} P^i D^{-1} b_st
// and beta^(L) = ||h||^2 - (1^T h)^2 / n (Eq. tr-beta-exp-Liu), FP64, for
// batches of queries (the deterministic quantity the paper's PUSH computes).
//
// 32 queries per pass, one warp lane per query column.  x, y and h are n x 32
// row-major (a node's 32 values are one 256-byte line), so gathering x over a
// node's neighbours reads whole lines.  Iteration i adds x_i to h and forms
// x_{i+1} = P x_i with (P x)_v = (sum_{u in N(v)} x_u) / d_v, neighbours taken
// from the same 16-byte records the walks use.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pw_device.cuh"
#include "pw_internal.h"

namespace pw {

constexpr int kSeriesCols = 32;

__global__ void series_init_kernel(double* __restrict__ x, double* __restrict__ h, uint32_t n) {
  const size_t total = (size_t)n * kSeriesCols;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    x[i] = 0.0;
    h[i] = 0.0;
  }
}

__global__ void series_seed_kernel(double* __restrict__ x, const int2* __restrict__ st, const int4* __restrict__ node,
                                   int ncols) {
  const int c = threadIdx.x;
  if (c >= ncols) return;
  const int s = st[c].x, t = st[c].y;
  if (s == t) return;
  x[(size_t)s * kSeriesCols + c] = 1.0 / (double)node[s].z;
  x[(size_t)t * kSeriesCols + c] = -1.0 / (double)node[t].z;
}

// One warp per node v: h_v += x_v; y_v = (sum over neighbours of x_u) / d_v.
__global__ void __launch_bounds__(256) series_step_kernel(const double* __restrict__ x, double* __restrict__ y,
                                                          double* __restrict__ h, const int4* __restrict__ rec,
                                                          const int4* __restrict__ node, uint32_t n, int last) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const size_t row = (size_t)v * kSeriesCols + lane;
    h[row] += x[row];
    if (last) continue;
    const int4 nv = __ldg(node + v);
    double acc = 0.0;
    for (int32_t e = nv.y; e < nv.y + nv.z; ++e) {
      const int u = __ldg(&rec[e].x);
      acc += x[(size_t)u * kSeriesCols + lane];
    }
    y[row] = acc / (double)nv.z;
  }
}

// Per column: sum of h^2 and of h over nodes (fixed order: per-thread strided
// partial sums, then a shared-memory tree), then beta = sq - tot^2 / n.
__global__ void series_reduce_kernel(const double* __restrict__ h, uint32_t n, int ncols, double* __restrict__ out) {
  __shared__ double ssq[256], stot[256];
  const int c = blockIdx.x;
  if (c >= ncols) return;
  double sq = 0.0, tot = 0.0;
  for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
    const double x = h[(size_t)v * kSeriesCols + c];
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
  const size_t bytes = sizeof(double) * n * kSeriesCols;
  DeviceBuffer xb, yb, hb, sb, ob;
  pw_status st;
  auto release = [&]() {
    free_buffer(xb);
    free_buffer(yb);
    free_buffer(hb);
    free_buffer(sb);
    free_buffer(ob);
  };
  if ((st = ensure_buffer(xb, bytes)) != PW_OK || (st = ensure_buffer(yb, bytes)) != PW_OK ||
      (st = ensure_buffer(hb, bytes)) != PW_OK || (st = ensure_buffer(sb, sizeof(int2) * kSeriesCols)) != PW_OK ||
      (st = ensure_buffer(ob, sizeof(double) * kSeriesCols)) != PW_OK) {
    release();
    return st;
  }
  cudaStream_t stream = g->stream;
  const int threads = 256;
  const int grid = g->sm_count * 8;
  std::vector<int2> stv(kSeriesCols);
  cudaError_t e = cudaSuccess;
  // queries with the same L share a pass: group by L in input order
  std::vector<int64_t> order((size_t)count);
  for (int64_t i = 0; i < count; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return L[a] < L[b]; });
  for (size_t pos = 0; pos < order.size() && e == cudaSuccess;) {
    const int32_t Lc = L[order[pos]];
    int ncols = 0;
    std::vector<int64_t> idx;
    while (pos < order.size() && ncols < kSeriesCols && L[order[pos]] == Lc) {
      const int64_t i = order[pos++];
      stv[(size_t)ncols++] = make_int2((int)s[i], (int)t[i]);
      idx.push_back(i);
    }
    double* x = (double*)xb.ptr;
    double* y = (double*)yb.ptr;
    double* h = (double*)hb.ptr;
    e = cudaMemcpyAsync(sb.ptr, stv.data(), sizeof(int2) * ncols, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) break;
    series_init_kernel<<<grid, threads, 0, stream>>>(x, h, (uint32_t)n);
    series_seed_kernel<<<1, kSeriesCols, 0, stream>>>(x, (const int2*)sb.ptr, g->d_node, ncols);
    count_launch();
    count_launch();
    for (int32_t i = 0; i <= Lc; ++i) {
      series_step_kernel<<<grid, threads, 0, stream>>>(x, y, h, g->d_rec, g->d_node, (uint32_t)n, i == Lc);
      count_launch();
      std::swap(x, y);
    }
    series_reduce_kernel<<<ncols, 256, 0, stream>>>(h, (uint32_t)n, ncols, (double*)ob.ptr);
    count_launch();
    std::vector<double> res((size_t)ncols);
    e = cudaMemcpyAsync(res.data(), ob.ptr, sizeof(double) * ncols, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    for (int c = 0; c < ncols && e == cudaSuccess; ++c) {
      const int64_t i = idx[(size_t)c];
      beta_L[i] = s[i] == t[i] ? 0.0 : res[(size_t)c];
    }
  }
  release();
  if (e != cudaSuccess) return cuda_error(e, "series");
  PW_CUDA_TRY(cudaGetLastError());
  return PW_OK;
}
