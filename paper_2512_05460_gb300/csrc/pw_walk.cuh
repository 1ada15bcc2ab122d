// Walk building blocks shared by the batch kernels and the server kernel:
// the two ways of reading probe entries (evaluated per visit, or from a
// per-probe shared-memory table) and one replica of Algorithm 1's inner loop.
#pragma once
#include <stdint.h>

#include "pw_device.cuh"

namespace pw {

// The graph as a walk reads it.  A node record is {v, row_start(v), deg(v),
// bits of the FP32 reciprocal 1/deg(v)}; a step from record `cur` with random
// word w moves to neighbour floor(w deg / 2^32) of the row (Algorithm 1's
// uniform neighbour) and yields that neighbour's record.
//   FusedRecords: rec[e] is the record of col[e]; one 16-byte gather per step.
//     For graphs whose 16 B per entry sit comfortably in L2.
//   SplitRecords: a 4-byte col[e] gather, then the neighbour's record from the
//     n-entry node array; two dependent gathers into arrays 4x and nnz/n times
//     smaller.  For graphs whose fused records would spill out of L2.
struct FusedRecords {
  const int4* __restrict__ rec;
  const int4* __restrict__ node;
  __device__ __forceinline__ int4 start(int32_t v) const { return __ldg(node + v); }
  __device__ __forceinline__ int4 next(const int4& cur, uint32_t w) const {
    return __ldg(rec + ((uint32_t)cur.y + __umulhi(w, (uint32_t)cur.z)));
  }
};

struct SplitRecords {
  const int32_t* __restrict__ col;
  const int4* __restrict__ node;
  __device__ __forceinline__ int4 start(int32_t v) const { return __ldg(node + v); }
  __device__ __forceinline__ int4 next(const int4& cur, uint32_t w) const {
    const int32_t u = __ldg(col + ((uint32_t)cur.y + __umulhi(w, (uint32_t)cur.z)));
    return __ldg(node + u);
  }
};

// Probe entries evaluated on the fly (Section 3.3 generator): one cycle-walk
// queue for the two walks so a lane pays iter(s) + iter(t) Feistel passes.
struct ZOnTheFly {
  const Probe& pr;
  __device__ __forceinline__ void pair(uint32_t vs, uint32_t vt, int& zs, int& zt) const {
    uint32_t pis, pit;
    probe_pi_pair(pr, vs, vt, pis, pit);
    zs = probe_z_from_pi(pr, pis);
    zt = probe_z_from_pi(pr, pit);
  }
};

// Probe entries read from the block's table of z^(k) (built once per probe):
// one sign bit per node (set = negative) plus the ids of the r <= 2 nodes of
// the zero set, which the bits cannot express.
struct ZTable {
  const uint32_t* tab;
  uint32_t zero0, zero1;  // zero-set nodes, 0xFFFFFFFF when absent
  __device__ __forceinline__ int from_word(uint32_t word, uint32_t v) const {
    const int neg = (int)((word >> (v & 31u)) & 1u);
    return (v == zero0 || v == zero1) ? 0 : 1 - 2 * neg;
  }
  __device__ __forceinline__ int one(uint32_t v) const { return from_word(tab[v >> 5], v); }
  __device__ __forceinline__ void pair(uint32_t vs, uint32_t vt, int& zs, int& zt) const {
    zs = one(vs);
    zt = one(vt);
  }
};

// One replica: walks from s and t interleaved, a and b summed in FP32 in step
// order (Eq. hatphi-def), U_p = a - b.  The load of X_{i+1} is issued before
// the probe entry of X_i is evaluated so the gather latency overlaps the
// integer work.
template <bool DEBUG, class GR, class ZP>
__device__ __forceinline__ float walk_pair(const GR& gr, uint32_t* visits, uint32_t walk_tag, const ZP& zp, int32_t s,
                                           int32_t t, int32_t L, uint64_t seed, uint64_t pair) {
  int4 xs = gr.start(s), xt = gr.start(t);
  int zs, zt;
  zp.pair((uint32_t)xs.x, (uint32_t)xt.x, zs, zt);
  float a = signed_term(zs, (uint32_t)xs.w);
  float b = signed_term(zt, (uint32_t)xt.w);
  if (DEBUG) {
    atomicAdd(visits + xs.x, 1u);
    atomicAdd(visits + xt.x, 1u);
  }
  if (L == 0) return __fsub_rn(a, b);
  const uint64_t ws = 2 * pair, wt = ws + 1;
  // Philox key schedule computed inside each call: this path already holds the
  // probe's Feistel keys, so hoisting the ten round keys would cost registers
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  Philox4 rs = philox4x32_10((uint32_t)ws, (uint32_t)(ws >> 32), 0u, walk_tag, k0, k1);
  Philox4 rt = philox4x32_10((uint32_t)wt, (uint32_t)(wt >> 32), 0u, walk_tag, k0, k1);
  int4 ns = gr.next(xs, rs.y);
  int4 nt = gr.next(xt, rt.y);
  for (uint32_t blk = 0;; ++blk) {
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      if (w == 0 && blk == 0) continue;
      const uint32_t i = blk * 4u + (uint32_t)w;  // ns, nt hold X_i
      const bool more = i < (uint32_t)L;
      int4 ns2 = ns, nt2 = nt;
      if (more) {
        uint32_t wsw, wtw;
        if (w == 3) {
          rs = philox4x32_10((uint32_t)ws, (uint32_t)(ws >> 32), blk + 1u, walk_tag, k0, k1);
          rt = philox4x32_10((uint32_t)wt, (uint32_t)(wt >> 32), blk + 1u, walk_tag, k0, k1);
          wsw = rs.x;
          wtw = rt.x;
        } else {
          wsw = (w == 0) ? rs.y : (w == 1) ? rs.z : rs.w;
          wtw = (w == 0) ? rt.y : (w == 1) ? rt.z : rt.w;
        }
        ns2 = gr.next(ns, wsw);
        nt2 = gr.next(nt, wtw);
      }
      zp.pair((uint32_t)ns.x, (uint32_t)nt.x, zs, zt);
      a = __fadd_rn(a, signed_term(zs, (uint32_t)ns.w));
      b = __fadd_rn(b, signed_term(zt, (uint32_t)nt.w));
      if (DEBUG) {
        atomicAdd(visits + ns.x, 1u);
        atomicAdd(visits + nt.x, 1u);
      }
      if (!more) return __fsub_rn(a, b);
      ns = ns2;
      nt = nt2;
    }
  }
}

// Words of the per-probe table: one sign bit per node, then two words for
// the zero set.
__host__ __device__ __forceinline__ uint32_t table_words(uint32_t n) { return (n + 31u) / 32u + 2u; }

// One replica with probe entries from the shared-memory table, software
// pipelined: at step i the gather of X_{i+1} and the table read of X_i are
// issued, and the term of X_{i-1} (whose table word was read one step
// earlier) is added.  The additions keep step order, so the result equals
// walk_pair's bit for bit.
template <bool DEBUG, class GR>
__device__ __forceinline__ float walk_pair_table(const GR& gr, uint32_t* visits, uint32_t walk_tag, const ZTable& zt,
                                                 int32_t s, int32_t t, int32_t L, uint64_t seed, uint64_t pair) {
  const int4 xs = gr.start(s), xt = gr.start(t);
  float a = signed_term(zt.one((uint32_t)xs.x), (uint32_t)xs.w);
  float b = signed_term(zt.one((uint32_t)xt.x), (uint32_t)xt.w);
  if (DEBUG) {
    atomicAdd(visits + xs.x, 1u);
    atomicAdd(visits + xt.x, 1u);
  }
  if (L == 0) return __fsub_rn(a, b);
  const uint64_t ws = 2 * pair, wt = ws + 1;
  const PhiloxKeys keys = philox_keys(seed);
  Philox4 rs = philox4x32_10((uint32_t)ws, (uint32_t)(ws >> 32), 0u, walk_tag, keys);
  Philox4 rt = philox4x32_10((uint32_t)wt, (uint32_t)(wt >> 32), 0u, walk_tag, keys);
  int4 ns = gr.next(xs, rs.y);
  int4 nt = gr.next(xt, rt.y);
  // pending term: table word, node and reciprocal of the previous step's nodes
  uint32_t ps_word = 0, pt_word = 0, ps_v = 0xFFFFFFFFu, pt_v = 0xFFFFFFFFu, ps_inv = 0, pt_inv = 0;
  bool pending = false;
  for (uint32_t blk = 0;; ++blk) {
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      if (w == 0 && blk == 0) continue;
      const uint32_t i = blk * 4u + (uint32_t)w;  // ns, nt hold X_i
      const bool more = i < (uint32_t)L;
      int4 ns2 = ns, nt2 = nt;
      if (more) {
        uint32_t wsw, wtw;
        if (w == 3) {
          rs = philox4x32_10((uint32_t)ws, (uint32_t)(ws >> 32), blk + 1u, walk_tag, keys);
          rt = philox4x32_10((uint32_t)wt, (uint32_t)(wt >> 32), blk + 1u, walk_tag, keys);
          wsw = rs.x;
          wtw = rt.x;
        } else {
          wsw = (w == 0) ? rs.y : (w == 1) ? rs.z : rs.w;
          wtw = (w == 0) ? rt.y : (w == 1) ? rt.z : rt.w;
        }
        ns2 = gr.next(ns, wsw);
        nt2 = gr.next(nt, wtw);
      }
      const uint32_t cs_word = zt.tab[(uint32_t)ns.x >> 5], ct_word = zt.tab[(uint32_t)nt.x >> 5];
      if (pending) {
        a = __fadd_rn(a, signed_term(zt.from_word(ps_word, ps_v), ps_inv));
        b = __fadd_rn(b, signed_term(zt.from_word(pt_word, pt_v), pt_inv));
      }
      if (DEBUG) {
        atomicAdd(visits + ns.x, 1u);
        atomicAdd(visits + nt.x, 1u);
      }
      ps_word = cs_word;
      pt_word = ct_word;
      ps_v = (uint32_t)ns.x;
      pt_v = (uint32_t)nt.x;
      ps_inv = (uint32_t)ns.w;
      pt_inv = (uint32_t)nt.w;
      pending = true;
      if (!more) {
        a = __fadd_rn(a, signed_term(zt.from_word(ps_word, ps_v), ps_inv));
        b = __fadd_rn(b, signed_term(zt.from_word(pt_word, pt_v), pt_inv));
        return __fsub_rn(a, b);
      }
      ns = ns2;
      nt = nt2;
    }
  }
}

// z^(k) of every node into the shared-memory table: one Feistel cycle-walk
// per node.  Each thread owns whole 32-node words and runs a flat queue (one
// Feistel pass per iteration; it moves to its next node when a pass lands in
// [n]), so lanes stay busy even though cycle-walk lengths vary.  Nodes of the
// zero set (pi >= n - r) are listed in the two words after the bits.
__device__ __forceinline__ void build_probe_table(const Probe& pr, uint32_t* tab, uint32_t n) {
  const uint32_t nwords = (n + 31u) / 32u;
  uint32_t* zero = tab + nwords;
  if (threadIdx.x < 2) zero[threadIdx.x] = 0xFFFFFFFFu;
  __syncthreads();
  uint32_t w = threadIdx.x, v = w * 32u, x = v, acc = 0;
  while (w < nwords) {
    x = feistel_once(pr, x);
    if (x < n) {
      const int z = probe_z_from_pi(pr, x);
      if (z == 0) zero[x - pr.n_active] = v;
      acc |= (uint32_t)(z < 0) << (v & 31u);
      ++v;
      if ((v & 31u) == 0 || v >= n) {
        tab[w] = acc;
        acc = 0;
        w += blockDim.x;
        v = w * 32u;
      }
      x = v;
    }
  }
}

__device__ __forceinline__ ZTable table_reader(const uint32_t* tab, uint32_t n) {
  const uint32_t nwords = (n + 31u) / 32u;
  return ZTable{tab, tab[nwords], tab[nwords + 1]};
}

}  // namespace pw
