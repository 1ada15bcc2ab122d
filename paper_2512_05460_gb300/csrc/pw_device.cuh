// Device-side building blocks of the ProbeWalk walk kernel (sm_103a).
//
//  * Philox4x32-10 (Salmon et al., SC'11), written from its published round
//    and key-schedule definition.
//  * The stateless Paired-Sign Probe of Section 3.3: a cycle-walking Feistel
//    permutation pi_k on [n], zero set U = {v : pi_k(v) >= n - r}, pair id
//    floor(pi_k(v)/2), 2-universal sign hash h_k(u) = ((a_k u + b_k) mod p) mod 2
//    with p = 2^31 - 1, and z_v = (-1)^(h_k(pair) + pi_k(v)).
//  * Graph records: every CSR entry e of row v holds the neighbour u = col[e] as
//    {u, row_start(u), deg(u), bits of the FP32 reciprocal 1/deg(u)}, so one
//    16-byte gather per step yields everything the next step and the
//    accumulation need (Algorithm 1, inner loop).
#pragma once
#include <stdint.h>

namespace pw {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Counter word 3 tags of the independent streams.
constexpr uint32_t kTagWalk = 1u, kTagWalkPilot = 2u, kTagProbe = 3u, kTagProbePilot = 4u, kTagSeed = 0x5EEDu;
constexpr uint64_t kHashPrime = 2147483647ull;  // p = 2^31 - 1

struct Philox4 {
  uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

// Ten rounds; round r uses key + r * (W0, W1).
__host__ __device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                           uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = mulhi32(kPhiloxM0, c0), lo0 = kPhiloxM0 * c0;
    const uint32_t hi1 = mulhi32(kPhiloxM1, c2), lo1 = kPhiloxM1 * c2;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return Philox4{c0, c1, c2, c3};
}

// Round keys of one query key, hoisted out of the walk loop (the key schedule
// is the same for every counter of the query).
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};

__host__ __device__ __forceinline__ PhiloxKeys philox_keys(uint64_t seed) {
  PhiloxKeys K;
  uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    K.k0[r] = a;
    K.k1[r] = b;
    a += kPhiloxW0;
    b += kPhiloxW1;
  }
  return K;
}

__host__ __device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                           const PhiloxKeys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = mulhi32(kPhiloxM0, c0), lo0 = kPhiloxM0 * c0;
    const uint32_t hi1 = mulhi32(kPhiloxM1, c2), lo1 = kPhiloxM1 * c2;
    c0 = hi1 ^ c1 ^ K.k0[r];
    c1 = lo1;
    c2 = hi0 ^ c3 ^ K.k1[r];
    c3 = lo0;
  }
  return Philox4{c0, c1, c2, c3};
}

__host__ __device__ __forceinline__ Philox4 philox_seeded(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                                                           uint32_t c3) {
  return philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
}

__host__ __device__ __forceinline__ uint64_t default_seed(uint64_t global_seed, int64_t s, int64_t t, double eps,
                                                          int32_t L) {
  uint64_t eb;
#ifdef __CUDA_ARCH__
  eb = (uint64_t)__double_as_longlong(eps);
#else
  __builtin_memcpy(&eb, &eps, sizeof eb);
#endif
  const Philox4 o = philox_seeded(global_seed ^ eb, (uint32_t)s, (uint32_t)t, (uint32_t)L, kTagSeed);
  return (uint64_t)o.x | ((uint64_t)o.y << 32);
}

// Seed of truncation level L of a stabilized query: the first two words of the
// Philox block keyed by the query seed with counter (L, 0, 0, 0x57AB).
constexpr uint32_t kTagLevel = 0x57ABu;
__host__ __device__ __forceinline__ uint64_t level_seed(uint64_t seed, int32_t L) {
  const Philox4 o = philox_seeded(seed, (uint32_t)L, 0u, 0u, kTagLevel);
  return (uint64_t)o.x | ((uint64_t)o.y << 32);
}

// ---- Paired-Sign Probe -------------------------------------------------------

struct Probe {
  uint32_t n;        // nodes
  uint32_t n_active; // n - r
  uint32_t hi, lo;   // Feistel halves: domain 2^(hi + lo) >= n, hi = lo or lo + 1
  uint32_t rounds;   // 8, or 12 when hi + lo <= 4
  uint32_t a, b;     // hash parameters, a in [1, p-1], b in [0, p-1]
  uint32_t key[12];  // round keys
};

// Domain bits: the smallest b >= 2 with 2^b >= n, with b = 3 raised to 4 (the
// 2+1-bit network on [8] pairs visibly non-uniformly for n = 5, 6).  Odd b
// splits into a left half one bit wider than the right half.
__host__ __device__ __forceinline__ void feistel_bits(uint32_t n, uint32_t& hi, uint32_t& lo) {
  uint32_t b = 2;
  while (b < 31 && (1ull << b) < (uint64_t)n) ++b;
  if (b == 3) b = 4;
  hi = (b + 1) / 2;
  lo = b / 2;
}

// Probe k of the query keyed by `seed` on stream tag `tag`:
//   words of (k,0,0,tag): a = 1 + (w0|w1<<32) mod (p-1), b = (w2|w3<<32) mod p;
//   words of (k,1,j,tag), j = 0,1,2: round keys 4j..4j+3;
//   word 0 of (k,2,0,tag): parity coin r = 2 (bit 0) for even n, r = 1 for odd n.
__host__ __device__ __forceinline__ Probe make_probe(uint32_t n, uint64_t seed, uint32_t k, uint32_t tag) {
  Probe P;
  P.n = n;
  feistel_bits(n, P.hi, P.lo);
  P.rounds = (P.hi + P.lo <= 4) ? 12u : 8u;
  const Philox4 ab = philox_seeded(seed, k, 0u, 0u, tag);
  const uint64_t wa = (uint64_t)ab.x | ((uint64_t)ab.y << 32);
  const uint64_t wb = (uint64_t)ab.z | ((uint64_t)ab.w << 32);
  P.a = (uint32_t)(1 + wa % (kHashPrime - 1));
  P.b = (uint32_t)(wb % kHashPrime);
#pragma unroll
  for (uint32_t j = 0; j < 3; ++j) {
    const Philox4 kk = philox_seeded(seed, k, 1u, j, tag);
    P.key[4 * j + 0] = kk.x;
    P.key[4 * j + 1] = kk.y;
    P.key[4 * j + 2] = kk.z;
    P.key[4 * j + 3] = kk.w;
  }
  const Philox4 coin = philox_seeded(seed, k, 2u, 0u, tag);
  const uint32_t r = (n & 1u) ? 1u : 2u * (coin.x & 1u);
  P.n_active = n - r;
  return P;
}

// Round function: top h bits of ((x ^ key) * C1, xor-folded by 16, * C2).
__host__ __device__ __forceinline__ uint32_t feistel_f(uint32_t x, uint32_t key, uint32_t h) {
  uint32_t y = (x ^ key) * 0x9E3779B1u;
  y ^= y >> 16;
  y *= 0x85EBCA6Bu;
  return y >> (32u - h);
}

// One pass of the Feistel network on [2^hi] x [2^lo] (the generalised
// construction for such domains, Black and Rogaway 2002): a round maps
// (left, right) to (right, left ^ F(right)) with F as wide as the left half,
// so the halves trade widths every round; after the even round count the left
// half has hi bits again.
template <int ROUNDS>
__host__ __device__ __forceinline__ uint32_t feistel_pass(const Probe& P, uint32_t x) {
  uint32_t left = x >> P.lo, right = x & ((1u << P.lo) - 1u);
#pragma unroll
  for (int i = 0; i < ROUNDS; ++i) {
    const uint32_t f = feistel_f(right, P.key[i], (i & 1) ? P.lo : P.hi);
    const uint32_t nr = left ^ f;
    left = right;
    right = nr;
  }
  return (left << P.lo) | right;
}

__host__ __device__ __forceinline__ uint32_t feistel_once(const Probe& P, uint32_t x) {
  return P.rounds == 8u ? feistel_pass<8>(P, x) : feistel_pass<12>(P, x);
}

// pi_k(v) by cycle-walking the permutation of [2^(hi + lo)] back into [n].
__host__ __device__ __forceinline__ uint32_t probe_pi(const Probe& P, uint32_t v) {
  uint32_t x = v;
  do {
    x = feistel_once(P, x);
  } while (x >= P.n);
  return x;
}

// (a*u + b) mod (2^31 - 1) by Mersenne folding; a < 2^31, u < 2^31, b < 2^31.
__host__ __device__ __forceinline__ uint32_t hash_mod_p(uint32_t a, uint32_t u, uint32_t b) {
  const uint64_t t = (uint64_t)a * (uint64_t)u + (uint64_t)b;  // < 2^62 + 2^31
  uint64_t m = (t & kHashPrime) + (t >> 31);                    // < 2^32
  m = (m & kHashPrime) + (m >> 31);                             // <= 2^31
  if (m >= kHashPrime) m -= kHashPrime;
  return (uint32_t)m;
}

// z from pi: 0 on the zero set, else +1 when h(pair) + pi is even.
__host__ __device__ __forceinline__ int probe_z_from_pi(const Probe& P, uint32_t pi) {
  if (pi >= P.n_active) return 0;
  const uint32_t hv = hash_mod_p(P.a, pi >> 1, P.b) & 1u;
  return ((hv ^ pi) & 1u) ? -1 : 1;
}

__host__ __device__ __forceinline__ int probe_z(const Probe& P, uint32_t v) { return probe_z_from_pi(P, probe_pi(P, v)); }

// Term z/d in FP32 from the stored correctly rounded reciprocal: +-1/d is the
// IEEE quotient of +-1 by d and 0/d is +0.
__device__ __forceinline__ float signed_term(int z, uint32_t inv_bits) {
  return z == 0 ? 0.0f : __uint_as_float(z > 0 ? inv_bits : (inv_bits ^ 0x80000000u));
}

// z for two nodes at once: one cycle-walk queue, so a lane runs iter(s)+iter(t)
// Feistel passes instead of the warp paying max(iter(s)) + max(iter(t)).
__device__ __forceinline__ void probe_pi_pair(const Probe& P, uint32_t vs, uint32_t vt, uint32_t& pis,
                                              uint32_t& pit) {
  uint32_t x = vs;
  bool second = false;
  while (true) {
    x = feistel_once(P, x);
    if (x < P.n) {
      if (!second) {
        pis = x;
        second = true;
        x = vt;
      } else {
        pit = x;
        break;
      }
    }
  }
}

}  // namespace pw
