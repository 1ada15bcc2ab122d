// Exact per-probe sums S1 = sum_p U_p and S2 = sum_p U_p^2 over the R replicas
// of a probe (Algorithm 1, the inputs of Eq. Q-Ustat), rounded once to FP64.
//
// Range of a replica value: every term of a walk sum is +-fl(1/d) with
// 1 <= d < 2^31, a multiple of 2^-54; FP32 sums of multiples of 2^-54 stay
// multiples of 2^-54 (a result below 2^-30 in magnitude is exact, a larger
// one is a multiple of its own ulp >= 2^-54); and |a|, |b| <= L + 1 < 2^32.
// So U_p 2^54 and U_p^2 2^108 are integers below 2^87 and 2^174.  They are
// kept as base-2^32 digits in signed 64-bit accumulators (4 digits for S1, 7
// for S2; room for 2^32 replicas), added without rounding in any order, by
// registers, warp shuffles or 64-bit atomics alike, and rounded once to the
// nearest double, ties to even: the value of the exact sum.  Results do not
// depend on which warp, block or launch ran which replica.
#pragma once
#include <stdint.h>

namespace pw {

constexpr int kS1Digits = 4, kS2Digits = 7, kSumDigits = kS1Digits + kS2Digits;
constexpr int kS1Scale = 54, kS2Scale = 108;  // bit 0 of digit 0 weighs 2^-54 (S1), 2^-108 (S2)

struct SumDigits {
  long long d[kSumDigits];
};

__device__ __forceinline__ void sum_clear(SumDigits& a) {
#pragma unroll
  for (int j = 0; j < kSumDigits; ++j) a.d[j] = 0;
}

// d[0..N) += (neg ? -1 : 1) * v * 2^off, for v < 2^48; the three 32-bit digits
// that v spans are selected without indexing registers dynamically.
template <int N>
__device__ __forceinline__ void digits_add(long long* d, unsigned long long v, int off, bool neg) {
  const int q = off >> 5, r = off & 31;
  const unsigned long long lo = v << r;
  const unsigned long long hi = r ? (v >> (64 - r)) : 0ull;
  long long x0 = (long long)(lo & 0xFFFFFFFFull), x1 = (long long)(lo >> 32), x2 = (long long)hi;
  if (neg) {
    x0 = -x0;
    x1 = -x1;
    x2 = -x2;
  }
#pragma unroll
  for (int j = 0; j < N; ++j) d[j] += (j == q) ? x0 : (j == q + 1) ? x1 : (j == q + 2) ? x2 : 0ll;
}

// Adds one replica value U (see the range argument above).
__device__ __forceinline__ void sum_add(SumDigits& a, float U) {
  const uint32_t bits = __float_as_uint(U);
  const uint32_t ex = (bits >> 23) & 0xFFu;
  if (ex == 0u) return;  // zero: nonzero replica values are at least 2^-54, never subnormal
  unsigned long long M = (bits & 0x7FFFFFu) | 0x800000u;
  int sh = (int)ex - 150 + kS1Scale;  // U = M 2^(ex - 150), so U 2^54 = M 2^sh
  if (sh < 0) {                       // exact: U is a multiple of 2^-54
    M >>= -sh;
    sh = 0;
  }
  digits_add<kS1Digits>(a.d, M, sh, (bits >> 31) != 0u);
  digits_add<kS2Digits>(a.d + kS1Digits, M * M, 2 * sh, false);
}

__device__ __forceinline__ void sum_warp_reduce(SumDigits& a) {
#pragma unroll
  for (int j = 0; j < kSumDigits; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a.d[j] += __shfl_xor_sync(0xffffffffu, a.d[j], o);
}

// atomics on 64-bit words add modulo 2^64, which is exact for signed digit sums
__device__ __forceinline__ void sum_atomic_add(unsigned long long* dst, const SumDigits& a) {
#pragma unroll
  for (int j = 0; j < kSumDigits; ++j)
    if (a.d[j] != 0) atomicAdd(dst + j, (unsigned long long)a.d[j]);
}

// The value of digits in[0..N) (bit 0 weighs 2^-scale) rounded to the nearest
// double, ties to even.
template <int N>
__device__ __forceinline__ double digits_round(const long long* in, int scale) {
  long long d[N];
#pragma unroll
  for (int j = 0; j < N; ++j) d[j] = in[j];
#pragma unroll
  for (int j = 0; j + 1 < N; ++j) {  // digits below the top into [0, 2^32)
    const long long c = d[j] >> 32;
    d[j] -= c * 4294967296ll;
    d[j + 1] += c;
  }
  const bool neg = d[N - 1] < 0;
  if (neg) {
#pragma unroll
    for (int j = 0; j < N; ++j) d[j] = -d[j];
#pragma unroll
    for (int j = 0; j + 1 < N; ++j) {
      const long long c = d[j] >> 32;
      d[j] -= c * 4294967296ll;
      d[j + 1] += c;
    }
  }
  int top = -1;
#pragma unroll
  for (int j = 0; j < N; ++j)
    if (d[j] != 0) top = j;
  if (top < 0) return 0.0;
  // the three leading digits as one 96-bit integer W; lower digits only as a sticky bit
  unsigned long long w2 = 0, w1 = 0, w0 = 0;
  bool sticky = false;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const unsigned long long v = (unsigned long long)d[j];
    if (j == top) w2 = v;
    if (j == top - 1) w1 = v;
    if (j == top - 2) w0 = v;
    if (j < top - 2 && v != 0ull) sticky = true;
  }
  const unsigned __int128 W = ((unsigned __int128)w2 << 64) | ((unsigned __int128)w1 << 32) | w0;
  const int bits = 128 - __clzll((long long)w2);  // w2 != 0: bits in [65, 96]
  const int drop = bits - 53;
  unsigned long long mant = (unsigned long long)(W >> drop);
  const unsigned __int128 rem = W - ((unsigned __int128)mant << drop);
  const unsigned __int128 half = (unsigned __int128)1 << (drop - 1);
  if (rem > half || (rem == half && (sticky || (mant & 1ull)))) mant += 1ull;
  const int e = 32 * (top - 2) + drop - scale;  // within [-160, 75]: a normal power of two
  const double p2 = __longlong_as_double((long long)(e + 1023) << 52);
  const double v = __dmul_rn(__ull2double_rn(mant), p2);  // mant <= 2^53: exact
  return neg ? -v : v;
}

__device__ __forceinline__ void sum_round(const long long* d, double& S1, double& S2) {
  S1 = digits_round<kS1Digits>(d, kS1Scale);
  S2 = digits_round<kS2Digits>(d + kS1Digits, kS2Scale);
}

}  // namespace pw
