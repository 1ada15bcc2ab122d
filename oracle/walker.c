/*
 * ProbeWalk ORACLE: a plain, serial CPU restatement of the estimator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * constant generator with the CUDA path: every routine below is written from
 * the paper (arXiv 2512.05460) and from the published Philox definition.
 *
 * What it computes, in the paper's order and notation:
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): the counter-based
 *     generator that both sides implement from its published definition.
 *   - The stateless Paired-Sign Probe generator of Section 3.3: a Feistel
 *     permutation pi_k on [n] (cycle-walking), the zero set U = {i : pi_k(i) >=
 *     n - r}, pair ids floor(pi_k(i)/2), the 2-universal sign hash
 *     h_k(u) = ((a_k u + b_k) mod p) mod 2, and z_i = (-1)^(h_k(pair(i)) + pi_k(i)).
 *   - Algorithm 1: for every probe k and replica p, two independent walks of
 *     length L from s and t; a and b accumulate z_X / d_X in FP32 in step order
 *     (Eq. hatphi-def); U_p = a - b; S1 = sum U_p, S2 = sum U_p^2 (exact sums
 *     rounded once to FP64); Q_R = (S1^2 - S2) / (R(R-1)) (Eq. Q-Ustat); block means over
 *     G contiguous blocks of B probes and their median (Eq. final-estimator).
 *   - The budget of Algorithm 1's parameter line (Eqs. B-value, G-value,
 *     R-value, K-value) and the readings used where the paper leaves the
 *     experimental budget open (THEORY, SCALED, FIXED, PILOT).
 *
 * The routines are deliberately unoptimised: the Philox block is recomputed
 * for every step, z is recomputed for every visit, sums over probes run in
 * index order.
 * Build with -ffp-contract=off (no fused multiply-add) and without fast-math.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------------
 * Philox4x32-10 from its published definition: ten rounds of the S-box
 * (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
 * c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), with the Weyl key schedule
 * k0 += W0, k1 += W1 between rounds.
 * ------------------------------------------------------------------------- */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += ORC_PHILOX_W0;
      k1 += ORC_PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_seeded(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                          uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox(ctr, key, out);
}

/* Stream tags (counter word 3): main walks, pilot walks, main probes, pilot probes. */
#define ORC_TAG_WALK 1u
#define ORC_TAG_WALK_PILOT 2u
#define ORC_TAG_PROBE 3u
#define ORC_TAG_PROBE_PILOT 4u
#define ORC_TAG_SEED 0x5EEDu

/* Default per-query seed: a Philox block keyed by the global seed mixed with
 * the bits of eps, over the counter (s, t, L, tag). */
uint64_t orc_default_seed(uint64_t global_seed, int64_t s, int64_t t, double eps, int32_t L) {
  uint64_t eb;
  memcpy(&eb, &eps, sizeof eb);
  uint64_t key = global_seed ^ eb;
  uint32_t out[4];
  philox_seeded(key, (uint32_t)s, (uint32_t)t, (uint32_t)L, ORC_TAG_SEED, out);
  return (uint64_t)out[0] | ((uint64_t)out[1] << 32);
}

/* Seed of truncation level L of a stabilized query: Philox block keyed by the
 * query seed over the counter (L, 0, 0, 0x57AB), first two words. */
uint64_t orc_level_seed(uint64_t seed, int32_t L) {
  uint32_t out[4];
  philox_seeded(seed, (uint32_t)L, 0u, 0u, 0x57ABu, out);
  return (uint64_t)out[0] | ((uint64_t)out[1] << 32);
}

/* ---------------------------------------------------------------------------
 * Paired-Sign Probe, stateless generator (Section 3.3).
 * ------------------------------------------------------------------------- */
#define ORC_PRIME 2147483647ull /* p = 2^31 - 1 > floor(n/2) for every n < 2^32 */

/* Feistel rounds: the probe needs a (near-)uniform random matching for
 * E[z z^T] = H (Definition 3.1, Lemma 3.2).  Four rounds leave the pairing
 * probability of inputs such as (x, x^1) 50-70% too high on domains of 16
 * elements and ~17% too high on 256; eight rounds (twelve when the domain has
 * at most 16 elements) bring every entry of E[z z^T] - H to sampling noise. */
#define ORC_FEISTEL_MAX_ROUNDS 12

typedef struct {
  uint64_t n;
  uint32_t hi_bits;     /* Feistel halves: domain 2^(hi_bits + lo_bits) >= n, */
  uint32_t lo_bits;     /* hi_bits = lo_bits or lo_bits + 1 */
  uint32_t rounds;
  uint32_t round_key[ORC_FEISTEL_MAX_ROUNDS];
  uint64_t a, b;        /* hash parameters a_k in [1, p-1], b_k in [0, p-1] */
  uint32_t r;           /* parity parameter: number of zero entries */
} orc_probe;

static uint32_t feistel_round_fn(uint32_t x, uint32_t key, uint32_t h) {
  uint32_t y = (x ^ key) * 0x9E3779B1u;
  y ^= y >> 16;
  y *= 0x85EBCA6Bu;
  return y >> (32u - h);
}

/* One pass of the Feistel network on [2^(hi + lo)] whose halves may differ by
 * one bit (the generalised Feistel construction on a domain of the form
 * [2^hi] x [2^lo], Black and Rogaway 2002): the left half has `wl` bits and
 * the right half `wr`; a round replaces (left, right) by (right, left XOR
 * F(right)), F giving `wl` bits, so the two widths trade places every round
 * and are back to (hi, lo) after the even number of rounds used here. */
static uint64_t feistel_once(const orc_probe* P, uint64_t x) {
  uint32_t wl = P->hi_bits, wr = P->lo_bits;
  uint32_t left = (uint32_t)(x >> wr);
  uint32_t right = (uint32_t)(x & (((uint64_t)1 << wr) - 1u));
  for (uint32_t i = 0; i < P->rounds; ++i) {
    uint32_t f = feistel_round_fn(right, P->round_key[i], wl);
    uint32_t new_right = left ^ f;
    uint32_t w = wl;
    left = right;
    right = new_right;
    wl = wr;
    wr = w;
  }
  return ((uint64_t)left << wr) | right;
}

/* pi_k(i): cycle-walk the Feistel permutation of [2^(hi + lo)] until it lands in [n]. */
uint64_t orc_probe_pi(const orc_probe* P, uint64_t i) {
  uint64_t x = i;
  do {
    x = feistel_once(P, x);
  } while (x >= P->n);
  return x;
}

static void probe_setup(orc_probe* P, uint64_t n, uint64_t seed, uint32_t k, uint32_t tag) {
  uint32_t w[4];
  P->n = n;
  /* smallest b >= 2 with 2^b >= n, except that b = 3 becomes 4 (on [8] the
   * 2+1-bit network leaves the matching visibly non-uniform for n = 5, 6);
   * halves of ceil(b/2) (left) and floor(b/2) (right) bits */
  uint32_t b = 2;
  while (b < 62 && ((uint64_t)1 << b) < n) b += 1;
  if (b == 3) b = 4;
  P->hi_bits = (b + 1) / 2;
  P->lo_bits = b / 2;
  P->rounds = (b <= 4) ? 12u : 8u;
  philox_seeded(seed, k, 0u, 0u, tag, w);
  uint64_t wa = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
  uint64_t wb = (uint64_t)w[2] | ((uint64_t)w[3] << 32);
  P->a = 1 + wa % (ORC_PRIME - 1);
  P->b = wb % ORC_PRIME;
  /* round keys: words of the blocks with counter (k, 1, j, tag), j = 0, 1, 2 */
  for (uint32_t j = 0; j < 3; ++j) {
    philox_seeded(seed, k, 1u, j, tag, w);
    for (int i = 0; i < 4; ++i) P->round_key[4 * j + i] = w[i];
  }
  philox_seeded(seed, k, 2u, 0u, tag, w);
  if (n % 2 == 1)
    P->r = 1;
  else
    P->r = 2u * (w[0] & 1u);
}

/* z_i^(k) in {-1, 0, +1}. */
static int probe_entry(const orc_probe* P, uint64_t i) {
  uint64_t pi = orc_probe_pi(P, i);
  if (pi >= P->n - P->r) return 0; /* i in U */
  uint64_t pair = pi / 2;
  uint64_t hv = ((P->a * pair + P->b) % ORC_PRIME) % 2;
  return ((hv + pi) % 2 == 0) ? 1 : -1;
}

/* Whole probe vector (tests only): z[0..n) and optionally pi[0..n). */
int orc_probe_vector(uint64_t n, uint64_t seed, uint32_t k, uint32_t tag, int8_t* z, uint64_t* pi) {
  if (n < 2) return -1;
  orc_probe P;
  probe_setup(&P, n, seed, k, tag);
  for (uint64_t i = 0; i < n; ++i) {
    if (z) z[i] = (int8_t)probe_entry(&P, i);
    if (pi) pi[i] = orc_probe_pi(&P, i);
  }
  return (int)P.r;
}

/* ---------------------------------------------------------------------------
 * Walks (Algorithm 1, inner loop).
 * Step i >= 1 of walk `walk_id` draws word (i mod 4) of the Philox block with
 * counter (walk_id lo, walk_id hi, floor(i/4), tag) under the query key, and
 * moves to neighbour index floor(word * d / 2^32) of the current node.
 * ------------------------------------------------------------------------- */
static uint32_t walk_word(uint64_t seed, uint64_t walk_id, uint32_t step, uint32_t tag) {
  uint32_t w[4];
  philox_seeded(seed, (uint32_t)walk_id, (uint32_t)(walk_id >> 32), step / 4u, tag, w);
  return w[step % 4u];
}

static int64_t next_node(const int64_t* row_ptr, const int32_t* col_idx, int64_t v, uint32_t word) {
  uint64_t d = (uint64_t)(row_ptr[v + 1] - row_ptr[v]);
  uint64_t j = ((uint64_t)word * d) >> 32;
  return col_idx[row_ptr[v] + (int64_t)j];
}

/* Trajectory X_0..X_L of one walk (tests only). */
int orc_walk(const int64_t* row_ptr, const int32_t* col_idx, int64_t start, int32_t L, uint64_t seed,
             uint64_t walk_id, uint32_t tag, int64_t* traj) {
  int64_t v = start;
  traj[0] = v;
  for (int32_t i = 1; i <= L; ++i) {
    v = next_node(row_ptr, col_idx, v, walk_word(seed, walk_id, (uint32_t)i, tag));
    traj[i] = v;
  }
  return 0;
}

/* One replica of the estimator: U_p = a - b with a, b summed in FP32 in step order. */
static float walk_pair(const int64_t* row_ptr, const int32_t* col_idx, const orc_probe* P, int64_t s,
                       int64_t t, int32_t L, uint64_t seed, uint64_t pair_index, uint32_t tag,
                       uint32_t* visits) {
  int64_t x = s, y = t;
  float dx = (float)(row_ptr[x + 1] - row_ptr[x]);
  float dy = (float)(row_ptr[y + 1] - row_ptr[y]);
  float a = (float)probe_entry(P, (uint64_t)x) / dx;
  float b = (float)probe_entry(P, (uint64_t)y) / dy;
  if (visits) { visits[x]++; visits[y]++; }
  uint64_t wid_s = 2 * pair_index, wid_t = 2 * pair_index + 1;
  for (int32_t i = 1; i <= L; ++i) {
    x = next_node(row_ptr, col_idx, x, walk_word(seed, wid_s, (uint32_t)i, tag));
    y = next_node(row_ptr, col_idx, y, walk_word(seed, wid_t, (uint32_t)i, tag));
    dx = (float)(row_ptr[x + 1] - row_ptr[x]);
    dy = (float)(row_ptr[y + 1] - row_ptr[y]);
    a = a + (float)probe_entry(P, (uint64_t)x) / dx;
    b = b + (float)probe_entry(P, (uint64_t)y) / dy;
    if (visits) { visits[x]++; visits[y]++; }
  }
  return a - b;
}

/* ---------------------------------------------------------------------------
 * Exact sums.  Algorithm 1 defines S1 = sum_p U_p and S2 = sum_p U_p^2 over the
 * R replicas of a probe.  The U_p are FP32 values, so U_p and U_p^2 are exact
 * doubles; they are added without any rounding into a long fixed-point
 * accumulator that spans every double (base-2^32 digits held in 64-bit
 * integers, so carries wait until the end), and the total is rounded once to
 * the nearest double, ties to even.  S1 and S2 are therefore the correctly
 * rounded values of the exact sums, independent of the order of the replicas.
 * ------------------------------------------------------------------------- */
#define ORC_ACC_DIGITS 72
#define ORC_ACC_LOW_EXP (-1152) /* weight of bit 0 of digit 0 */

typedef struct {
  int64_t d[ORC_ACC_DIGITS];
} orc_exact_sum;

static void exact_clear(orc_exact_sum* A) { memset(A, 0, sizeof *A); }

static void exact_add(orc_exact_sum* A, double x) {
  if (x == 0.0) return;
  int e;
  double m = frexp(fabs(x), &e);              /* |x| = m 2^e, m in [0.5, 1) */
  uint64_t M = (uint64_t)ldexp(m, 53);        /* |x| = M 2^(e - 53), exactly */
  int pos = e - 53 - ORC_ACC_LOW_EXP;         /* >= 26 for the smallest subnormal */
  int q = pos / 32, r = pos % 32;
  unsigned __int128 w = (unsigned __int128)M << r;
  int64_t sign = x < 0 ? -1 : 1;
  A->d[q] += sign * (int64_t)(uint32_t)w;
  A->d[q + 1] += sign * (int64_t)(uint32_t)(w >> 32);
  A->d[q + 2] += sign * (int64_t)(uint32_t)(w >> 64);
}

/* Bring every digit but the last into [0, 2^32), carrying upwards. */
static void exact_carry(int64_t* d) {
  for (int i = 0; i + 1 < ORC_ACC_DIGITS; ++i) {
    int64_t c = d[i] >> 32; /* floor(d / 2^32) */
    d[i] -= c * ((int64_t)1 << 32);
    d[i + 1] += c;
  }
}

/* The exact sum rounded to the nearest double, ties to even.  (Nonzero sums
 * of FP32 values and of their squares are at least 2^-298 in magnitude, far
 * from the subnormal range, so the final scaling by a power of two is exact.) */
static double exact_round(const orc_exact_sum* A) {
  int64_t d[ORC_ACC_DIGITS];
  memcpy(d, A->d, sizeof d);
  exact_carry(d);
  int neg = d[ORC_ACC_DIGITS - 1] < 0;
  if (neg) {
    for (int i = 0; i < ORC_ACC_DIGITS; ++i) d[i] = -d[i];
    exact_carry(d);
  }
  int top = ORC_ACC_DIGITS - 1;
  while (top >= 0 && d[top] == 0) --top;
  if (top < 0) return 0.0;
  /* the three most significant digits as one integer, the rest as a sticky bit */
  unsigned __int128 W = 0;
  for (int i = top; i >= top - 2; --i) W = (W << 32) | (uint64_t)(i >= 0 ? d[i] : 0);
  int sticky = 0;
  for (int i = top - 3; i >= 0; --i) sticky |= d[i] != 0;
  int bits = 0;
  for (unsigned __int128 v = W; v; v >>= 1) ++bits;
  int drop = bits - 53; /* >= 12: the top digit is nonzero */
  unsigned __int128 mant = W >> drop;
  unsigned __int128 rem = W - (mant << drop);
  unsigned __int128 half = (unsigned __int128)1 << (drop - 1);
  if (rem > half || (rem == half && (sticky || (mant & 1)))) mant += 1;
  double v = ldexp((double)(uint64_t)mant, ORC_ACC_LOW_EXP + 32 * (top - 2) + drop);
  return neg ? -v : v;
}

/* Tests: the exact sum of n FP32 values (square != 0: of their squares). */
double orc_exact_sum_f32(const float* u, int64_t n, int square) {
  orc_exact_sum A;
  exact_clear(&A);
  for (int64_t i = 0; i < n; ++i) {
    double x = (double)u[i];
    exact_add(&A, square ? x * x : x);
  }
  return exact_round(&A);
}

/* ---------------------------------------------------------------------------
 * Budget (Algorithm 1 line 1; Eqs. B-value, G-value, R-value, K-value).
 * ------------------------------------------------------------------------- */
enum { ORC_PILOT = 0, ORC_THEORY = 1, ORC_SCALED = 2, ORC_FIXED = 3, ORC_ADAPTIVE = 4 };

typedef struct {
  int32_t mode;
  int32_t K0, R0;     /* pilot probes and replicas */
  double delta, c_B, c_R;
  uint64_t B, G, R;   /* FIXED mode */
  uint64_t R_max;
  double z;           /* ADAPTIVE: normal quantile of the stopping rule */
  double cap;         /* ADAPTIVE: the most probes per block, as a multiple of PILOT's B */
} orc_budget_cfg;

/* ceil that forgives the last-place error of expressions such as 448/0.1^2 */
static double ceil_tol(double x) { return ceil(x * (1.0 - 1e-12)); }

typedef struct {
  uint64_t B, G, K, R;
  double sigma2_hat, q_bar, theta_hat; /* PILOT diagnostics */
  uint64_t B1;                         /* ADAPTIVE: probes per block of the first stage */
} orc_budget;

static void fill_defaults(const orc_budget_cfg* in, orc_budget_cfg* c) {
  *c = *in;
  if (!(c->delta > 0)) c->delta = 0.01;
  if (c->K0 <= 0) c->K0 = 64;
  if (c->R0 <= 1) c->R0 = 32;
  if (c->R_max == 0) c->R_max = 4096;
  if (!(c->c_R > 0)) c->c_R = 1.0;
  /* PILOT's c_B default (0.5) is the calibrated reading of the experimental
   * budget, which the paper leaves open; SCALED scales Eq. B-value by c_B = 1. */
  if (!(c->c_B > 0)) c->c_B = (c->mode == ORC_PILOT || c->mode == ORC_ADAPTIVE) ? 0.5 : 1.0;
  /* ADAPTIVE defaults, calibrated on 1024 queries per workload: z = 3 with
   * B allowed up to twice PILOT's */
  if (!(c->z > 0)) c->z = 3.0;
  if (!(c->cap > 0)) c->cap = 2.0;
}

/* R of Eq. R-value before the ceiling. */
static double r_theory_raw(double eps, int32_t L, double d_min, double ds, double dt) {
  double inv = 1.0 / ds + 1.0 / dt;
  return 128.0 * (double)(L + 1) * (double)(L + 1) / (d_min * d_min * (1.0 - eps / 2.0) * inv * inv);
}

/* Q_R for one probe: S1 and S2 are the exact sums over the replicas, rounded once. */
static double probe_q(const int64_t* row_ptr, const int32_t* col_idx, uint64_t n, int64_t s, int64_t t,
                      int32_t L, uint64_t seed, uint32_t k, uint64_t R, uint32_t probe_tag,
                      uint32_t walk_tag, float* u_out, double* s1_out, double* s2_out, uint32_t* visits) {
  orc_probe P;
  probe_setup(&P, n, seed, k, probe_tag);
  orc_exact_sum A1, A2;
  exact_clear(&A1);
  exact_clear(&A2);
  for (uint64_t p = 0; p < R; ++p) {
    float U = walk_pair(row_ptr, col_idx, &P, s, t, L, seed, (uint64_t)k * R + p, walk_tag, visits);
    if (u_out) u_out[p] = U;
    double u = (double)U;
    exact_add(&A1, u);
    exact_add(&A2, u * u); /* exact: the square of an FP32 value fits a double */
  }
  double S1 = exact_round(&A1), S2 = exact_round(&A2);
  if (s1_out) *s1_out = S1;
  if (s2_out) *s2_out = S2;
  double Rd = (double)R;
  return (S1 * S1 - S2) / (Rd * (Rd - 1.0));
}

static int compute_budget(const int64_t* row_ptr, const int32_t* col_idx, uint64_t n, int64_t s, int64_t t,
                          double eps, int32_t L, uint64_t seed, const orc_budget_cfg* cfg_in, orc_budget* out) {
  orc_budget_cfg c;
  fill_defaults(cfg_in, &c);
  memset(out, 0, sizeof *out);
  double ds = (double)(row_ptr[s + 1] - row_ptr[s]);
  double dt = (double)(row_ptr[t + 1] - row_ptr[t]);
  double d_min = 1e300;
  for (uint64_t v = 0; v < n; ++v) {
    double d = (double)(row_ptr[v + 1] - row_ptr[v]);
    if (d < d_min) d_min = d;
  }
  uint64_t G = (uint64_t)ceil_tol(8.0 * log(1.0 / c.delta));
  if (G < 1) G = 1;
  switch (c.mode) {
    case ORC_THEORY: {
      out->B = (uint64_t)ceil_tol(448.0 / (eps * eps));
      out->G = G;
      double R = ceil_tol(r_theory_raw(eps, L, d_min, ds, dt));
      out->R = R < 2.0 ? 2 : (uint64_t)R;
      break;
    }
    case ORC_SCALED: {
      double B = ceil_tol(c.c_B * 448.0 / (eps * eps));
      out->B = B < 1.0 ? 1 : (uint64_t)B;
      out->G = G;
      double R = ceil_tol(c.c_R * r_theory_raw(eps, L, d_min, ds, dt));
      if (R < 2.0) R = 2.0;
      if (R > (double)c.R_max) R = (double)c.R_max;
      out->R = (uint64_t)R;
      break;
    }
    case ORC_FIXED: {
      if (c.B < 1 || c.G < 1 || c.R < 2) return -1;
      out->B = c.B;
      out->G = c.G;
      out->R = c.R;
      break;
    }
    case ORC_PILOT:
    case ORC_ADAPTIVE: {
      double B = ceil_tol(c.c_B / (eps * eps));
      out->B = B < 1.0 ? 1 : (uint64_t)B;
      out->G = G;
      /* Pilot: K0 probes x R0 replicas on the reserved pilot streams.  The
       * paper's sufficient condition R >= 4 sigma^2 / theta (Lemma 3.7) is
       * evaluated with the pooled within-probe variance of U_p and the mean
       * pilot Q, floored by theta_0 of the proof of Theorem 3.8. */
      double sum_var = 0.0, sum_q = 0.0;
      double R0 = (double)c.R0;
      for (int32_t k = 0; k < c.K0; ++k) {
        double S1, S2;
        double q = probe_q(row_ptr, col_idx, n, s, t, L, seed, (uint32_t)k, (uint64_t)c.R0, ORC_TAG_PROBE_PILOT,
                           ORC_TAG_WALK_PILOT, NULL, &S1, &S2, NULL);
        sum_var = sum_var + (S2 - S1 * S1 / R0) / (R0 - 1.0);
        sum_q = sum_q + q;
      }
      double sigma2 = sum_var / (double)c.K0;
      double q_bar = sum_q / (double)c.K0;
      double inv = 1.0 / ds + 1.0 / dt;
      double theta0 = (1.0 / 8.0) * (1.0 - eps / 2.0) * inv * inv;
      double theta = q_bar > theta0 ? q_bar : theta0;
      double R = ceil_tol(c.c_R * 4.0 * sigma2 / theta);
      if (R < 2.0) R = 2.0;
      R = 32.0 * ceil(R / 32.0); /* whole warps of replicas */
      if (R > (double)c.R_max) R = (double)c.R_max;
      out->R = (uint64_t)R;
      out->sigma2_hat = sigma2;
      out->q_bar = q_bar;
      out->theta_hat = theta;
      out->B1 = (out->B + 3) / 4; /* ceil(B / 4) */
      if (c.mode == ORC_ADAPTIVE) out->B = (uint64_t)ceil_tol(c.cap * (double)out->B); /* the largest B */
      break;
    }
    default:
      return -1;
  }
  out->K = out->B * out->G;
  return 0;
}

/* ---------------------------------------------------------------------------
 * ADAPTIVE budget: B per query from its own variance.  The median of G block means of
 * B probes each has, for block means that are near normal, a standard error
 * of sqrt(pi/2) sd(Q) / sqrt(G B) (the asymptotic variance of a sample median
 * is pi/2 times that of the mean).  After a first stage of B1 = ceil(B_P/4)
 * probes per block (B_P: PILOT's B), sd(Q) and the mean of Q are estimated
 * from those G B1 values, and the query keeps the smallest B at which z
 * standard errors fit in eps times the estimated distance:
 *     B* = ceil( (pi/2) z^2 s^2 / (G eps^2 theta^2) ),  B1 <= B* <= cap B_P,
 * theta = max(mean Q, theta_0) with theta_0 of the PILOT budget.  The
 * second stage runs probes G B1 .. G B* - 1 and the estimate is the median of
 * the G contiguous blocks of B* probes (Eq. final-estimator).
 * ------------------------------------------------------------------------- */
static uint64_t adaptive_B(const double* q, uint64_t B1, uint64_t B, uint64_t G, double eps, double z, double ds,
                           double dt) {
  uint64_t K1 = G * B1;
  double sum = 0.0;
  for (uint64_t k = 0; k < K1; ++k) sum = sum + q[k];
  double mean = sum / (double)K1;
  double ss = 0.0;
  for (uint64_t k = 0; k < K1; ++k) ss = ss + (q[k] - mean) * (q[k] - mean);
  double s2 = K1 > 1 ? ss / (double)(K1 - 1) : 0.0;
  double inv = 1.0 / ds + 1.0 / dt;
  double theta0 = (1.0 / 8.0) * (1.0 - eps / 2.0) * inv * inv;
  double theta = mean > theta0 ? mean : theta0;
  double x = 1.5707963267948966 * z * z * s2; /* (pi/2) z^2 s^2 */
  x = x / (theta * theta);
  x = x / ((double)G * eps * eps);
  double Bs = ceil_tol(x);
  if (Bs < (double)B1) Bs = (double)B1;
  if (Bs > (double)B) Bs = (double)B;
  return (uint64_t)Bs;
}

/* ---------------------------------------------------------------------------
 * Median-of-means (Eq. final-estimator).
 * ------------------------------------------------------------------------- */
static int cmp_double(const void* x, const void* y) {
  double a = *(const double*)x, b = *(const double*)y;
  return (a > b) - (a < b);
}

static double median_of_means(const double* q, uint64_t B, uint64_t G) {
  double* means = (double*)malloc(sizeof(double) * G);
  for (uint64_t g = 0; g < G; ++g) {
    double sum = 0.0;
    for (uint64_t k = g * B; k < (g + 1) * B; ++k) sum = sum + q[k];
    means[g] = sum / (double)B;
  }
  qsort(means, G, sizeof(double), cmp_double);
  double med = (G % 2 == 1) ? means[G / 2] : (means[G / 2 - 1] + means[G / 2]) / 2.0;
  free(means);
  return med;
}

/* ---------------------------------------------------------------------------
 * One query: Algorithm 1 from the budget to the median.
 *   budget_out (nullable): B, G, K, R.   pilot_out (nullable): sigma2_hat,
 *   q_bar, theta_hat.   q_out (nullable): K values of Q_R.   u_out (nullable):
 *   K*R values of U_p, probe-major.   visits (nullable, n counters): visits of
 *   every main walk, X_0 included.
 * Returns 0, or -1 on invalid arguments.
 * ------------------------------------------------------------------------- */
int orc_query(const int64_t* row_ptr, const int32_t* col_idx, int64_t n, int64_t s, int64_t t, double eps,
              int32_t L, uint64_t seed, const orc_budget_cfg* cfg, double* beta_hat, uint64_t* budget_out,
              double* pilot_out, double* q_out, float* u_out, uint32_t* visits) {
  if (n < 2 || s < 0 || t < 0 || s >= n || t >= n || L < 0 || !(eps > 0.0 && eps < 1.0)) return -1;
  if (s == t) {
    *beta_hat = 0.0;
    if (budget_out) memset(budget_out, 0, 4 * sizeof(uint64_t));
    return 0;
  }
  orc_budget bud;
  if (compute_budget(row_ptr, col_idx, (uint64_t)n, s, t, eps, L, seed, cfg, &bud) != 0) return -1;
  if (budget_out) {
    budget_out[0] = bud.B; budget_out[1] = bud.G; budget_out[2] = bud.K; budget_out[3] = bud.R;
  }
  if (pilot_out) {
    pilot_out[0] = bud.sigma2_hat; pilot_out[1] = bud.q_bar; pilot_out[2] = bud.theta_hat;
  }
  double* q = q_out ? q_out : (double*)calloc(bud.K ? bud.K : 1, sizeof(double));
  uint64_t K = bud.K, B = bud.B;
  if (cfg->mode == ORC_ADAPTIVE) { /* first stage, then the stopping rule */
    orc_budget_cfg c;
    fill_defaults(cfg, &c);
    uint64_t K1 = bud.G * bud.B1;
    for (uint64_t k = 0; k < K1; ++k)
      q[k] = probe_q(row_ptr, col_idx, (uint64_t)n, s, t, L, seed, (uint32_t)k, bud.R, ORC_TAG_PROBE, ORC_TAG_WALK,
                     u_out ? u_out + k * bud.R : NULL, NULL, NULL, visits);
    B = adaptive_B(q, bud.B1, bud.B, bud.G, eps, c.z, (double)(row_ptr[s + 1] - row_ptr[s]),
                   (double)(row_ptr[t + 1] - row_ptr[t]));
    K = bud.G * B;
    for (uint64_t k = K1; k < K; ++k)
      q[k] = probe_q(row_ptr, col_idx, (uint64_t)n, s, t, L, seed, (uint32_t)k, bud.R, ORC_TAG_PROBE, ORC_TAG_WALK,
                     u_out ? u_out + k * bud.R : NULL, NULL, NULL, visits);
    if (budget_out) {
      budget_out[0] = B;
      budget_out[2] = K;
    }
  } else {
    for (uint64_t k = 0; k < K; ++k)
      q[k] = probe_q(row_ptr, col_idx, (uint64_t)n, s, t, L, seed, (uint32_t)k, bud.R, ORC_TAG_PROBE, ORC_TAG_WALK,
                     u_out ? u_out + k * bud.R : NULL, NULL, NULL, visits);
  }
  *beta_hat = median_of_means(q, B, bud.G);
  if (!q_out) free(q);
  return 0;
}

/* The ADAPTIVE stopping rule on given first-stage values (tests pin it directly). */
uint64_t orc_adaptive_B(const double* q, uint64_t B1, uint64_t B, uint64_t G, double eps, double z, double ds,
                        double dt) {
  return adaptive_B(q, B1, B, G, eps, z, ds, dt);
}

/* Median of the G block means of q[0 .. B*G) (tests pin it directly). */
double orc_median_of_means(const double* q, uint64_t B, uint64_t G) { return median_of_means(q, B, G); }

/* U_p of the PILOT stage's K0 probes x R0 replicas, probe-major (tests pin the
 * pilot's sigma^2 and theta against these replicas). */
int orc_pilot_u(const int64_t* row_ptr, const int32_t* col_idx, int64_t n, int64_t s, int64_t t, int32_t L,
                uint64_t seed, int32_t K0, int32_t R0, float* u_out) {
  if (n < 2 || s < 0 || t < 0 || s >= n || t >= n || s == t || L < 0 || K0 < 1 || R0 < 2) return -1;
  for (int32_t k = 0; k < K0; ++k)
    probe_q(row_ptr, col_idx, (uint64_t)n, s, t, L, seed, (uint32_t)k, (uint64_t)R0, ORC_TAG_PROBE_PILOT,
            ORC_TAG_WALK_PILOT, u_out + (uint64_t)k * (uint64_t)R0, NULL, NULL, NULL);
  return 0;
}

/* Budget alone (runs the pilot in PILOT mode). */
int orc_budget_query(const int64_t* row_ptr, const int32_t* col_idx, int64_t n, int64_t s, int64_t t, double eps,
                     int32_t L, uint64_t seed, const orc_budget_cfg* cfg, uint64_t* budget_out, double* pilot_out) {
  if (n < 2 || s < 0 || t < 0 || s >= n || t >= n || s == t || L < 0 || !(eps > 0.0 && eps < 1.0)) return -1;
  orc_budget bud;
  if (compute_budget(row_ptr, col_idx, (uint64_t)n, s, t, eps, L, seed, cfg, &bud) != 0) return -1;
  budget_out[0] = bud.B; budget_out[1] = bud.G; budget_out[2] = bud.K; budget_out[3] = bud.R;
  if (pilot_out) {
    pilot_out[0] = bud.sigma2_hat; pilot_out[1] = bud.q_bar; pilot_out[2] = bud.theta_hat;
  }
  return 0;
}

/* Q_R of selected probes of a query whose budget is given (tests compare
 * sampled per-probe values of large runs one by one). */
int orc_probe_q(const int64_t* row_ptr, const int32_t* col_idx, int64_t n, int64_t s, int64_t t, int32_t L,
                uint64_t seed, uint64_t R, int64_t count, const uint32_t* ks, double* q_out) {
  for (int64_t i = 0; i < count; ++i)
    q_out[i] = probe_q(row_ptr, col_idx, (uint64_t)n, s, t, L, seed, ks[i], R, ORC_TAG_PROBE, ORC_TAG_WALK, NULL,
                       NULL, NULL, NULL);
  return 0;
}

/* Many independent queries, one thread per query (the paper's setting), the
 * queries spread over `threads` OpenMP threads (<= 0: all available). */
int orc_query_many(const int64_t* row_ptr, const int32_t* col_idx, int64_t n, int64_t count, const int64_t* s,
                   const int64_t* t, const double* eps, const int32_t* L, const uint64_t* seeds,
                   const orc_budget_cfg* cfg, int threads, double* beta_hat, uint64_t* budgets, int32_t* status) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t i = 0; i < count; ++i) {
    status[i] = orc_query(row_ptr, col_idx, n, s[i], t[i], eps[i], L[i], seeds[i], cfg, &beta_hat[i],
                          budgets ? budgets + 4 * i : NULL, NULL, NULL, NULL, NULL);
  }
  return 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
