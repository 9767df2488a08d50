/*
 * sg_oracle_gauss.c -- plain CPU oracle for the Edwards-Anderson model with general
 * (e.g. Gaussian) couplings, Eq. 1 with H = 0 and J_ij drawn by the caller (Sec. 2.1:
 * "a standard normal distribution").  TEST INFRASTRUCTURE ONLY, like sg_oracle.c; it
 * shares no code with the CUDA library.
 *
 * Readings (each is listed in the design notes):
 *   - couplings are fixed-point integers in units of 2^-20 (J = J_int 2^-20), passed in
 *     by the caller, so that every energy is an exact int64 in those units and no sum
 *     depends on its order;
 *   - Metropolis (Sec. 2.2): dE = 2 s_i sum_j J_ij s_j; accept iff dE <= 0 or
 *     r < thr, r the replica's Philox word (the same counters as the +-J model) and
 *     thr = floor(e 2^32) (2^32 - 1 at e = 1), e an fp32 evaluation of
 *     exp(-beta dE) written out below (Cody & Waite's range reduction by ln 2 and a
 *     degree-6 Taylor polynomial, every operation a single IEEE fp32 add or multiply in
 *     a fixed order), so that any IEEE implementation reproduces it bit for bit;
 *     beta_f = (float) beta, x = -(beta_f (float) dE) 2^-20, and x < -23 gives thr = 0;
 *   - replica exchange as in the +-J oracle (Eq. 5, fp64), with
 *     delta = (beta_k - beta_k+1) ((E_a - E_b) 2^-20);
 *   - checkerboard order, hot start and Philox counters as in the +-J oracle.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

#define OG_TAG_METRO 0u
#define OG_TAG_PT 1u
#define OG_TAG_INIT 3u

typedef struct {
  int ndim, L[3], N, S, s0, C, T;
  double *beta;
  float *beta_f;
  uint64_t sim_seed;
  int32_t *J;    /* [S][N][d] fixed point, bond (i, mu) joins i and i + e_mu */
  int8_t *spin;  /* [S][C][T][N] */
  int64_t *E;    /* [S][C][T] by replica, units 2^-20 */
  int32_t *perm, *slot;
  uint32_t t_metro, t_pt;
  uint64_t near_threshold;
  uint64_t *pt_accept, *pt_tries;
} og_state;

static uint32_t og_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int w) {
  uint32_t ctr[4] = {c0, c1, c2, c3}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)}, out[4];
  or_philox4x32_10(ctr, key, out);
  return out[w];
}

/* exp(x) for -23 <= x <= 0 in fp32: x = k ln2 + r with k = floor(x / ln2 + 1/2) and
 * ln 2 split into a head with a short mantissa (k ln2_hi exact) and a tail; then
 * exp(r) by its Taylor series to r^6 in Horner form, times 2^k. */
float og_exp_f(float x) {
  volatile float vx = x; /* keep the compiler from reassociating anything below */
  float xv = vx;
  /* 1/ln 2 and ln 2 = ln2_hi + ln2_lo rounded to fp32 (ln2_hi has 16 significant bits,
   * so k ln2_hi is exact for |k| < 2^8); the series coefficients 1/n! likewise */
  const float inv_ln2 = 0x1.715476p+0f;
  const float ln2_hi = 0x1.62e4p-1f;
  const float ln2_lo = 0x1.7f7d1cp-20f;
  float t = xv * inv_ln2;
  t = t + 0.5f;
  const float kf = floorf(t);
  const int k = (int)kf;
  float r = xv - kf * ln2_hi;
  r = r - kf * ln2_lo;
  float p = 0x1.6c16c2p-10f; /* 1/720 */
  p = p * r;
  p = p + 0x1.111112p-7f; /* 1/120 */
  p = p * r;
  p = p + 0x1.555556p-5f; /* 1/24 */
  p = p * r;
  p = p + 0x1.555556p-3f; /* 1/6 */
  p = p * r;
  p = p + 0.5f;
  p = p * r;
  p = p + 1.0f;
  p = p * r;
  p = p + 1.0f;
  /* 2^k as a float built from its exponent bits (k in [-34, 1]) */
  union {
    uint32_t u;
    float f;
  } two;
  two.u = (uint32_t)(k + 127) << 23;
  return p * two.f;
}

uint32_t og_threshold(float beta_f, int32_t dE) {
  const float xs = (float)dE * 0x1p-20f;
  const float x = -(beta_f * xs);
  if (x < -23.0f) return 0u;
  const float e = og_exp_f(x);
  if (e >= 1.0f) return 0xFFFFFFFFu;
  return (uint32_t)(e * 4294967296.0f);
}

static int og_site(const og_state *st, int x, int y, int z) { return x + st->L[0] * (y + st->L[1] * z); }

static void og_coords(const og_state *st, int i, int c[3]) {
  c[0] = i % st->L[0];
  c[1] = (i / st->L[0]) % st->L[1];
  c[2] = i / (st->L[0] * st->L[1]);
}

static int og_nbr(const og_state *st, int i, int mu, int dir) {
  int c[3];
  og_coords(st, i, c);
  c[mu] = (c[mu] + dir + st->L[mu]) % st->L[mu];
  return og_site(st, c[0], c[1], c[2]);
}

static int8_t *og_spins(og_state *st, int s, int c, int j) {
  return st->spin + (((size_t)s * st->C + c) * st->T + j) * st->N;
}

/* h_i = sum over the 2d bonds of i of J s_j (fixed point) */
static int64_t og_field(const og_state *st, int s, const int8_t *sp, int i) {
  const int d = st->ndim;
  const int32_t *J = st->J + (size_t)s * st->N * d;
  int64_t h = 0;
  for (int mu = 0; mu < d; ++mu) {
    h += (int64_t)J[(size_t)i * d + mu] * sp[og_nbr(st, i, mu, +1)];
    const int b = og_nbr(st, i, mu, -1);
    h += (int64_t)J[(size_t)b * d + mu] * sp[b];
  }
  return h;
}

/* Eq. 1 (H = 0): E = -sum over bonds of J s_i s_j, fixed point */
int64_t og_energy_of(const og_state *st, int s, const int8_t *sp) {
  const int d = st->ndim;
  const int32_t *J = st->J + (size_t)s * st->N * d;
  int64_t e = 0;
  for (int i = 0; i < st->N; ++i)
    for (int mu = 0; mu < d; ++mu) e -= (int64_t)J[(size_t)i * d + mu] * sp[i] * sp[og_nbr(st, i, mu, +1)];
  return e;
}

static void og_recompute(og_state *st) {
  for (int s = 0; s < st->S; ++s)
    for (int c = 0; c < st->C; ++c)
      for (int j = 0; j < st->T; ++j)
        st->E[((size_t)s * st->C + c) * st->T + j] = og_energy_of(st, s, og_spins(st, s, c, j));
}

og_state *og_create(int ndim, const int32_t *dims, int S, int s0, int C, int T, const double *temps,
                    uint64_t sim_seed, const int32_t *J) {
  og_state *st = (og_state *)calloc(1, sizeof(og_state));
  st->ndim = ndim;
  st->N = 1;
  for (int a = 0; a < 3; ++a) {
    st->L[a] = a < ndim ? dims[a] : 1;
    st->N *= st->L[a];
  }
  st->S = S;
  st->s0 = s0;
  st->C = C;
  st->T = T;
  st->sim_seed = sim_seed;
  const size_t R = (size_t)S * C * T;
  st->beta = (double *)malloc(sizeof(double) * T);
  st->beta_f = (float *)malloc(sizeof(float) * T);
  for (int k = 0; k < T; ++k) {
    st->beta[k] = 1.0 / temps[k];
    st->beta_f[k] = (float)st->beta[k];
  }
  st->J = (int32_t *)malloc(sizeof(int32_t) * ((size_t)S * st->N * ndim + 1));
  memcpy(st->J, J, sizeof(int32_t) * (size_t)S * st->N * ndim);
  st->spin = (int8_t *)malloc(R * st->N + 1);
  st->E = (int64_t *)malloc(sizeof(int64_t) * (R + 1));
  st->perm = (int32_t *)malloc(sizeof(int32_t) * (R + 1));
  st->slot = (int32_t *)malloc(sizeof(int32_t) * (R + 1));
  st->pt_accept = (uint64_t *)calloc((size_t)T, sizeof(uint64_t));
  st->pt_tries = (uint64_t *)calloc((size_t)T, sizeof(uint64_t));
  for (int s = 0; s < S; ++s)
    for (int c = 0; c < C; ++c)
      for (int j = 0; j < T; ++j) {
        int8_t *sp = og_spins(st, s, c, j);
        const uint32_t c3 = ((uint32_t)c << 20) | ((uint32_t)(j >> 2) << 8) | OG_TAG_INIT;
        for (int i = 0; i < st->N; ++i)
          sp[i] = (og_word(sim_seed, (uint32_t)i, 0u, (uint32_t)(s0 + s), c3, j & 3) >> 31) ? -1 : 1;
        st->perm[((size_t)s * C + c) * T + j] = j;
        st->slot[((size_t)s * C + c) * T + j] = j;
      }
  og_recompute(st);
  return st;
}

void og_destroy(og_state *st) {
  if (!st) return;
  free(st->beta);
  free(st->beta_f);
  free(st->J);
  free(st->spin);
  free(st->E);
  free(st->perm);
  free(st->slot);
  free(st->pt_accept);
  free(st->pt_tries);
  free(st);
}

/* Checkerboard Metropolis sweeps (Sec. 2.2): colour 0, then colour 1. */
void og_sweep(og_state *st, int n) {
  for (int a = 0; a < n; ++a) {
    const uint32_t t = st->t_metro;
    for (int col = 0; col < 2; ++col)
      for (int s = 0; s < st->S; ++s)
        for (int c = 0; c < st->C; ++c)
          for (int j = 0; j < st->T; ++j) {
            int8_t *sp = og_spins(st, s, c, j);
            const int k = st->slot[((size_t)s * st->C + c) * st->T + j];
            const uint32_t c3 = ((uint32_t)c << 20) | ((uint32_t)(j >> 2) << 8) | OG_TAG_METRO;
            for (int i = 0; i < st->N; ++i) {
              int cc[3];
              og_coords(st, i, cc);
              if (((cc[0] + cc[1] + cc[2]) & 1) != col) continue;
              const int64_t dE = 2 * (int64_t)sp[i] * og_field(st, s, sp, i);
              int accept = dE <= 0;
              if (!accept) {
                const uint32_t r = og_word(st->sim_seed, (uint32_t)i, t, (uint32_t)(st->s0 + s), c3, j & 3);
                accept = r < og_threshold(st->beta_f[k], (int32_t)dE);
              }
              if (accept) {
                sp[i] = (int8_t)-sp[i];
                st->E[((size_t)s * st->C + c) * st->T + j] += dE;
              }
            }
          }
    st->t_metro++;
  }
}

/* Replica exchange (Eq. 5), per chain, pairs k = 0..T-2 in ascending order. */
void og_exchange(og_state *st) {
  const uint32_t t = st->t_pt;
  for (int s = 0; s < st->S; ++s)
    for (int c = 0; c < st->C; ++c) {
      int32_t *perm = st->perm + ((size_t)s * st->C + c) * st->T;
      int32_t *slot = st->slot + ((size_t)s * st->C + c) * st->T;
      const int64_t *E = st->E + ((size_t)s * st->C + c) * st->T;
      for (int k = 0; k + 1 < st->T; ++k) {
        const int a = perm[k], b = perm[k + 1];
        const double dbeta = st->beta[k] - st->beta[k + 1];
        const double delta = dbeta * ((double)(E[a] - E[b]) * 0x1p-20);
        const uint32_t u =
            og_word(st->sim_seed, (uint32_t)k, t, (uint32_t)(st->s0 + s), ((uint32_t)c << 20) | OG_TAG_PT, 0);
        int accept;
        if (delta >= 0.0) {
          accept = 1;
        } else {
          const double x = (double)u * 0x1p-32, e = exp(delta);
          if (fabs(x - e) < 1e-12) st->near_threshold++;
          accept = x < e;
        }
        st->pt_tries[k]++;
        if (accept) {
          st->pt_accept[k]++;
          perm[k] = b;
          perm[k + 1] = a;
          slot[a] = k + 1;
          slot[b] = k;
        }
      }
    }
  st->t_pt++;
}

void og_mcs(og_state *st, int n, int n_metro) {
  for (int a = 0; a < n; ++a) {
    og_sweep(st, n_metro);
    og_exchange(st);
  }
}

void og_get_spins(const og_state *st, uint8_t *out) {
  const size_t n = (size_t)st->S * st->C * st->T * st->N;
  for (size_t i = 0; i < n; ++i) out[i] = st->spin[i] < 0;
}
void og_set_spins(og_state *st, const uint8_t *in) {
  const size_t n = (size_t)st->S * st->C * st->T * st->N;
  for (size_t i = 0; i < n; ++i) st->spin[i] = in[i] ? -1 : 1;
  og_recompute(st);
}
void og_get_energies(const og_state *st, int64_t *out) {
  memcpy(out, st->E, sizeof(int64_t) * (size_t)st->S * st->C * st->T);
}
void og_get_perm(const og_state *st, int32_t *perm) {
  memcpy(perm, st->perm, sizeof(int32_t) * (size_t)st->S * st->C * st->T);
}
/* E by slot [S][C][T] and N q [S][T] (Eq. 4) */
void og_measure(const og_state *st, int64_t *E_by_slot, int32_t *NQ) {
  for (int s = 0; s < st->S; ++s)
    for (int c = 0; c < st->C; ++c)
      for (int k = 0; k < st->T; ++k) {
        const size_t b = ((size_t)s * st->C + c) * st->T;
        E_by_slot[b + k] = st->E[b + st->perm[b + k]];
      }
  if (NQ && st->C >= 2)
    for (int s = 0; s < st->S; ++s)
      for (int k = 0; k < st->T; ++k) {
        const int8_t *sa = og_spins((og_state *)st, s, 0, st->perm[((size_t)s * st->C + 0) * st->T + k]);
        const int8_t *sb = og_spins((og_state *)st, s, 1, st->perm[((size_t)s * st->C + 1) * st->T + k]);
        int32_t q = 0;
        for (int i = 0; i < st->N; ++i) q += sa[i] * sb[i];
        NQ[(size_t)s * st->T + k] = q;
      }
}
void og_get_counters(const og_state *st, uint64_t *out4) {
  out4[0] = st->t_metro;
  out4[1] = st->t_pt;
  out4[2] = st->near_threshold;
  out4[3] = 0;
}
int og_check_energies(const og_state *st) {
  int bad = 0;
  for (int s = 0; s < st->S; ++s)
    for (int c = 0; c < st->C; ++c)
      for (int j = 0; j < st->T; ++j)
        bad += og_energy_of(st, s, og_spins((og_state *)st, s, c, j)) != st->E[((size_t)s * st->C + c) * st->T + j];
  return bad;
}
/* Every 2^N configuration's energy for sample s (N <= 24): a brute-force pin. */
int og_enumerate(const og_state *st, int s, int64_t *out) {
  const int N = st->N;
  if (N > 24) return -1;
  int8_t *sp = (int8_t *)malloc((size_t)N);
  for (uint64_t conf = 0; conf < (1ull << N); ++conf) {
    for (int i = 0; i < N; ++i) sp[i] = ((conf >> i) & 1) ? -1 : 1;
    out[conf] = og_energy_of(st, s, sp);
  }
  free(sp);
  return 0;
}
void og_run_binned(og_state *st, int n_mcs, int n_bins, double *sumE, double *sumE2) {
  const int per = n_mcs / n_bins;
  for (int a = 0; a < n_bins * per; ++a) {
    og_sweep(st, 1);
    og_exchange(st);
    const int bin = a / per;
    for (int s = 0; s < st->S; ++s)
      for (int c = 0; c < st->C; ++c)
        for (int k = 0; k < st->T; ++k) {
          const size_t b = ((size_t)s * st->C + c) * st->T;
          const double e = (double)st->E[b + st->perm[b + k]] * 0x1p-20;
          sumE[k * n_bins + bin] += e;
          sumE2[k * n_bins + bin] += e * e;
        }
  }
}
