/*
 * sg_oracle.c -- plain CPU oracle for the +-J Edwards-Anderson parallel-tempering
 * Monte Carlo of Kumar, Gross, Janke & Weigel, "Massively parallel simulations for
 * disordered systems" (arXiv:2003.04621).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, import or call
 * this file: only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code with the CUDA library (no headers, helpers,
 * tables or generators); the two meet only through the seeded inputs (lattice dims,
 * temperatures, seeds) that both receive.
 *
 * Everything here is deliberately plain: spins are int8 +-1, couplings are int8 +-1,
 * every energy change is computed from the definition (Eq. 1), and every random word
 * is drawn by a fresh Philox4x32-10 call.  Floating point is fp64 and only where the
 * paper puts it (the Metropolis threshold exp(-beta dE) and the replica-exchange test,
 * Eq. 5).  Build with -ffp-contract=off so that no a*b+c is fused.
 *
 * What each function follows:
 *   model, couplings             Sec. 2.1, Eq. 1 (H = 0) and Eq. 2 (bimodal, p)
 *   energy, overlap              Sec. 2.1, Eqs. 3-4
 *   overlap plane sums           Sec. 3 (two-replica measurements), Eq. 4 per plane
 *   Metropolis sweep             Sec. 2.2 / 2.4 step 1 (single-spin flip, Metropolis
 *                                rule), visited in checkerboard order
 *   replica exchange             Sec. 2.2, Eq. 5; temperature<->replica maps as two
 *                                arrays whose entries are swapped (Sec. 3)
 *   Houdayer move                Sec. 2.4, Eq. 10 and the text after it
 *   multi-cluster variant        Sec. 3 (every cluster exchanged with probability 1/2)
 *   MCS composition              Sec. 2.4 (Metropolis, then Houdayer, then PT)
 *   round trips in temperature   Sec. 2.3 (tunnelling time), counted after each pass
 *   random numbers               counter-based Philox (Sec. 3, Salmon et al. 2011)
 *   exact enumeration            brute force over all 2^N states (a pin, not a method
 *                                of the paper)
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - sweep order: two colours c(i) = (x+y+z) mod 2, colour 0 first; every extent even.
 *   - bonds: forward bonds only, bond (i,mu) joins i and i+e_mu mod L_mu; on an L=2 axis
 *     both bonds of a pair are kept (a multigraph).
 *   - Metropolis: dE = 2 s_i h_i; accept iff dE <= 0 or r < thr[T][dE/4] with
 *     thr = min(floor(exp(-beta dE) 2^32), 2^32-1) computed in fp64.
 *   - Philox key/counter layout (tags METRO 0, PT 1, HOUD 2, INIT 3, J 4):
 *       J     key=coupling_seed, ctr=(i, mu, s, 4), word 0; J=+1 iff w < floor(p 2^32)
 *       INIT  key=sim_seed, ctr=(i, 0, s, c<<20 | (j>>2)<<8 | 3), word j&3, s=-1 iff top bit
 *       METRO key=sim_seed, ctr=(i, t_metro, s, c<<20 | (j>>2)<<8 | 0), word j&3
 *       PT    key=sim_seed, ctr=(k, t_pt, s, c<<20 | 1), word 0
 *       HOUD  key=sim_seed, ctr=(k, t_houd, s, 2), word 0
 *     s = sample index within the job (sample_offset + local index), c = chain,
 *     j = replica within the chain, k = temperature slot, t_* = calls made so far.
 *   - PT: within each chain, pairs k = 0..T-2 in ascending order each call; accept iff
 *     delta >= 0 or u 2^-32 < exp(delta), delta = (beta_k - beta_k+1)(E_a - E_b).
 *     |u 2^-32 - exp(delta)| < 1e-12 (delta < 0) is counted as a near-threshold draw.
 *   - Houdayer: pairs (chain 0, chain 1) at each temperature slot; seed = the
 *     floor(u M / 2^32)-th site with q = -1 in increasing site index; no move if M = 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_TAG_METRO 0u
#define OR_TAG_PT 1u
#define OR_TAG_HOUD 2u
#define OR_TAG_INIT 3u
#define OR_TAG_J 4u
#define OR_TAG_HMULTI 5u

/* ------------------------------------------------------------------------------ */
/* Philox4x32-10, from Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11.  Each round multiplies counter words 0 and 2 by the     */
/* round multipliers, and forms the new state from the high halves xor the other    */
/* counter words xor the round key, and the low halves.  The key is bumped by the   */
/* Weyl constants between rounds.                                                   */
/* ------------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

static uint32_t philox_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                            int word) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
  uint32_t out[4];
  or_philox4x32_10(ctr, key, out);
  return out[word];
}

/* ------------------------------------------------------------------------------ */
/* State                                                                          */
/* ------------------------------------------------------------------------------ */
typedef struct {
  int32_t ndim;
  int32_t dims[3];
  int32_t n_samples;     /* samples simulated by this oracle instance            */
  int32_t sample_offset; /* job-wide index of the first one (keys use it)        */
  int32_t n_chains;      /* independent copies per temperature (paper: N_C = 2)  */
  int32_t n_temps;
  const double *temps; /* ascending T_0 < ... < T_{n_temps-1}; copied            */
  uint64_t coupling_seed;
  double p_plus; /* P(J = +1), Eq. 2                                            */
  uint64_t sim_seed;
} or_params;

typedef struct {
  int ndim, L[3], N, S, s0, C, T;
  double *temps, *beta;
  uint32_t *thr; /* [T][d+1], entry m is the threshold for dE = 4m (m >= 1)    */
  uint64_t coupling_seed, sim_seed;
  double p_plus;
  int8_t *J;     /* [S][N][d], +-1: bond (i, mu) joins i and i + e_mu           */
  int8_t *spin;  /* [S][C][T][N], +-1, indexed by replica j (not temperature)   */
  int32_t *E;    /* [S][C][T] energy of replica j                               */
  int32_t *perm; /* [S][C][T] temperature slot k -> replica j                   */
  int32_t *slot; /* [S][C][T] replica j -> temperature slot k                   */
  uint32_t t_metro, t_pt, t_houd;
  uint64_t near_threshold;
  uint64_t *pt_accept; /* [T-1] accepted swaps per pair (k, k+1), all chains    */
  uint64_t *pt_tries;  /* [T-1]                                                  */
  /* Metropolis statistics per temperature slot and dE class m = dE/4 (m >= 1):  */
  uint64_t *cls_tries; /* [T][d+1] */
  uint64_t *cls_acc;   /* [T][d+1] */
  uint64_t houd_moves, houd_flipped; /* moves with M > 0, total cluster sites    */
  int houd_slots;      /* the cluster move acts on slots k < houd_slots (0: all)    */
  int typewriter;      /* 1: sweeps visit sites in index order i = 0..N-1 (lattices  */
                       /* with an odd extent, which have no checkerboard colouring)  */
  /* Round trips in temperature (the tunnelling time of Sec. 2.3), per replica j:   */
  int8_t *trip_dir;    /* [S][C][T] 0: no extreme seen, 1: bottom last, 2: top last */
  uint32_t *trip_t0;   /* [S][C][T] exchange pass of the trip's arrival at the bottom */
  uint32_t *trip_n;    /* [S][C] round trips completed                                */
  uint64_t *trip_sum;  /* [S][C] their total duration, in exchange passes             */
  int error;                         /* set if an internal consistency check fails */
} or_state;

static int site_index(const or_state *st, int x, int y, int z) {
  return x + st->L[0] * (y + st->L[1] * z);
}

static void site_coords(const or_state *st, int i, int *x, int *y, int *z) {
  *x = i % st->L[0];
  *y = (i / st->L[0]) % st->L[1];
  *z = i / (st->L[0] * st->L[1]);
}

/* Neighbour of site i one step along axis mu in direction dir (+1 or -1), periodic. */
static int neighbour(const or_state *st, int i, int mu, int dir) {
  int c[3];
  site_coords(st, i, &c[0], &c[1], &c[2]);
  c[mu] = (c[mu] + dir + st->L[mu]) % st->L[mu];
  return site_index(st, c[0], c[1], c[2]);
}

static int colour(const or_state *st, int i) {
  int x, y, z;
  site_coords(st, i, &x, &y, &z);
  return (x + y + z) & 1;
}

static int8_t *spins_of(or_state *st, int s, int c, int j) {
  return st->spin + (((size_t)s * st->C + c) * st->T + j) * st->N;
}
static int32_t *at3(int32_t *a, const or_state *st, int s, int c, int j) {
  return a + ((size_t)s * st->C + c) * st->T + j;
}

/* Eq. 1 with H = 0: E = - sum over bonds J_ij s_i s_j. */
static int32_t energy(const or_state *st, int s, const int8_t *sp) {
  const int8_t *J = st->J + (size_t)s * st->N * st->ndim;
  int32_t e = 0;
  for (int i = 0; i < st->N; ++i)
    for (int mu = 0; mu < st->ndim; ++mu) {
      int j = neighbour(st, i, mu, +1);
      e -= (int32_t)J[i * st->ndim + mu] * sp[i] * sp[j];
    }
  return e;
}

/* Local field h_i = sum over the 2d bonds of i of J_ij s_j. */
static int32_t local_field(const or_state *st, int s, const int8_t *sp, int i) {
  const int8_t *J = st->J + (size_t)s * st->N * st->ndim;
  int32_t h = 0;
  for (int mu = 0; mu < st->ndim; ++mu) {
    int fwd = neighbour(st, i, mu, +1);
    int bwd = neighbour(st, i, mu, -1);
    h += (int32_t)J[i * st->ndim + mu] * sp[fwd];
    h += (int32_t)J[bwd * st->ndim + mu] * sp[bwd];
  }
  return h;
}

static uint32_t threshold_of(double beta, int dE) {
  double x = beta * (double)dE;
  double v = floor(ldexp(exp(-x), 32));
  if (v >= 4294967295.0) return 0xFFFFFFFFu;
  return (uint32_t)v;
}

/* ------------------------------------------------------------------------------ */
/* Creation: couplings (Eq. 2), hot start, energies, identity temperature maps.   */
/* ------------------------------------------------------------------------------ */
void or_destroy(or_state *st);

or_state *or_create(const or_params *p) {
  if (p->ndim < 1 || p->ndim > 3 || p->n_samples < 0 || p->n_chains < 1 || p->n_temps < 1)
    return NULL;
  or_state *st = (or_state *)calloc(1, sizeof(or_state));
  st->ndim = p->ndim;
  st->N = 1;
  for (int a = 0; a < 3; ++a) {
    st->L[a] = a < p->ndim ? p->dims[a] : 1;
    if (st->L[a] < 1) {
      free(st);
      return NULL;
    }
    st->N *= st->L[a];
  }
  st->S = p->n_samples;
  st->s0 = p->sample_offset;
  st->C = p->n_chains;
  st->T = p->n_temps;
  st->coupling_seed = p->coupling_seed;
  st->sim_seed = p->sim_seed;
  st->p_plus = p->p_plus;
  const int d = st->ndim, T = st->T, C = st->C, S = st->S, N = st->N;

  st->temps = (double *)malloc(sizeof(double) * T);
  st->beta = (double *)malloc(sizeof(double) * T);
  st->thr = (uint32_t *)calloc((size_t)T * (d + 1), sizeof(uint32_t));
  for (int k = 0; k < T; ++k) {
    st->temps[k] = p->temps[k];
    st->beta[k] = 1.0 / p->temps[k];
    for (int m = 1; m <= d; ++m) st->thr[k * (d + 1) + m] = threshold_of(st->beta[k], 4 * m);
  }
  st->J = (int8_t *)malloc((size_t)S * N * d + 1);
  st->spin = (int8_t *)malloc((size_t)S * C * T * N + 1);
  st->E = (int32_t *)malloc(sizeof(int32_t) * ((size_t)S * C * T + 1));
  st->perm = (int32_t *)malloc(sizeof(int32_t) * ((size_t)S * C * T + 1));
  st->slot = (int32_t *)malloc(sizeof(int32_t) * ((size_t)S * C * T + 1));
  st->pt_accept = (uint64_t *)calloc((size_t)T, sizeof(uint64_t));
  st->trip_dir = (int8_t *)calloc((size_t)S * C * T + 1, 1);
  st->trip_t0 = (uint32_t *)calloc((size_t)S * C * T + 1, sizeof(uint32_t));
  st->trip_n = (uint32_t *)calloc((size_t)S * C + 1, sizeof(uint32_t));
  st->trip_sum = (uint64_t *)calloc((size_t)S * C + 1, sizeof(uint64_t));
  st->pt_tries = (uint64_t *)calloc((size_t)T, sizeof(uint64_t));
  st->cls_tries = (uint64_t *)calloc((size_t)T * (d + 1), sizeof(uint64_t));
  st->cls_acc = (uint64_t *)calloc((size_t)T * (d + 1), sizeof(uint64_t));

  /* Eq. 2: J = +1 with probability p.  The cut floor(p 2^32) is compared in 64 bits so
   * that p = 1 gives J = +1 always. */
  double cut_d = floor(ldexp(p->p_plus, 32));
  if (cut_d < 0.0) cut_d = 0.0;
  if (cut_d > 4294967296.0) cut_d = 4294967296.0;
  uint64_t cut = (uint64_t)cut_d;
  for (int s = 0; s < S; ++s) {
    uint32_t sg = (uint32_t)(st->s0 + s);
    for (int i = 0; i < N; ++i)
      for (int mu = 0; mu < d; ++mu) {
        uint32_t w = philox_word(st->coupling_seed, (uint32_t)i, (uint32_t)mu, sg, OR_TAG_J, 0);
        st->J[((size_t)s * N + i) * d + mu] = ((uint64_t)w < cut) ? 1 : -1;
      }
  }
  /* Hot start: each spin is -1 iff the top bit of its INIT word is set. */
  for (int s = 0; s < S; ++s) {
    uint32_t sg = (uint32_t)(st->s0 + s);
    for (int c = 0; c < C; ++c)
      for (int j = 0; j < T; ++j) {
        int8_t *sp = spins_of(st, s, c, j);
        uint32_t c3 = ((uint32_t)c << 20) | ((uint32_t)(j >> 2) << 8) | OR_TAG_INIT;
        for (int i = 0; i < N; ++i) {
          uint32_t w = philox_word(st->sim_seed, (uint32_t)i, 0u, sg, c3, j & 3);
          sp[i] = (w >> 31) ? -1 : 1;
        }
      }
  }
  for (int s = 0; s < S; ++s)
    for (int c = 0; c < C; ++c)
      for (int j = 0; j < T; ++j) {
        *at3(st->E, st, s, c, j) = energy(st, s, spins_of(st, s, c, j));
        *at3(st->perm, st, s, c, j) = j;
        *at3(st->slot, st, s, c, j) = j;
      }
  return st;
}

void or_destroy(or_state *st) {
  if (!st) return;
  free(st->temps);
  free(st->beta);
  free(st->thr);
  free(st->J);
  free(st->spin);
  free(st->E);
  free(st->perm);
  free(st->slot);
  free(st->pt_accept);
  free(st->pt_tries);
  free(st->cls_tries);
  free(st->cls_acc);
  free(st->trip_dir);
  free(st->trip_t0);
  free(st->trip_n);
  free(st->trip_sum);
  free(st);
}

/* ------------------------------------------------------------------------------ */
/* Metropolis sweep (Sec. 2.4 step 1) in checkerboard order, or in the sequential   */
/* typewriter order i = 0..N-1 (the paper's own per-thread walk through the lattice, */
/* Sec. 3) for lattices with an odd extent, where the two colours would not be       */
/* independent.  The random word of an attempt is the same in both orders.           */
/* ------------------------------------------------------------------------------ */
static void metropolis_sweep(or_state *st) {
  const int d = st->ndim;
  const uint32_t t = st->t_metro;
  const int passes = st->typewriter ? 1 : 2;
  for (int col = 0; col < passes; ++col)
    for (int i = 0; i < st->N; ++i) {
      if (!st->typewriter && colour(st, i) != col) continue;
      for (int s = 0; s < st->S; ++s) {
        uint32_t sg = (uint32_t)(st->s0 + s);
        for (int c = 0; c < st->C; ++c)
          for (int j = 0; j < st->T; ++j) {
            int8_t *sp = spins_of(st, s, c, j);
            int32_t dE = 2 * (int32_t)sp[i] * local_field(st, s, sp, i);
            int k = *at3(st->slot, st, s, c, j);
            int accept;
            if (dE <= 0) {
              accept = 1;
            } else {
              uint32_t c3 = ((uint32_t)c << 20) | ((uint32_t)(j >> 2) << 8) | OR_TAG_METRO;
              uint32_t r = philox_word(st->sim_seed, (uint32_t)i, t, sg, c3, j & 3);
              int m = dE / 4;
              accept = r < st->thr[k * (d + 1) + m];
              st->cls_tries[k * (d + 1) + m]++;
              st->cls_acc[k * (d + 1) + m] += (uint64_t)accept;
            }
            if (accept) {
              sp[i] = (int8_t)-sp[i];
              *at3(st->E, st, s, c, j) += dE;
            }
          }
      }
    }
  st->t_metro++;
}

void or_set_typewriter(or_state *st, int on) { st->typewriter = on ? 1 : 0; }

void or_sweep(or_state *st, int n) {
  for (int a = 0; a < n; ++a) metropolis_sweep(st);
}

/* ------------------------------------------------------------------------------ */
/* Replica exchange (Eq. 5): exchange temperatures, i.e. swap the two map entries. */
/* ------------------------------------------------------------------------------ */
void or_exchange(or_state *st) {
  const uint32_t t = st->t_pt;
  for (int s = 0; s < st->S; ++s) {
    uint32_t sg = (uint32_t)(st->s0 + s);
    for (int c = 0; c < st->C; ++c) {
      int32_t *perm = at3(st->perm, st, s, c, 0);
      int32_t *slot = at3(st->slot, st, s, c, 0);
      int32_t *E = at3(st->E, st, s, c, 0);
      for (int k = 0; k + 1 < st->T; ++k) {
        int a = perm[k], b = perm[k + 1];
        double dbeta = st->beta[k] - st->beta[k + 1];
        double delta = dbeta * (double)(E[a] - E[b]);
        uint32_t u = philox_word(st->sim_seed, (uint32_t)k, t, sg, ((uint32_t)c << 20) | OR_TAG_PT, 0);
        int accept;
        if (delta >= 0.0) {
          accept = 1;
        } else {
          double x = (double)u * 0x1p-32;
          double e = exp(delta);
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
      /* Round trips (Sec. 2.3: the time to go from the lowest to the highest
       * temperature and back): after pass t + 1, a replica at the lowest slot whose
       * last extreme was the highest completes a trip that began at its previous
       * arrival at the bottom; at the highest slot it turns around. */
      if (st->T >= 2) {
        const size_t cb = ((size_t)s * st->C + c) * st->T;
        for (int j = 0; j < st->T; ++j) {
          int8_t *dir = &st->trip_dir[cb + j];
          uint32_t *t0 = &st->trip_t0[cb + j];
          if (slot[j] == 0) {
            if (*dir == 2) {
              st->trip_n[(size_t)s * st->C + c]++;
              st->trip_sum[(size_t)s * st->C + c] += (uint64_t)(t + 1 - *t0);
              *t0 = t + 1;
              *dir = 1;
            } else if (*dir == 0) {
              *t0 = t + 1;
              *dir = 1;
            }
          } else if (slot[j] == st->T - 1 && *dir == 1) {
            *dir = 2;
          }
        }
      }
    }
  }
  st->t_pt++;
}

/* Round-trip counters per chain: n[S][C] trips completed, sum[S][C] total duration. */
void or_get_trips(const or_state *st, uint32_t *n, uint64_t *sum) {
  memcpy(n, st->trip_n, sizeof(uint32_t) * (size_t)st->S * st->C);
  memcpy(sum, st->trip_sum, sizeof(uint64_t) * (size_t)st->S * st->C);
}

/* ------------------------------------------------------------------------------ */
/* Houdayer cluster move (Sec. 2.4, Eq. 10), one per (sample, temperature slot).  */
/* ------------------------------------------------------------------------------ */
/* The slots the move acts on: all T, or only the lowest houd_slots temperatures.      */
/* Reading of the 3D modification that Secs. 1 and 2.4 point to (a manual cut of the    */
/* effective cluster size): the move is kept to low temperatures, below the point where */
/* q = -1 clusters percolate.  Pairs at other slots are left alone.                     */
static int houd_kmax(const or_state *st) {
  return (st->houd_slots > 0 && st->houd_slots < st->T) ? st->houd_slots : st->T;
}

void or_set_houdayer_slots(or_state *st, int k) {
  if (k < 0 || k > st->T) st->error = 1;
  else st->houd_slots = k;
}

void or_houdayer(or_state *st) {
  if (st->C < 2) {
    st->error = 1;
    return;
  }
  const int N = st->N, d = st->ndim, kmax = houd_kmax(st);
  const uint32_t t = st->t_houd;
  int8_t *q = (int8_t *)malloc((size_t)N);
  uint8_t *in = (uint8_t *)malloc((size_t)N);
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  for (int s = 0; s < st->S; ++s) {
    uint32_t sg = (uint32_t)(st->s0 + s);
    for (int k = 0; k < kmax; ++k) {
      int a = *at3(st->perm, st, s, 0, k);
      int b = *at3(st->perm, st, s, 1, k);
      int8_t *sa = spins_of(st, s, 0, a);
      int8_t *sb = spins_of(st, s, 1, b);
      uint32_t M = 0;
      for (int i = 0; i < N; ++i) {
        q[i] = (int8_t)(sa[i] * sb[i]); /* Eq. 10 */
        M += (q[i] == -1);
      }
      if (M == 0) continue;
      uint32_t u = philox_word(st->sim_seed, (uint32_t)k, t, sg, OR_TAG_HOUD, 0);
      uint32_t n = (uint32_t)(((uint64_t)u * (uint64_t)M) >> 32);
      int i0 = -1;
      for (int i = 0, seen = 0; i < N; ++i)
        if (q[i] == -1) {
          if ((uint32_t)seen == n) {
            i0 = i;
            break;
          }
          ++seen;
        }
      /* Breadth-first search over neighbouring sites with q = -1. */
      memset(in, 0, (size_t)N);
      int head = 0, tail = 0;
      queue[tail++] = i0;
      in[i0] = 1;
      while (head < tail) {
        int i = queue[head++];
        for (int mu = 0; mu < d; ++mu)
          for (int dir = -1; dir <= 1; dir += 2) {
            int j = neighbour(st, i, mu, dir);
            if (!in[j] && q[j] == -1) {
              in[j] = 1;
              queue[tail++] = j;
            }
          }
      }
      /* Exchange the two configurations on the cluster. */
      int32_t before = *at3(st->E, st, s, 0, a) + *at3(st->E, st, s, 1, b);
      for (int x = 0; x < tail; ++x) {
        int i = queue[x];
        int8_t tmp = sa[i];
        sa[i] = sb[i];
        sb[i] = tmp;
      }
      int32_t ea = energy(st, s, sa), eb = energy(st, s, sb);
      if (ea + eb != before) st->error = 2; /* E1 + E2 must be conserved */
      *at3(st->E, st, s, 0, a) = ea;
      *at3(st->E, st, s, 1, b) = eb;
      st->houd_moves++;
      st->houd_flipped += (uint64_t)tail;
    }
  }
  free(q);
  free(in);
  free(queue);
  st->t_houd++;
}

/* ------------------------------------------------------------------------------ */
/* Multi-cluster variant of the move (Sec. 3, the remedy for idle threads named    */
/* there): every q = -1 cluster of a pair is exchanged with probability 1/2, each  */
/* by its own coin (q = +1 clusters would leave both replicas unchanged).  Reading */
/* of the coin: the top bit of the Philox word with counter                        */
/* (i_min, t_houd, s, k << 8 | 5), i_min the cluster's smallest site index.        */
/* ------------------------------------------------------------------------------ */
void or_houdayer_multi(or_state *st) {
  if (st->C < 2) {
    st->error = 1;
    return;
  }
  const int N = st->N, d = st->ndim, kmax = houd_kmax(st);
  const uint32_t t = st->t_houd;
  int8_t *q = (int8_t *)malloc((size_t)N);
  uint8_t *in = (uint8_t *)malloc((size_t)N);
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  for (int s = 0; s < st->S; ++s) {
    uint32_t sg = (uint32_t)(st->s0 + s);
    for (int k = 0; k < kmax; ++k) {
      int a = *at3(st->perm, st, s, 0, k);
      int b = *at3(st->perm, st, s, 1, k);
      int8_t *sa = spins_of(st, s, 0, a);
      int8_t *sb = spins_of(st, s, 1, b);
      uint32_t M = 0;
      for (int i = 0; i < N; ++i) {
        q[i] = (int8_t)(sa[i] * sb[i]); /* Eq. 10 */
        M += (q[i] == -1);
      }
      if (M == 0) continue;
      int32_t before = *at3(st->E, st, s, 0, a) + *at3(st->E, st, s, 1, b);
      memset(in, 0, (size_t)N);
      for (int i0 = 0; i0 < N; ++i0) {
        if (q[i0] != -1 || in[i0]) continue;
        /* a new cluster; i0 is its smallest site (sites are visited in increasing order) */
        int head = 0, tail = 0;
        queue[tail++] = i0;
        in[i0] = 1;
        while (head < tail) {
          int i = queue[head++];
          for (int mu = 0; mu < d; ++mu)
            for (int dir = -1; dir <= 1; dir += 2) {
              int j = neighbour(st, i, mu, dir);
              if (!in[j] && q[j] == -1) {
                in[j] = 1;
                queue[tail++] = j;
              }
            }
        }
        uint32_t u = philox_word(st->sim_seed, (uint32_t)i0, t, sg, ((uint32_t)k << 8) | OR_TAG_HMULTI, 0);
        if (u >> 31) {
          for (int x = 0; x < tail; ++x) {
            int i = queue[x];
            int8_t tmp = sa[i];
            sa[i] = sb[i];
            sb[i] = tmp;
          }
          st->houd_flipped += (uint64_t)tail;
        }
      }
      int32_t ea = energy(st, s, sa), eb = energy(st, s, sb);
      if (ea + eb != before) st->error = 2; /* E1 + E2 must be conserved */
      *at3(st->E, st, s, 0, a) = ea;
      *at3(st->E, st, s, 1, b) = eb;
      st->houd_moves++;
    }
  }
  free(q);
  free(in);
  free(queue);
  st->t_houd++;
}

/* One MCS (Sec. 2.4): n_metro sweeps, one Houdayer move per pair (houdayer = 1: the
 * single-cluster move, 2: the multi-cluster variant), one PT pass. */
void or_mcs(or_state *st, int n_mcs, int n_metro, int houdayer) {
  for (int a = 0; a < n_mcs; ++a) {
    or_sweep(st, n_metro);
    if (houdayer == 1) or_houdayer(st);
    else if (houdayer == 2) or_houdayer_multi(st);
    or_exchange(st);
  }
}

/* ------------------------------------------------------------------------------ */
/* Measurement: E by temperature slot and N q (Eq. 4) per (sample, slot).         */
/* ------------------------------------------------------------------------------ */
void or_measure(const or_state *st_c, int32_t *E_by_slot, int32_t *NQ) {
  or_state *st = (or_state *)st_c;
  for (int s = 0; s < st->S; ++s)
    for (int c = 0; c < st->C; ++c)
      for (int k = 0; k < st->T; ++k) {
        int j = *at3(st->perm, st, s, c, k);
        E_by_slot[((size_t)s * st->C + c) * st->T + k] = *at3(st->E, st, s, c, j);
      }
  if (NQ && st->C >= 2)
    for (int s = 0; s < st->S; ++s)
      for (int k = 0; k < st->T; ++k) {
        const int8_t *sa = spins_of(st, s, 0, *at3(st->perm, st, s, 0, k));
        const int8_t *sb = spins_of(st, s, 1, *at3(st->perm, st, s, 1, k));
        int32_t qsum = 0;
        for (int i = 0; i < st->N; ++i) qsum += sa[i] * sb[i];
        NQ[(size_t)s * st->T + k] = qsum;
      }
}

/* Plane sums of the overlap field, the integer part of the Fourier modes behind the
 * spin-glass susceptibility and the correlation length (two-replica quantities, Sec. 3):
 * P[s][k][mu][x] = sum of q_i = s_i^(a) s_i^(b) (Eq. 4 before the sum) over the sites
 * i with coordinate x along axis mu, a and b the chain-0 and chain-1 replicas at slot
 * k.  Lmax = max extent; entries x >= L_mu are 0.  Then q(k e_mu) = (1/N) sum_x
 * e^{i k x} P[mu][x]. */
void or_qmodes(const or_state *st_c, int32_t *P) {
  or_state *st = (or_state *)st_c;
  const int d = st->ndim;
  int Lmax = st->L[0];
  for (int mu = 1; mu < d; ++mu)
    if (st->L[mu] > Lmax) Lmax = st->L[mu];
  memset(P, 0, sizeof(int32_t) * (size_t)st->S * st->T * d * Lmax);
  if (st->C < 2) return;
  for (int s = 0; s < st->S; ++s)
    for (int k = 0; k < st->T; ++k) {
      const int8_t *sa = spins_of(st, s, 0, *at3(st->perm, st, s, 0, k));
      const int8_t *sb = spins_of(st, s, 1, *at3(st->perm, st, s, 1, k));
      int32_t *Pk = P + ((size_t)s * st->T + k) * d * Lmax;
      for (int i = 0; i < st->N; ++i) {
        int c[3];
        site_coords(st, i, &c[0], &c[1], &c[2]);
        const int q = sa[i] * sb[i];
        for (int mu = 0; mu < d; ++mu) Pk[mu * Lmax + c[mu]] += q;
      }
    }
}

/* Recompute every energy from Eq. 1 and report how many differ from the kept ones. */
int or_check_energies(const or_state *st_c) {
  or_state *st = (or_state *)st_c;
  int bad = 0;
  for (int s = 0; s < st->S; ++s)
    for (int c = 0; c < st->C; ++c)
      for (int j = 0; j < st->T; ++j)
        bad += energy(st, s, spins_of(st, s, c, j)) != *at3(st->E, st, s, c, j);
  return bad;
}

/* ------------------------------------------------------------------------------ */
/* Accessors used by the tests.                                                   */
/* ------------------------------------------------------------------------------ */
/* spins as bits: out[s][c][j][i] = 1 iff s = -1 */
void or_get_spins(const or_state *st, uint8_t *out) {
  size_t n = (size_t)st->S * st->C * st->T * st->N;
  for (size_t a = 0; a < n; ++a) out[a] = st->spin[a] < 0;
}
void or_set_spins(or_state *st, const uint8_t *in) {
  size_t n = (size_t)st->S * st->C * st->T * st->N;
  for (size_t a = 0; a < n; ++a) st->spin[a] = in[a] ? -1 : 1;
  for (int s = 0; s < st->S; ++s)
    for (int c = 0; c < st->C; ++c)
      for (int j = 0; j < st->T; ++j)
        *at3(st->E, st, s, c, j) = energy(st, s, spins_of(st, s, c, j));
}
void or_get_couplings(const or_state *st, int8_t *out) {
  memcpy(out, st->J, (size_t)st->S * st->N * st->ndim);
}
void or_set_couplings(or_state *st, const int8_t *in) {
  memcpy(st->J, in, (size_t)st->S * st->N * st->ndim);
  for (int s = 0; s < st->S; ++s)
    for (int c = 0; c < st->C; ++c)
      for (int j = 0; j < st->T; ++j)
        *at3(st->E, st, s, c, j) = energy(st, s, spins_of(st, s, c, j));
}
void or_get_energies(const or_state *st, int32_t *out) {
  memcpy(out, st->E, sizeof(int32_t) * (size_t)st->S * st->C * st->T);
}
void or_get_perm(const or_state *st, int32_t *perm, int32_t *slot) {
  size_t n = (size_t)st->S * st->C * st->T;
  memcpy(perm, st->perm, sizeof(int32_t) * n);
  if (slot) memcpy(slot, st->slot, sizeof(int32_t) * n);
}
void or_get_thresholds(const or_state *st, uint32_t *out) { /* [T][d], m = 1..d */
  for (int k = 0; k < st->T; ++k)
    for (int m = 1; m <= st->ndim; ++m) out[k * st->ndim + (m - 1)] = st->thr[k * (st->ndim + 1) + m];
}
/* counters: t_metro, t_pt, t_houd, near_threshold, houd_moves, houd_flipped, error */
void or_get_counters(const or_state *st, uint64_t *out7) {
  out7[0] = st->t_metro;
  out7[1] = st->t_pt;
  out7[2] = st->t_houd;
  out7[3] = st->near_threshold;
  out7[4] = st->houd_moves;
  out7[5] = st->houd_flipped;
  out7[6] = (uint64_t)st->error;
}
void or_get_pt_stats(const or_state *st, uint64_t *acc, uint64_t *tries) {
  for (int k = 0; k + 1 < st->T; ++k) {
    acc[k] = st->pt_accept[k];
    tries[k] = st->pt_tries[k];
  }
}
void or_get_class_stats(const or_state *st, uint64_t *tries, uint64_t *acc) { /* [T][d] */
  for (int k = 0; k < st->T; ++k)
    for (int m = 1; m <= st->ndim; ++m) {
      tries[k * st->ndim + m - 1] = st->cls_tries[k * (st->ndim + 1) + m];
      acc[k * st->ndim + m - 1] = st->cls_acc[k * (st->ndim + 1) + m];
    }
}
/* Set the call counters (checkpoint/resume tests). */
void or_set_counters(or_state *st, uint32_t t_metro, uint32_t t_pt, uint32_t t_houd) {
  st->t_metro = t_metro;
  st->t_pt = t_pt;
  st->t_houd = t_houd;
}
void or_set_perm(or_state *st, const int32_t *perm) {
  size_t n = (size_t)st->S * st->C * st->T;
  memcpy(st->perm, perm, sizeof(int32_t) * n);
  for (int s = 0; s < st->S; ++s)
    for (int c = 0; c < st->C; ++c)
      for (int k = 0; k < st->T; ++k) *at3(st->slot, st, s, c, *at3(st->perm, st, s, c, k)) = k;
}

/* Run n MCS (sweeps, then Houdayer if on, then PT if on) and accumulate, per
 * temperature slot (all samples and chains pooled), bin sums of E and E^2 measured
 * after every MCS.  sumE/sumE2 are [T][n_bins]; the run is cut into n_bins
 * consecutive bins of n_mcs / n_bins MCS. */
void or_run_binned(or_state *st, int n_mcs, int n_metro, int houdayer, int pt, int n_bins,
                   double *sumE, double *sumE2) {
  int32_t *Eb = (int32_t *)malloc(sizeof(int32_t) * (size_t)st->S * st->C * st->T);
  int per_bin = n_mcs / n_bins;
  for (int a = 0; a < n_bins * per_bin; ++a) {
    or_sweep(st, n_metro);
    if (houdayer == 1) or_houdayer(st);
    else if (houdayer == 2) or_houdayer_multi(st);
    if (pt) or_exchange(st);
    or_measure(st, Eb, NULL);
    int bin = a / per_bin;
    for (int s = 0; s < st->S; ++s)
      for (int c = 0; c < st->C; ++c)
        for (int k = 0; k < st->T; ++k) {
          double e = (double)Eb[((size_t)s * st->C + c) * st->T + k];
          sumE[k * n_bins + bin] += e;
          sumE2[k * n_bins + bin] += e * e;
        }
  }
  free(Eb);
}

/* ------------------------------------------------------------------------------ */
/* Exact enumeration over all 2^N states of one sample (a pin, N <= 24).           */
/* Writes the energy histogram: hist[e + d N] = number of states with energy e.    */
/* ------------------------------------------------------------------------------ */
int or_enumerate(const or_state *st_c, int s, uint64_t *hist) {
  or_state *st = (or_state *)st_c;
  const int N = st->N, d = st->ndim;
  if (N > 24) return -1;
  int8_t *sp = (int8_t *)malloc((size_t)N);
  memset(hist, 0, sizeof(uint64_t) * (size_t)(2 * d * N + 1));
  for (uint64_t conf = 0; conf < (1ull << N); ++conf) {
    for (int i = 0; i < N; ++i) sp[i] = ((conf >> i) & 1) ? -1 : 1;
    int32_t e = energy(st, s, sp);
    hist[e + d * N]++;
  }
  free(sp);
  return 0;
}
