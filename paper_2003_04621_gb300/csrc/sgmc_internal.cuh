// sgmc_internal.cuh -- device-side definitions shared by the engine's kernels.
//
// Data layout in HBM (all inside the caller's buffer, each array 256-byte aligned):
//   spins, packed   uint32 [S][W][N]      W = C * Wc words per site, Wc = ceil(T/32);
//                                         word w holds chain c = w / Wc, replicas
//                                         j = 32 (w % Wc) + lane, lane = bit
//   spins, int8     int8   [S][C][N][Tp]  +-1, Tp = T rounded up to 4
//   couplings       uint32 [S][d][NW]     one bit plane per axis mu, bit p of plane mu is
//                                         1 iff J(i(p), mu) = -1; NW = ceil(N/32)
//   E, perm, slot   int32  [S][C][T]      energy of replica j; replica at slot k; slot of j
//   thr             uint32 [T][4]         thr[k][m] for m = 1..d (entry 0 unused)
//   beta            double [T]
//   counters        u64    [CTR_PT + T]   see CTR_* below
// Sites are stored in colour-split order p: the N/2 colour-0 sites first, then the
// colour-1 sites; inside a colour, row = y + L1 z and half-column k = x / 2, so
// p = c N/2 + row H + k with H = L0 / 2, and x = 2k + (c ^ ((y + z) & 1)).  A
// colour's neighbours are all in the other colour's half, at the same k (or k +- 1
// along x) of the neighbouring rows, so a half-sweep reads both halves contiguously.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sgmc {

// Philox stream tags (the last counter word's low byte).
constexpr uint32_t TAG_METRO = 0u, TAG_PT = 1u, TAG_HOUD = 2u, TAG_INIT = 3u, TAG_J = 4u, TAG_HMULTI = 5u;

// Counter slots in the device counter array.
constexpr int CTR_NEAR = 0;   // near-threshold exchange decisions
constexpr int CTR_HSITES = 1; // sites flipped by Houdayer moves
constexpr int CTR_ERROR = 2;  // bit flags of device-side errors (bounded waits that expired)
constexpr int CTR_HMOVES = 3; // Houdayer moves with M > 0
constexpr int CTR_TMETRO = 4; // Metropolis sweeps made (the t of the sweep counters)
constexpr int CTR_TPT = 5;    // exchange passes made
constexpr int CTR_THOUD = 6;  // Houdayer passes made
constexpr int CTR_DONE = 7;   // finished-CTA ticket of the running kernel
constexpr int CTR_XEXACT = 8; // exchange decisions of the warp exchanges decided by the exact fp64 test
constexpr int CTR_GBAND = 9;  // general-coupling Metropolis draws inside the screening band
constexpr int CTR_PT = 10;    // [T-1] accepted exchanges per pair

constexpr unsigned long long ERR_TMA_TIMEOUT = 1ull;
constexpr unsigned long long ERR_HOUD_ROUNDS = 2ull; // a cluster fill hit its round limit (never expected)

// Shared-memory budget the Houdayer kernel's bitmaps may use; above it they go to a
// scratch region of the caller's buffer.  A fixed number (not the device's) so that the
// buffer size does not depend on the device.
constexpr int HOUD_SMEM_BUDGET = 200 * 1024;

struct Geo {
  int d;          // 2 or 3
  int L0, L1, L2; // L2 = 1 in 2D
  int N;          // sites
  int H;          // L0 / 2
  int R;          // rows, L1 * L2
  int Nh;         // N / 2
  int NW;         // 32-bit words per coupling bit plane
};

struct Job {
  Geo g;
  int S, s_off, C, T, Wc, W, Tp;
  int hK;                  // the cluster move acts on the pairs at slots k < hK (<= T)
  uint32_t sk0, sk1;       // sim_seed as a Philox key
  uint32_t ck0, ck1;       // coupling_seed as a Philox key
  unsigned long long jcut; // J = +1 iff the word is below this (floor(p 2^32), up to 2^32)
  uint32_t rk0[10], rk1[10]; // sim_seed round keys (k + r W) so kernels read them as constants
};

struct Dev {
  uint32_t *spins;
  uint32_t *jbits;
  int32_t *E;
  int32_t *perm;
  int32_t *slot;
  const uint32_t *thr;
  const double *beta;
  unsigned long long *ctr;
  // general (fixed-point) couplings; null for +-J jobs
  int32_t *jfix;  // [S][d][N] colour-split site order, units of 2^-20
  long long *E64; // [S][C][T] energies by replica, units of 2^-20
  // round trips in temperature (null when the job does not track them)
  int32_t *trip_dir;             // [S][C][T] 0: no extreme yet, 1: lowest slot last, 2: highest last
  uint32_t *trip_t0;             // [S][C][T] exchange pass of the trip's arrival at the lowest slot
  uint32_t *trip_n;              // [S][C] round trips completed
  unsigned long long *trip_sum;  // [S][C] their total duration in exchange passes
};

// Round-trip bookkeeping of one replica after exchange pass t (counted from 1) (the
// tunnelling time of Sec. 2.3: lowest -> highest -> lowest temperature): at the lowest
// slot a replica whose last extreme was the highest completes a trip that began at its
// previous arrival at the bottom; at the highest slot it turns around.
__device__ __forceinline__ void trip_step(int T, int k, int32_t &dir, uint32_t &t0, uint32_t t, uint32_t &n_add,
                                          unsigned long long &sum_add) {
  if (T < 2) return;
  if (k == 0) {
    if (dir == 2) {
      n_add += 1u;
      sum_add += (unsigned long long)(t - t0);
      t0 = t;
      dir = 1;
    } else if (dir == 0) {
      t0 = t;
      dir = 1;
    }
  } else if (k == T - 1 && dir == 1) {
    dir = 2;
  }
}

// The same for every replica of one chain, by one thread, in global memory.
__device__ __forceinline__ void trip_chain(const Dev &dv, size_t chain, int T, const int32_t *slot, uint32_t t) {
  if (!dv.trip_dir) return;
  const size_t cb = chain * (size_t)T;
  uint32_t n_add = 0u;
  unsigned long long sum_add = 0ull;
  for (int j = 0; j < T; ++j) {
    int32_t dir = dv.trip_dir[cb + j];
    uint32_t t0 = dv.trip_t0[cb + j];
    trip_step(T, slot[j], dir, t0, t, n_add, sum_add);
    dv.trip_dir[cb + j] = dir;
    dv.trip_t0[cb + j] = t0;
  }
  dv.trip_n[chain] += n_add;
  dv.trip_sum[chain] += sum_add;
}

// One job of a resident-kernel launch: its description, the CTAs it owns (a contiguous
// range of the grid), whether its exchange runs inside the kernel, and its sweeps per MCS.
struct JobDesc {
  Job jb;
  Dev dv;
  int first_item; // first CTA of this job
  int n_items;    // CTAs of this job
  int fuse;       // 1: every CTA holds whole chains and runs their exchange between MCS
  int n_metro;    // sweeps per MCS
};

// Kernel parameters of the resident kernel: up to MAXJ jobs of one lattice shape.  The
// table lives in the kernel's parameter space (read through constant memory).
// The Houdayer move's bitmap scratch of one job, for the sweep kernels that take the
// move's first and last phases (the q bitmaps after the sweeps, the cluster flips before
// the energies): [S][T][NBW] q and cluster bitmaps and [S][32] M per pair.
struct HoudMaps {
  uint32_t *Qg;
  uint32_t *Cg;
  uint32_t *Mg;
  int RW;  // words per bitmap row
  int NBW; // words per bitmap
};

template <int MAXJ>
struct ResidentParams {
  int n_jobs;
  int n_mcs;
  int pad0; // energy-only single-job launches: 1 right after a Houdayer move (E_a + E_b kept)
  int pad1;
  // single-job launches of two one-word chains per CTA: after the last MCS, E by slot
  // [S][2][T] and N q [S][T] into these device arrays (null: no measurement)
  int32_t *mE, *mQ;
  HoudMaps hm; // single-job launches that take a phase of the Houdayer move
  JobDesc jobs[MAXJ];
};
constexpr int MAX_BATCH_JOBS = 96;
using resident_fn1 = void (*)(ResidentParams<1>);
using resident_fnB = void (*)(ResidentParams<MAX_BATCH_JOBS>);

// ---------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two 32x32->64
// multiplies; the new state is (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0); the key is
// bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------------
constexpr uint32_t PH_M0 = 0xD2511F53u, PH_M1 = 0xCD9E8D57u;
constexpr uint32_t PH_W0 = 0x9E3779B9u, PH_W1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox10(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3,
                                          uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(PH_M0, x0), lo0 = PH_M0 * x0;
    const uint32_t hi1 = __umulhi(PH_M1, x2), lo1 = PH_M1 * x2;
    const uint32_t y0 = hi1 ^ x1 ^ k0;
    const uint32_t y2 = hi0 ^ x3 ^ k1;
    x0 = y0;
    x1 = lo1;
    x2 = y2;
    x3 = lo0;
    k0 += PH_W0;
    k1 += PH_W1;
  }
  return make_uint4(x0, x1, x2, x3);
}

// As grid_done_advance, for the `n_items` CTAs of one job inside a larger grid.
__device__ __forceinline__ void job_done_advance(unsigned long long *ctr, int n_items, unsigned long long d_metro,
                                                 unsigned long long d_pt, unsigned long long d_houd) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long ticket = atomicAdd(&ctr[CTR_DONE], 1ull);
    if (ticket == (unsigned long long)n_items - 1ull) {
      ctr[CTR_TMETRO] += d_metro;
      ctr[CTR_TPT] += d_pt;
      ctr[CTR_THOUD] += d_houd;
      ctr[CTR_DONE] = 0ull;
      __threadfence();
    }
  }
}

// Step counters live on the device, so that any sequence of calls can be captured in a
// CUDA graph and replayed: every kernel reads the counters it needs when it starts, and
// the last CTA of the grid to finish (by an atomic ticket; every CTA has read the
// counters before taking one) advances them.  Every CTA must call this exactly once.
__device__ __forceinline__ void grid_done_advance(unsigned long long *ctr, unsigned long long d_metro,
                                                  unsigned long long d_pt, unsigned long long d_houd) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long ticket = atomicAdd(&ctr[CTR_DONE], 1ull);
    if (ticket == (unsigned long long)(gridDim.x * gridDim.y * gridDim.z) - 1ull) {
      ctr[CTR_TMETRO] += d_metro;
      ctr[CTR_TPT] += d_pt;
      ctr[CTR_THOUD] += d_houd;
      ctr[CTR_DONE] = 0ull;
      __threadfence();
    }
  }
}

// Philox4x32-10 with the ten round keys given explicitly (kernel-parameter arrays).
__device__ __forceinline__ uint4 philox10_rk(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3,
                                             const uint32_t *rk0, const uint32_t *rk1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(PH_M0, x0), lo0 = PH_M0 * x0;
    const uint32_t hi1 = __umulhi(PH_M1, x2), lo1 = PH_M1 * x2;
    const uint32_t y0 = hi1 ^ x1 ^ rk0[r];
    const uint32_t y2 = hi0 ^ x3 ^ rk1[r];
    x0 = y0;
    x1 = lo1;
    x2 = y2;
    x3 = lo0;
  }
  return make_uint4(x0, x1, x2, x3);
}

__device__ __forceinline__ uint32_t word_of(const uint4 &v, int w) {
  return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
}

// ---------------------------------------------------------------------------------
// Geometry helpers (colour-split order)
// ---------------------------------------------------------------------------------
struct SiteGeo {
  int c, row, k, y, z, xodd;
};

__device__ __forceinline__ SiteGeo site_geo(const Geo &g, int p) {
  SiteGeo s;
  s.c = p >= g.Nh;
  const int q = p - s.c * g.Nh;
  s.row = q / g.H;
  s.k = q - s.row * g.H;
  s.y = s.row % g.L1;
  s.z = s.row / g.L1;
  s.xodd = s.c ^ ((s.y + s.z) & 1);
  return s;
}

// canonical site index i = x + L0 (y + L1 z)
__device__ __forceinline__ int canonical_of(const Geo &g, const SiteGeo &s) {
  return g.L0 * s.row + 2 * s.k + s.xodd;
}

__device__ __forceinline__ int cs_of_canonical(const Geo &g, int i) {
  const int x = i % g.L0;
  const int row = i / g.L0;
  const int y = row % g.L1;
  const int z = row / g.L1;
  const int c = (x + y + z) & 1;
  return c * g.Nh + row * g.H + (x >> 1);
}

// Colour-split index of the neighbour of site s one step along axis mu (dir = +1/-1).
__device__ __forceinline__ int nbr_cs(const Geo &g, const SiteGeo &s, int mu, int dir) {
  const int base = (1 - s.c) * g.Nh;
  if (mu == 0) {
    int k2;
    if (dir > 0) k2 = s.xodd ? (s.k + 1 == g.H ? 0 : s.k + 1) : s.k;
    else k2 = s.xodd ? s.k : (s.k == 0 ? g.H - 1 : s.k - 1);
    return base + s.row * g.H + k2;
  }
  if (mu == 1) {
    int y2 = s.y + dir;
    y2 = y2 < 0 ? g.L1 - 1 : (y2 == g.L1 ? 0 : y2);
    return base + (y2 + g.L1 * s.z) * g.H + s.k;
  }
  int z2 = s.z + dir;
  z2 = z2 < 0 ? g.L2 - 1 : (z2 == g.L2 ? 0 : z2);
  return base + (s.y + g.L1 * z2) * g.H + s.k;
}

// In-warp 32x32 bit transpose: afterwards lane l holds bit i = (input of lane i, bit l).
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int j = 16 >> st;
    const uint32_t m = masks[st];
    const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, j);
    if (lane & j) x = (x & ~m) | ((y & ~m) >> j);
    else x = (x & m) | ((y & m) << j);
  }
  return x;
}

// r / d (d >= 1) for 0 <= r < 2^26 by a multiply-high with m = ceil((2^32 - 1) / d) (an estimate
// off by at most one) and one correction each way.
// div_magic(d) gives m.
__device__ __forceinline__ int div_by(int r, int d, uint32_t m) {
  int q = (int)__umulhi((uint32_t)r, m);
  q += (q + 1) * d <= r ? 1 : 0;
  q -= q * d > r ? 1 : 0;
  return q;
}
__host__ __device__ inline uint32_t div_magic(int d) {
  // d = 1: m = 2^32 - 1 gives r - 1 (r >= 1), which the upward correction makes r
  return d <= 1 ? 0xFFFFFFFFu : (uint32_t)((0xFFFFFFFFull + (unsigned)d) / (unsigned)d);
}

// Byte-table permutation of a word: out = OR over bytes of tab[byte index][byte value].
__device__ __forceinline__ uint32_t permute_word(const uint32_t *tab, uint32_t w) {
  return tab[w & 255u] | tab[256 + ((w >> 8) & 255u)] | tab[512 + ((w >> 16) & 255u)] | tab[768 + (w >> 24)];
}

// Bit-sliced full adder: sum and carry of three 32-lane bit planes.
__device__ __forceinline__ void fadd(uint32_t a, uint32_t b, uint32_t c, uint32_t &s, uint32_t &cy) {
  s = a ^ b ^ c;
  cy = (a & b) | (c & (a ^ b));
}

// ---------------------------------------------------------------------------------
// Replica exchange of one chain (Eq. 5), run by ONE thread: for k = 0..T-2 in order,
// delta = (beta_k - beta_k+1)(E_perm[k] - E_perm[k+1]); accept iff delta >= 0 or
// u 2^-32 < exp(delta), u the chain's Philox word for (k, t).  perm/slot/E may live in
// shared or global memory.  on_accept(k) and on_near() report to the caller.  The fp64
// arithmetic uses explicit round-to-nearest intrinsics so that no contraction can
// make it differ from the host oracle.
// ---------------------------------------------------------------------------------
template <class OnAccept, class OnNear>
__device__ __forceinline__ void exchange_chain(int T, const double *beta, int32_t *perm, int32_t *slot,
                                               const int32_t *E, uint32_t s_glob, uint32_t c,
                                               uint32_t t, uint32_t k0, uint32_t k1, OnAccept on_accept,
                                               OnNear on_near) {
  for (int k = 0; k + 1 < T; ++k) {
    const int a = perm[k], b = perm[k + 1];
    const double dbeta = __dsub_rn(beta[k], beta[k + 1]);
    const double delta = __dmul_rn(dbeta, (double)(E[a] - E[b]));
    bool accept;
    if (delta >= 0.0) {
      accept = true;
    } else {
      const uint32_t u = philox10((uint32_t)k, t, s_glob, (c << 20) | TAG_PT, k0, k1).x;
      const double x = __dmul_rn((double)u, 0x1p-32);
      const double e = exp(delta);
      if (fabs(__dsub_rn(x, e)) < 1e-12) on_near();
      accept = x < e;
    }
    if (accept) {
      on_accept(k);
      perm[k] = b;
      perm[k + 1] = a;
      slot[a] = k + 1;
      slot[b] = k;
    }
  }
}

} // namespace sgmc

namespace sgmc {

__host__ __device__ constexpr int round16(int x) { return (x + 15) & ~15; }

// Shared-memory map of the resident packed kernel: `wpc` 32-replica word lattices of one
// sample, its expanded couplings, per-lane threshold tables, energy partial sums and the
// per-chain exchange scratch.
// per chain (<= 64 replicas): perm, slot, E, accepts; near-threshold and exact-path
// counts; round-trip state (direction, start) and counters (an even count of words, so
// that each chain's 64-bit trip total stays 8-byte aligned)
constexpr int PT_WORDS = 6 * 64 + 8;
struct PackedSmem {
  int spin, jbyte, jpl, thr, epart, pt, bar, total;
};
// chains: the chain slots of the exchange state (default one per word; two when a CTA
// pairs the two chains' partial words of a sample).
__host__ __device__ inline PackedSmem packed_smem(int N, int NW, int d, int nthreads, int wpc, int chains = 0) {
  PackedSmem L;
  L.spin = 0;
  L.jbyte = L.spin + 4 * N * wpc;
  L.jpl = L.jbyte + round16(N);
  L.thr = L.jpl + round16(4 * d * NW);
  L.epart = L.thr + wpc * 256 * 8; // lane-pair threshold tables, 16 pairs x 16 codes x 8 bytes
  L.pt = L.epart + 4 * nthreads * wpc;
  L.bar = L.pt + round16(4 * PT_WORDS * (chains > 0 ? chains : wpc));
  L.total = L.bar + 16;
  return L;
}

constexpr int INT8_THK_MAX = 256;
// Shared-memory map of the resident int8 kernel (one chain, all its replicas).
struct Int8Smem {
  int spin, jbyte, jpl, thr, thk, eacc, pm, sl, pacc, near, xch, bar, total;
};
__host__ __device__ inline Int8Smem int8_smem(int N, int NW, int d, int T, int Tp) {
  Int8Smem L;
  L.spin = 0;
  L.jbyte = L.spin + round16(N * Tp);
  L.jpl = L.jbyte + round16(N);
  L.thr = L.jpl + round16(4 * d * NW);
  // the job's table by slot [T][4] for chains of up to 256 replicas, so that the refresh
  // after an exchange stays on chip (longer chains refresh from global memory)
  L.thk = L.thr + 16 * Tp;
  L.eacc = L.thk + (T <= INT8_THK_MAX ? 16 * T : 0);
  L.pm = L.eacc + round16(4 * Tp);
  L.sl = L.pm + round16(4 * T);
  L.pacc = L.sl + round16(4 * T);
  L.near = L.pacc + round16(4 * T);
  L.xch = L.near + 16; // warp exchange (T <= 64): its exact-path count
  L.bar = L.xch + 16;
  L.total = L.bar + 16;
  return L;
}

// Host-side launchers (each .cu file keeps its kernels to itself and exposes these).
// houd = 1: after the last sweep, the Houdayer q bitmaps and M of every pair into *hm;
// houd = 2 (energy-only after a move): first the cluster flips from *hm; houd = 3 (one
// MCS, fused): first the previous move's flips, the energies after it and the exchange,
// then the sweeps and the next move's q bitmaps.  All need a CTA that holds both
// one-word chains of a sample (wpc 2, two chains of T <= 32).
cudaError_t launch_resident(const Job &jb, const Dev &dv, bool int8fmt, int nthreads, int wpc, bool fuse_pt,
                            bool energy_only, size_t smem, cudaStream_t st, int n_mcs, int n_metro,
                            int32_t *meas_E = nullptr, int32_t *meas_Q = nullptr, bool after_move = false,
                            const HoudMaps *hm = nullptr, int houd = 0, bool allow_pair = false);
// Several jobs of the same lattice shape in one launch (chunks of MAX_BATCH_JOBS).
// jobs[i].n_items/fuse/n_metro must be filled; first_item is set here.
cudaError_t launch_resident_batch(JobDesc *jobs, int n_jobs, int nthreads, int wpc, size_t smem, cudaStream_t st,
                                  int n_mcs, bool pair = false);
cudaError_t launch_exchange(const Job &jb, const Dev &dv, cudaStream_t st);
// Paired last words (k_metro_pair.cu): the words per CTA (1: two chains of T <= 16 in one
// word; 3: two chains of 33..48 replicas, their full first words and one paired word) of
// a two-chain job whose sweeps run with the exchange fused, or 0 where pairing does not
// apply.  *nthreads is raised to the smallest CTA that has a warp per word and
// *smem set to the launch's shared memory, which must fit smem_limit.
int pair_words(const Job &jb, int *nthreads, int smem_limit, size_t *smem);
resident_fn1 pair_kernel_1(int d, int nthreads, int wpc);
resident_fnB pair_kernel_batch(int d, int nthreads, int wpc);
cudaError_t prepare_pair_kernels(int max_smem);
cudaError_t launch_exchange_batch(JobDesc *jobs, int n_jobs, cudaStream_t st);
cudaError_t prepare_resident_kernels(int max_smem);
cudaError_t prepare_houdayer_kernels(int max_smem);
cudaError_t launch_global_sweep(const Job &jb, const Dev &dv, uint2 *tables, uint32_t *esum, cudaStream_t st);
// Capacity of the allocation-free streaming sweep's static scratch: (sample, word) pairs,
// each a 2 KB lane-pair table and 128 bytes of bond sums (about 8.9 MB in all).
constexpr int STATIC_SWEEP_ITEMS = 4096;
constexpr size_t STATIC_SWEEP_TABLES = (size_t)STATIC_SWEEP_ITEMS * 256 * 8;
constexpr size_t STATIC_SWEEP_BYTES = STATIC_SWEEP_TABLES + (size_t)STATIC_SWEEP_ITEMS * 32 * 4;
cudaError_t static_sweep_scratch(void **ptr);
cudaError_t launch_global_energy(const Job &jb, const Dev &dv, uint2 *tables, uint32_t *esum, cudaStream_t st);
int houdayer_smem(const Job &jb, int bitmaps_smem);
size_t houdayer_scratch_bytes(const Job &jb);
// Whether the labelling kernel (and so the multi-cluster variant) runs for this lattice.
bool houdayer_labels(const Job &jb);
// fused: the sweep launch before wrote the q bitmaps and M, and the energy launch after
// applies the flips (launch_resident houd = 1 / 2), so only the cluster phase runs here.
cudaError_t launch_houdayer(const Job &jb, const Dev &dv, uint32_t *scratch, int smem_limit, bool multi,
                            cudaStream_t st, bool fused = false);
// The bitmap scratch layout of the split form inside `scratch`.
HoudMaps houd_maps_of(const Job &jb, uint32_t *scratch);
} // namespace sgmc

namespace sgmc {
cudaError_t launch_init(const Job &jb, const Dev &dv, bool int8fmt, cudaStream_t st);
cudaError_t launch_export_spins(const Job &jb, const Dev &dv, bool int8fmt, uint8_t *out, cudaStream_t st);
cudaError_t launch_import_spins(const Job &jb, const Dev &dv, bool int8fmt, const uint8_t *in, cudaStream_t st);
cudaError_t launch_export_couplings(const Job &jb, const Dev &dv, int8_t *out, cudaStream_t st);
cudaError_t launch_import_couplings(const Job &jb, const Dev &dv, const int8_t *in, cudaStream_t st);
cudaError_t launch_measure(const Job &jb, const Dev &dv, bool int8fmt, int32_t *E_out, int32_t *Q_out,
                           cudaStream_t st);
// Overlap plane sums [S][T][d][Lmax] (Lmax = qmodes_lmax); needs C >= 2.
int qmodes_lmax(const Job &jb);
cudaError_t launch_qmodes(const Job &jb, const Dev &dv, bool int8fmt, int32_t *P_out, cudaStream_t st);
cudaError_t prepare_state_kernels(int max_smem);
// A bounded wait that runs out by design (failure detection self-test).
cudaError_t launch_wait_selftest(const Dev &dv, uint32_t max_tries, cudaStream_t st);
// General couplings (k_gauss.cu).
size_t gauss_smem_bytes(const Job &jb);
cudaError_t launch_gauss(const Job &jb, const Dev &dv, bool fuse_pt, bool energy_only, cudaStream_t st, int n_mcs,
                         int n_metro);
cudaError_t launch_gauss_import(const Job &jb, const Dev &dv, const int32_t *stage, cudaStream_t st);
cudaError_t launch_gather_energy64(const Job &jb, const Dev &dv, long long *E_out, cudaStream_t st);
cudaError_t prepare_gauss_kernels(int max_smem);
} // namespace sgmc
