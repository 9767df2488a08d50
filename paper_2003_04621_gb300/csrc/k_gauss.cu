// k_gauss.cu -- Metropolis sweeps, energies and the replica exchange for general
// couplings (Sec. 2.1: e.g. drawn from a standard normal distribution), int8 spins (one
// replica per byte, the paper's layout, Sec. 3).
//
// Couplings are fixed point in units of 2^-20, so every local field, energy change and
// energy is an exact integer and no sum depends on its order.  The Metropolis threshold
// for a change dE > 0 is floor(e 2^32), e an fp32 evaluation of exp(-beta dE) written out
// below with single IEEE adds and multiplies in a fixed order (Cody & Waite's reduction
// by ln 2 and a Taylor series to r^6): a fixed, portable function, so every IEEE
// implementation reproduces each decision bit for bit.  The exchange is Eq. 5 in fp64 on
// the exact energies.
//
// One CTA owns one chain (sample s, chain c) for the whole launch: its spins [N][Tp]
// (colour-split site order) and the sample's couplings [d][N] are bulk-copied into shared
// memory; a thread item is (site of the colour, group of four replicas), one Philox call.
#include "sgmc_internal.cuh"
#include "sgmc_tma.cuh"

namespace sgmc {

namespace {

// exp(x) for -23 <= x <= 0: x = k ln2 + r, k = floor(x / ln2 + 1/2), ln 2 = ln2_hi + ln2_lo
// (ln2_hi has 16 significant bits, so k ln2_hi is exact); exp(r) by its Taylor series to
// r^6 in Horner form; times 2^k built from its exponent bits (k in [-34, 0]).
__device__ __forceinline__ float gauss_exp(float x) {
  const float kf = floorf(__fadd_rn(__fmul_rn(x, 0x1.715476p+0f), 0.5f));
  const int k = (int)kf;
  float r = __fsub_rn(x, __fmul_rn(kf, 0x1.62e4p-1f));
  r = __fsub_rn(r, __fmul_rn(kf, 0x1.7f7d1cp-20f));
  float p = 0x1.6c16c2p-10f;                      // 1/720
  p = __fadd_rn(__fmul_rn(p, r), 0x1.111112p-7f); // 1/120
  p = __fadd_rn(__fmul_rn(p, r), 0x1.555556p-5f); // 1/24
  p = __fadd_rn(__fmul_rn(p, r), 0x1.555556p-3f); // 1/6
  p = __fadd_rn(__fmul_rn(p, r), 0.5f);
  p = __fadd_rn(__fmul_rn(p, r), 1.0f);
  p = __fadd_rn(__fmul_rn(p, r), 1.0f);
  return __fmul_rn(p, __int_as_float((k + 127) << 23));
}

// floor(exp(-beta dE 2^-20) 2^32) in fp32 (2^32 - 1 where e rounds to 1; 0 below
// x = -23, where it would be below 1 anyway).
__device__ __forceinline__ uint32_t gauss_threshold(float beta, int dE) {
  const float xs = __fmul_rn(__int2float_rn(dE), 0x1p-20f);
  const float x = -__fmul_rn(beta, xs);
  if (x < -23.0f) return 0u;
  const float e = gauss_exp(x);
  if (e >= 1.0f) return 0xFFFFFFFFu;
  return __float2uint_rz(__fmul_rn(e, 4294967296.0f));
}

// The Metropolis decision r < gauss_threshold(beta, dE) for dE > 0, decided first against
// the hardware exponential.  __expf's documented error is at most 2 + floor(1.16 |x|)
// ulp, under 3.4e-6 relative on [-23, 0]; gauss_exp is within 2e-6 of exp (a pinned
// bound); fp32 r and the products add about 2e-7.  So for r below e_a 2^32 (1 - 2^-14) or
// above e_a 2^32 (1 + 2^-14), e_a = __expf(x), the exact threshold gives the same answer
// with a margin above ten times the error.  Only draws inside that band (a fraction of
// about 1e-4) evaluate gauss_threshold.  Below x = -23 the exact threshold is 0: no draw
// is accepted.
// Returns 1 (accept: dE <= 0, or r clearly below), -1 (reject) or 0 (r inside the band:
// the caller evaluates r < gauss_threshold(beta, dE)).
__device__ __forceinline__ int gauss_fast(float beta, int dE, uint32_t r) {
  const float xs = __fmul_rn(__int2float_rn(dE), 0x1p-20f);
  const float x = -__fmul_rn(beta, xs);
  const float ea = __fmul_rn(__expf(x), 4294967296.0f);
  const float rf = __uint2float_rn(r);
  const bool dead = x < -23.0f; // the exact threshold is 0 there
  const bool lo = !dead && rf < __fmul_rn(ea, 1.0f - 0x1p-14f);
  const bool hi = dead || rf > __fmul_rn(ea, 1.0f + 0x1p-14f);
  return (dE <= 0 || lo) ? 1 : (hi ? -1 : 0);
}

__device__ __forceinline__ uint32_t word_of4(const uint4 &r, int i) {
  return i == 0 ? r.x : (i == 1 ? r.y : (i == 2 ? r.z : r.w));
}

// Shared-memory map: spins, couplings, per-replica beta and energy sums, the chain's maps.
struct GaussSmem {
  int spin, jfix, betaf, eacc, pm, sl, pacc, accb, rejb, uw, slow, near, bar, total;
};
__host__ __device__ inline GaussSmem gauss_smem(int N, int d, int T, int Tp) {
  GaussSmem L;
  L.spin = 0;
  L.jfix = round16(N * Tp);
  L.betaf = L.jfix + round16(4 * d * N);
  L.eacc = L.betaf + round16(4 * Tp);
  L.pm = L.eacc + round16(8 * Tp);
  L.sl = L.pm + round16(4 * T);
  L.pacc = L.sl + round16(4 * T);
  L.accb = L.pacc + round16(4 * T); // exchange bounds, words and slow flags per pair
  L.rejb = L.accb + round16(8 * T);
  L.uw = L.rejb + round16(8 * T);
  L.slow = L.uw + round16(4 * T);
  L.near = L.slow + round16(T);
  L.bar = L.near + 16;
  L.total = L.bar + 16;
  return L;
}

// Replica exchange of one chain (Eq. 5) on int64 fixed-point energies, by one warp.  The
// lanes first draw every pair's word u_k and turn the exact fp64 test into integer bounds
// on dE = E_k - E_k+1 (fixed point) that are safe by a wide margin; the sequential pass
// over k = 0..T-2 (lane 0) then compares integers, and only a decision inside the margin
// (or u = 0) takes the exact path with the fp64 exp.  With x = u 2^-32 and
// dbeta = beta_k - beta_k+1 > 0, the rule "accept iff delta >= 0 or x < exp(delta)",
// delta = dbeta dE 2^-20, is for dE < 0 "dE 2^-20 > theta", theta = ln(x) / dbeta.  In
// fp32, theta is within 5e-7 |theta| and the margin mg = max(4e-6 (1 + |theta|),
// 1e-10 / (dbeta x)) covers that error many times, so dE 2^-20 >= theta + mg implies
// exp(delta) >= x + 5e-11 and dE 2^-20 <= theta - mg implies x - exp(delta) >= 2.5e-11: both
// agree with the fp64 test and lie outside the 1e-12 near-threshold window.  The bounds
// are scaled by 2^20 and rounded outwards to integers (|theta| 2^20 < 2^62).
__device__ void exchange_chain64_warp(int T, const double *beta, int32_t *perm, int32_t *slot, const long long *E,
                                      long long *accb, long long *rejb, uint32_t *uw, uint8_t *slow,
                                      uint32_t s_glob, uint32_t c, uint32_t t, uint32_t k0, uint32_t k1,
                                      unsigned int *pacc, unsigned int *pnear, unsigned int *pexact) {
  const int lane = threadIdx.x & 31;
  for (int k = lane; k + 1 < T; k += 32) {
    const uint32_t u = philox10((uint32_t)k, t, s_glob, (c << 20) | TAG_PT, k0, k1).x;
    const float dbeta = (float)__dsub_rn(beta[k], beta[k + 1]);
    bool sl = u == 0u;
    long long A = 0, R = 0;
    if (!sl) {
      const float x = (float)u * 0x1p-32f;
      const float lnx = u > 0x80000000u ? log1pf(-(float)(0u - u) * 0x1p-32f) : logf(x);
      const float theta = lnx / dbeta;
      const float mg = fmaxf(4e-6f * (1.0f + fabsf(theta)), 1e-10f / (dbeta * x));
      const float hi = (theta + mg) * 1048576.0f, lo = (theta - mg) * 1048576.0f;
      const float LIM = 4.0e18f;
      if (!(hi == hi) || !(lo == lo) || fabsf(hi) >= LIM || fabsf(lo) >= LIM) {
        sl = true;
      } else {
        A = (long long)ceilf(hi);
        R = (long long)floorf(lo);
      }
    }
    accb[k] = A;
    rejb[k] = R;
    uw[k] = u;
    slow[k] = sl ? 1 : 0;
  }
  __syncwarp();
  if (lane == 0) {
    for (int k = 0; k + 1 < T; ++k) {
      const int a = perm[k], b = perm[k + 1];
      const long long dE = E[a] - E[b];
      bool accept;
      if (dE >= 0) {
        accept = true;
      } else if (!slow[k] && dE >= accb[k]) {
        accept = true;
      } else if (!slow[k] && dE <= rejb[k]) {
        accept = false;
      } else {
        const double dbeta = __dsub_rn(beta[k], beta[k + 1]);
        const double delta = __dmul_rn(dbeta, __dmul_rn((double)dE, 0x1p-20));
        const double x = __dmul_rn((double)uw[k], 0x1p-32);
        const double e = exp(delta);
        if (fabs(__dsub_rn(x, e)) < 1e-12) *pnear += 1u;
        *pexact += 1u;
        accept = x < e;
      }
      if (accept) {
        pacc[k] += 1u;
        perm[k] = b;
        perm[k + 1] = a;
        slot[a] = k + 1;
        slot[b] = k;
      }
    }
  }
  __syncwarp();
}

constexpr int GNT = 128;

template <int D, bool FUSE_PT, bool ENERGY_ONLY>
__global__ void __launch_bounds__(GNT) k_gauss_int8(Job jb, Dev dv, int n_mcs, int n_metro) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Geo g = jb.g;
  const int T = jb.T, Tp = jb.Tp, G = Tp / 4, N = g.N;
  const GaussSmem L = gauss_smem(N, D, T, Tp);
  int8_t *sp8 = reinterpret_cast<int8_t *>(smem + L.spin);
  int32_t *jf = reinterpret_cast<int32_t *>(smem + L.jfix); // [D][N], forward bond (i, mu) at p(i)
  float *betaf = reinterpret_cast<float *>(smem + L.betaf);  // [Tp] beta of each replica's slot
  unsigned long long *eacc = reinterpret_cast<unsigned long long *>(smem + L.eacc);
  int32_t *pm = reinterpret_cast<int32_t *>(smem + L.pm);
  int32_t *sl = reinterpret_cast<int32_t *>(smem + L.sl);
  unsigned int *pacc = reinterpret_cast<unsigned int *>(smem + L.pacc);
  unsigned int *pnear = reinterpret_cast<unsigned int *>(smem + L.near);
  unsigned int *pexact = pnear + 1; // exchange decisions by the exact test
  unsigned int *pband = pnear + 2;  // Metropolis draws inside the screening band
  long long *accb = reinterpret_cast<long long *>(smem + L.accb);
  long long *rejb = reinterpret_cast<long long *>(smem + L.rejb);
  uint32_t *uw = reinterpret_cast<uint32_t *>(smem + L.uw);
  uint8_t *slowf = smem + L.slow;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);

  const int tid = threadIdx.x;
  const uint32_t t_metro0 = (uint32_t)dv.ctr[CTR_TMETRO], t_pt0 = (uint32_t)dv.ctr[CTR_TPT];
  const unsigned long long adv_metro = ENERGY_ONLY ? 0ull : (unsigned long long)n_mcs * n_metro;
  const unsigned long long adv_pt = FUSE_PT ? (unsigned long long)n_mcs : 0ull;
  const int s = blockIdx.x / jb.C;
  const int c = blockIdx.x - s * jb.C;
  const uint32_t s_glob = (uint32_t)(jb.s_off + s);
  int8_t *gsp = reinterpret_cast<int8_t *>(dv.spins) + ((size_t)s * jb.C + c) * N * Tp;
  const int32_t *gj = dv.jfix + (size_t)s * D * N;
  const size_t chain_base = ((size_t)s * jb.C + c) * T;

  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  if (tid == 0) {
    const uint32_t sbytes = (uint32_t)(N * Tp), jbytes = 4u * (uint32_t)(D * N);
    mbar_expect_tx(bar, sbytes + jbytes);
    bulk_g2s(sp8, gsp, sbytes, bar);
    bulk_g2s(jf, gj, jbytes, bar);
  }
  for (int j = tid; j < T; j += GNT) {
    pm[j] = dv.perm[chain_base + j];
    sl[j] = dv.slot[chain_base + j];
    pacc[j] = 0u;
  }
  if (tid == 0) {
    *pnear = 0u;
    *pexact = 0u;
    *pband = 0u;
  }
  __syncthreads();
  for (int j = tid; j < Tp; j += GNT) betaf[j] = j < T ? __double2float_rn(dv.beta[sl[j]]) : 0.0f;
  const bool ok = mbar_wait(bar, 0, MBAR_MAX_TRIES);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      atomicOr(&dv.ctr[CTR_ERROR], ERR_TMA_TIMEOUT);
      mbar_wait(bar, 0, MBAR_MAX_TRIES);
    }
    grid_done_advance(dv.ctr, adv_metro, adv_pt, 0ull);
    return;
  }

  const int H = g.H, L1 = g.L1, Nh = g.Nh;
  const uint32_t mH = div_magic(H), mL1 = div_magic(L1 < 2 ? 2 : L1);
  // when G divides the CTA, a thread keeps one replica group gi = tid % G and walks the
  // sites q = tid / G, tid / G + GNT / G, ...; its energy terms stay in registers and are
  // summed over the warp's lanes of the same group before one shared add each
  const bool fixed_g = (GNT % G) == 0;
  uint32_t nband = 0u; // this thread's draws that took the exact threshold
  const int n_outer = ENERGY_ONLY ? 1 : n_mcs;
  const int n_inner = ENERGY_ONLY ? 1 : n_metro;
  for (int m = 0; m < n_outer; ++m) {
    for (int swp = 0; swp < n_inner; ++swp) {
      const uint32_t t = t_metro0 + (uint32_t)(m * n_metro + swp);
      for (int col = ENERGY_ONLY ? 1 : 0; col < 2; ++col) {
        if (col == 1) {
          for (int j = tid; j < Tp; j += GNT) eacc[j] = 0ull;
          __syncthreads();
        }
        long long el[4] = {0, 0, 0, 0};
        const int gfix = fixed_g ? tid % G : 0, qstep = fixed_g ? GNT / G : 0;
        int qf = fixed_g ? tid / G : 0;
        for (int it = tid; it < Nh * G; it += GNT, qf += qstep) {
          const int q = fixed_g ? qf : it / G;
          const int gi = fixed_g ? gfix : it - q * G;
          SiteGeo sg;
          sg.c = col;
          sg.row = div_by(q, H, mH);
          sg.k = q - sg.row * H;
          sg.z = D == 3 ? div_by(sg.row, L1, mL1) : 0;
          sg.y = D == 3 ? sg.row - sg.z * L1 : sg.row;
          sg.xodd = col ^ ((sg.y + sg.z) & 1);
          const int p = col * Nh + q;
          char4 s4 = *reinterpret_cast<const char4 *>(sp8 + (size_t)p * Tp + 4 * gi);
          int h[4] = {0, 0, 0, 0};
#pragma unroll
          for (int mu = 0; mu < D; ++mu) {
            const int pf = nbr_cs(g, sg, mu, 1), pb = nbr_cs(g, sg, mu, -1);
            const int Jf = jf[mu * N + p], Jb = jf[mu * N + pb];
            const char4 nf = *reinterpret_cast<const char4 *>(sp8 + (size_t)pf * Tp + 4 * gi);
            const char4 nb = *reinterpret_cast<const char4 *>(sp8 + (size_t)pb * Tp + 4 * gi);
            h[0] += Jf * nf.x + Jb * nb.x;
            h[1] += Jf * nf.y + Jb * nb.y;
            h[2] += Jf * nf.z + Jb * nb.z;
            h[3] += Jf * nf.w + Jb * nb.w;
          }
          int sv[4] = {s4.x, s4.y, s4.z, s4.w};
          if (!ENERGY_ONLY) {
            const uint32_t i = (uint32_t)(g.L0 * sg.row + 2 * sg.k + sg.xodd);
            const uint4 rnd =
                philox10(i, t, s_glob, ((uint32_t)c << 20) | ((uint32_t)gi << 8) | TAG_METRO, jb.sk0, jb.sk1);
            // decisions without branches; the rare draws near the threshold take the exact
            // test afterwards
            uint32_t acc = 0u, near = 0u;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const int dE = 2 * sv[r] * h[r];
              const int f = gauss_fast(betaf[4 * gi + r], dE, word_of4(rnd, r));
              acc |= (f > 0 ? 1u : 0u) << r;
              near |= (f == 0 ? 1u : 0u) << r;
            }
            if (near) {
              nband += __popc(near & (T - 4 * gi >= 4 ? 0xFu : ((1u << (T - 4 * gi)) - 1u)));
#pragma unroll
              for (int r = 0; r < 4; ++r)
                if ((near >> r) & 1u)
                  acc |= (word_of4(rnd, r) < gauss_threshold(betaf[4 * gi + r], 2 * sv[r] * h[r]) ? 1u : 0u) << r;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
              if (4 * gi + r < T && ((acc >> r) & 1u)) sv[r] = -sv[r];
            s4 = make_char4((signed char)sv[0], (signed char)sv[1], (signed char)sv[2], (signed char)sv[3]);
            *reinterpret_cast<char4 *>(sp8 + (size_t)p * Tp + 4 * gi) = s4;
          }
          if (col == 1) {
            // every bond has exactly one colour-1 end: E = -sum over colour-1 sites of s h
            if (fixed_g) {
#pragma unroll
              for (int r = 0; r < 4; ++r) el[r] -= (long long)sv[r] * h[r];
            } else {
#pragma unroll
              for (int r = 0; r < 4; ++r)
                if (4 * gi + r < T) atomicAdd(&eacc[4 * gi + r], (unsigned long long)(-(long long)sv[r] * h[r]));
            }
          }
        }
        if (col == 1 && fixed_g) {
          // lanes l and l ^ o hold the same group for o a multiple of G (G | 32), else
          // every lane of the warp has its own group
          if (G < 32)
            for (int o = 16; o >= G; o >>= 1)
#pragma unroll
              for (int r = 0; r < 4; ++r) el[r] += __shfl_xor_sync(0xFFFFFFFFu, el[r], o);
          if ((tid & 31) < G || G >= 32)
#pragma unroll
            for (int r = 0; r < 4; ++r)
              if (4 * gfix + r < T && el[r]) atomicAdd(&eacc[4 * gfix + r], (unsigned long long)el[r]);
        }
        __syncthreads();
      }
    }
    if (FUSE_PT) {
      if (tid < 32) {
        exchange_chain64_warp(T, dv.beta, pm, sl, reinterpret_cast<const long long *>(eacc), accb, rejb, uw, slowf,
                              s_glob, (uint32_t)c, t_pt0 + (uint32_t)m, jb.sk0, jb.sk1, pacc, pnear, pexact);
        if (tid == 0) trip_chain(dv, (size_t)s * jb.C + c, T, sl, t_pt0 + (uint32_t)m + 1u);
      }
      __syncthreads();
      if (!ENERGY_ONLY)
        for (int j = tid; j < T; j += GNT) betaf[j] = __double2float_rn(dv.beta[sl[j]]);
      __syncthreads();
    }
  }

  for (int j = tid; j < T; j += GNT) {
    dv.E64[chain_base + j] = (long long)eacc[j];
    if (FUSE_PT) {
      dv.perm[chain_base + j] = pm[j];
      dv.slot[chain_base + j] = sl[j];
      if (j + 1 < T && pacc[j]) atomicAdd(&dv.ctr[CTR_PT + j], (unsigned long long)pacc[j]);
    }
  }
  nband = __reduce_add_sync(0xFFFFFFFFu, nband);
  if ((tid & 31) == 0 && nband) atomicAdd(pband, nband);
  __syncthreads();
  if (FUSE_PT && tid == 0 && *pnear) atomicAdd(&dv.ctr[CTR_NEAR], (unsigned long long)*pnear);
  if (FUSE_PT && tid == 0 && *pexact) atomicAdd(&dv.ctr[CTR_XEXACT], (unsigned long long)*pexact);
  if (tid == 0 && *pband) atomicAdd(&dv.ctr[CTR_GBAND], (unsigned long long)*pband);
  if (!ENERGY_ONLY) {
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) bulk_s2g_and_release(gsp, sp8, (uint32_t)(N * Tp));
  }
  grid_done_advance(dv.ctr, adv_metro, adv_pt, 0ull);
}

// Canonical [S][N][d] fixed-point couplings -> the device layout [S][d][N] (colour-split).
__global__ void k_gauss_import(Job jb, Dev dv, const int32_t *stage) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int N = jb.g.N, d = jb.g.d;
  if (idx >= (long long)jb.S * N * d) return;
  const int mu = (int)(idx % d);
  const int i = (int)((idx / d) % N);
  const int s = (int)(idx / ((long long)N * d));
  dv.jfix[((size_t)s * d + mu) * N + cs_of_canonical(jb.g, i)] = stage[idx];
}

// E by temperature slot, int64.
__global__ void k_gather_energy64(Job jb, Dev dv, long long *E_out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)jb.S * jb.C * jb.T) return;
  const long long base = idx - idx % jb.T;
  E_out[idx] = dv.E64[base + dv.perm[idx]];
}

typedef void (*gauss_fn)(Job, Dev, int, int);
template <bool FUSE, bool EONLY>
gauss_fn pick_gauss(int d) {
  return d == 2 ? k_gauss_int8<2, FUSE, EONLY> : k_gauss_int8<3, FUSE, EONLY>;
}

} // namespace

size_t gauss_smem_bytes(const Job &jb) { return (size_t)gauss_smem(jb.g.N, jb.g.d, jb.T, jb.Tp).total; }

cudaError_t launch_gauss(const Job &jb, const Dev &dv, bool fuse_pt, bool energy_only, cudaStream_t st, int n_mcs,
                         int n_metro) {
  gauss_fn fn;
  if (energy_only && fuse_pt) fn = pick_gauss<true, true>(jb.g.d);
  else if (energy_only) fn = pick_gauss<false, true>(jb.g.d);
  else if (fuse_pt) fn = pick_gauss<true, false>(jb.g.d);
  else fn = pick_gauss<false, false>(jb.g.d);
  fn<<<(unsigned)(jb.S * jb.C), GNT, gauss_smem_bytes(jb), st>>>(jb, dv, n_mcs, n_metro);
  return cudaGetLastError();
}

cudaError_t launch_gauss_import(const Job &jb, const Dev &dv, const int32_t *stage, cudaStream_t st) {
  const long long n = (long long)jb.S * jb.g.N * jb.g.d;
  k_gauss_import<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(jb, dv, stage);
  return cudaGetLastError();
}

cudaError_t launch_gather_energy64(const Job &jb, const Dev &dv, long long *E_out, cudaStream_t st) {
  const long long n = (long long)jb.S * jb.C * jb.T;
  k_gather_energy64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(jb, dv, E_out);
  return cudaGetLastError();
}

cudaError_t prepare_gauss_kernels(int max_smem) {
  const void *fns[8] = {(const void *)pick_gauss<false, false>(2), (const void *)pick_gauss<true, false>(2),
                        (const void *)pick_gauss<false, true>(2),  (const void *)pick_gauss<true, true>(2),
                        (const void *)pick_gauss<false, false>(3), (const void *)pick_gauss<true, false>(3),
                        (const void *)pick_gauss<false, true>(3),  (const void *)pick_gauss<true, true>(3)};
  for (const void *fn : fns) {
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

} // namespace sgmc
