// sgmc_resident.cuh -- the resident packed-spin sweep kernel (Sec. 2.2 / 2.4 step 1) with
// the energy (Eq. 1) and, when a chain fits in one CTA, the replica exchange (Eq. 5)
// fused in, as a template that k_metro.cu and k_metro_pair.cu instantiate.
//
// Packed kernel: one CTA owns WPC 32-replica word lattices of one sample (usually both
// one-word chains) for the whole launch.  TMA bulk-copies the N words and the sample's
// coupling bit planes into shared memory, runs n_mcs x n_metro checkerboard sweeps there
// (colour 0 then colour 1, each site updating its 32 replicas at once), keeps the
// energies exact, optionally performs the chains' exchange passes between MCS, and
// bulk-copies the lattice back.  Template flags add the fused measurement (MEAS), leave
// out the partial-word code (FULLW), take phases of the Houdayer move (HOUD) or pair the
// two chains' partial last words in one word (PAIR); see the kernel's comment.
// The sweep is integer-only: per site, 2d unsatisfied-bond planes
// (s_i ^ s_nb ^ J), a bit-sliced count u of them per replica (lane), auto-accept where
// u >= d (dE = 4(d - u) <= 0), else accept iff the replica's Philox word is below
// thr[T(replica)][d - u].  One Philox4x32-10 call serves four replicas of a site.
//
// Energies: every bond has exactly one colour-1 end, so after the colour-1 half-sweep
// the number U of unsatisfied bonds of each replica is the sum over colour-1 sites of
// their (post-update) unsatisfied count; E = 2U - dN.  The sums are kept as bit-sliced
// vertical counters per thread and reduced across the CTA once per sweep, so E is
// recomputed exactly every sweep instead of being accumulated from flips.
#pragma once
#include "sgmc_houd.cuh"
#include "sgmc_internal.cuh"
#include "sgmc_sweep.cuh"
#include "sgmc_tma.cuh"

namespace sgmc {

// Expand the sample's coupling bit planes into one byte per site with the 2d bonds of
// the site: bit 2 mu = forward bond (i, mu), bit 2 mu + 1 = backward bond (i - e_mu, mu).
template <int D, int NT>
__device__ __forceinline__ void expand_couplings(const Geo &g, const uint32_t *jpl, uint8_t *jbyte) {
  for (int p = threadIdx.x; p < g.N; p += NT) {
    const SiteGeo s = site_geo(g, p);
    uint32_t b = 0;
#pragma unroll
    for (int mu = 0; mu < D; ++mu) {
      const uint32_t *pl = jpl + mu * g.NW;
      b |= ((pl[p >> 5] >> (p & 31)) & 1u) << (2 * mu);
      const int qn = nbr_cs(g, s, mu, -1);
      b |= ((pl[qn >> 5] >> (qn & 31)) & 1u) << (2 * mu + 1);
    }
    jbyte[p] = (uint8_t)b;
  }
}

// One checkerboard half-sweep over the colour-`col` sites of WPC resident word lattices
// (all of one sample).  Site geometry, couplings and the site-level Philox parts are
// shared by the WPC words.  `accum` adds each site's post-update count to V[w] (a
// run-time flag, so that both colours run one copy of the code); NOFLIP counts only.
// PAIR: the last word pairs two chains' partial words (decide_pair), the others are full.
template <int D, int NT, int WPC, bool NOFLIP, bool FULLW, bool PAIR>
__device__ __forceinline__ void half_sweep(const Geo &g, int col, bool accum, uint32_t *__restrict__ sp,
                                           const uint8_t *__restrict__ jbyte,
                                           const uint2 *__restrict__ pair_tab, const uint32_t *vmask,
                                           const int *ngroups, const uint32_t *c3base, const PhiloxSweep &P,
                                           const Job &jb, uint32_t (&V)[WPC][NB], int wcount = WPC) {
  const int H = g.H, L1 = g.L1, Nh = g.Nh, N = g.N;
  // q / H and row / L1 as a multiply-high by ceil(2^32 / divisor) (division by an
  // invariant integer, Granlund and Montgomery 1994): exact while the dividend times the
  // divisor stays below 2^32, which holds for every lattice that fits in shared memory
  const uint32_t mH = H > 1 ? 0xFFFFFFFFu / (uint32_t)H + 1u : 0u;
  const uint32_t mL1 = L1 > 1 ? 0xFFFFFFFFu / (uint32_t)L1 + 1u : 0u;
  for (int q = threadIdx.x; q < Nh; q += NT) {
    const int row = H > 1 ? (int)__umulhi((uint32_t)q, mH) : q;
    const int k = q - row * H;
    int y, z;
    if (D == 3) {
      z = L1 > 1 ? (int)__umulhi((uint32_t)row, mL1) : row;
      y = row - z * L1;
    } else {
      y = row;
      z = 0;
    }
    const int xodd = col ^ ((y + z) & 1);
    const int rb = row * H;
    int nidx[2 * D];
    nidx[0] = rb + (xodd ? (k + 1 == H ? 0 : k + 1) : k);
    nidx[1] = rb + (xodd ? k : (k == 0 ? H - 1 : k - 1));
    nidx[2] = ((y + 1 == L1) ? row - (L1 - 1) : row + 1) * H + k;
    nidx[3] = ((y == 0) ? row + (L1 - 1) : row - 1) * H + k;
    if (D == 3) {
      const int L2 = g.L2;
      nidx[4] = ((z + 1 == L2) ? row - (L2 - 1) * L1 : row + L1) * H + k;
      nidx[5] = ((z == 0) ? row + (L2 - 1) * L1 : row - L1) * H + k;
    }
    const uint32_t jsite = jbyte[col * Nh + q];
    uint32_t jm[2 * D];
#pragma unroll
    for (int b = 0; b < 2 * D; ++b) jm[b] = 0u - ((jsite >> b) & 1u);
    PhiloxSite Q;
    if (!NOFLIP) Q = philox_site(P, (uint32_t)(g.L0 * row + 2 * k + xodd), jb);
#pragma unroll
    for (int w = 0; w < WPC; ++w) {
      if (NOFLIP && w >= wcount) continue; // counting only the first wcount words
      uint32_t *own = sp + w * N + col * Nh;
      const uint32_t *oth = sp + w * N + (1 - col) * Nh;
      uint32_t nb[2 * D];
#pragma unroll
      for (int b = 0; b < 2 * D; ++b) nb[b] = oth[nidx[b]];
      const uint32_t s0 = own[q];
      const SiteCount<D> cnt = count_site<D>(s0, nb, jm);
      uint32_t F = 0;
      if (!NOFLIP) {
        if (PAIR && w == WPC - 1) // the two chains' paired last words
          F = decide_pair<D>(cnt, P, Q, c3base[w], ngroups[w], pair_tab + w * 256, jb) & vmask[w];
        else // (with paired last words every other word is full)
          F = decide_site<D, FULLW || PAIR>(cnt, P, Q, c3base[w], ngroups[w], pair_tab + w * 256, jb) & vmask[w];
        own[q] = s0 ^ F;
      }
      if (accum) {
        uint32_t v1, v2;
        recount<D>(cnt, F, v1, v2);
        vcount_add(V[w], cnt.u0, v1, v2);
      }
    }
  }
}

// Replica exchange of one chain (T <= 64) from shared memory (Eq. 5), by one warp.  The
// lanes first draw every pair's word u_k and turn the exact fp64 test into integer bounds
// on dE = E_k - E_k+1 that are safe by a wide margin (see below); the sequential pass over
// k = 0..T-2 then compares integers, and only a decision inside the margin (or u = 0)
// takes the exact path with exp, identical to the standalone kernel and to the oracle.
//
// Bounds: with x = u 2^-32 and dbeta = beta_k - beta_k+1 > 0, delta = dbeta dE and the
// exact rule "accept iff delta >= 0 or x < exp(delta)" is, for dE < 0, "dE > ln(x)/dbeta".
// With theta = ln(x)/dbeta and margin mg = max(4e-6 (1 + |theta|), 1e-10/(dbeta x)),
// evaluated in fp32 (theta's error is below mg/8): dE >= theta + mg gives
// exp(delta) >= x exp(1e-10/(2x)) >= x + 5e-11, and dE <= theta - mg gives
// x - exp(delta) >= 2.5e-11, so both fast outcomes agree with the fp64 test and are
// never within the 1e-12 near-threshold window, whatever the last-bit errors of exp and
// the products.
//
// The pass: at step k the pair is (replica now at slot k, replica at slot k+1), and the
// replica at slot k+1 is still the one from before the pass.  So the replica that may keep
// climbing and its energy are carried in registers, and the other operands of step k
// (the replica at slot k+1, its energy, the bounds of pair k) come from the lanes that
// hold them by shuffles that do not depend on earlier decisions.  Every lane runs the pass
// (same values, same branches); lane k % 32 keeps the replica that ends at slot k.
// pacc, pnear and pexact accumulate; pm and sl are rewritten at the end.
__device__ __forceinline__ void exchange_chain_smem(int T, const double *beta, int32_t *pm, int32_t *sl,
                                                    const int32_t *el, unsigned int *pacc, unsigned int *pnear,
                                                    unsigned int *pexact, uint32_t s_glob, uint32_t c, uint32_t t,
                                                    const Job &jb) {
  const int lane = threadIdx.x & 31;
  int Ar[2] = {0, 0}, Rr[2] = {0, 0};
  uint32_t ur[2] = {0u, 0u}, slowm[2] = {0u, 0u};
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int k = lane + 32 * half;
    bool slow = false;
    if (k + 1 < T) {
      const uint32_t u = philox10_rk((uint32_t)k, t, s_glob, (c << 20) | TAG_PT, jb.rk0, jb.rk1).x;
      const float dbeta = (float)__dsub_rn(beta[k], beta[k + 1]);
      slow = (u == 0u);
      if (!slow) {
        // bounds in fp32: ln x to ~3e-7 relative (log1p near x = 1, where 1 - x is exact),
        // dbeta to 6e-8, so theta is within 5e-7 |theta| and the margin covers it 8 times
        const float x = (float)u * 0x1p-32f;
        const float lnx = u > 0x80000000u ? log1pf(-(float)(0u - u) * 0x1p-32f) : logf(x);
        const float theta = lnx / dbeta;
        const float mg = fmaxf(4e-6f * (1.0f + fabsf(theta)), 1e-10f / (dbeta * x));
        const float hi = theta + mg, lo = theta - mg;
        const float LIM = 1073741824.0f; // 2^30, beyond any |dE| <= 2 d N
        if (!(hi == hi) || !(lo == lo)) {
          slow = true;
        } else {
          Ar[half] = hi >= LIM ? (int)LIM : (hi <= -LIM ? -(int)LIM : (int)ceilf(hi));
          Rr[half] = lo <= -LIM ? -(int)LIM : (lo >= LIM ? (int)LIM : (int)floorf(lo));
        }
      }
      ur[half] = u;
    }
    slowm[half] = __ballot_sync(FULL, slow);
  }
  const int p0 = lane < T ? pm[lane] : 0, p1 = lane + 32 < T ? pm[lane + 32] : 0;
  const int e0 = lane < T ? el[p0] : 0, e1 = lane + 32 < T ? el[p1] : 0;
  int np0 = p0, np1 = p1;
  uint32_t acc0 = 0u, acc1 = 0u;
  unsigned int n_exact = 0u, n_near = 0u;
  int cur = __shfl_sync(FULL, p0, 0), ecur = __shfl_sync(FULL, e0, 0);
  for (int k = 0; k + 1 < T; ++k) {
    const int kn = k + 1;
    const bool lo_n = kn < 32, lo_k = k < 32; // warp-uniform
    const int b = __shfl_sync(FULL, lo_n ? p0 : p1, kn & 31);
    const int eb = __shfl_sync(FULL, lo_n ? e0 : e1, kn & 31);
    const int Ak = __shfl_sync(FULL, lo_k ? Ar[0] : Ar[1], k & 31);
    const int Rk = __shfl_sync(FULL, lo_k ? Rr[0] : Rr[1], k & 31);
    const bool slow = (((lo_k ? slowm[0] : slowm[1]) >> (k & 31)) & 1u) != 0u;
    const int dE = ecur - eb;
    bool accept;
    if (dE >= 0) {
      accept = true;
    } else if (!slow && dE >= Ak) {
      accept = true;
    } else if (!slow && dE <= Rk) {
      accept = false;
    } else {
      const uint32_t uk = __shfl_sync(FULL, lo_k ? ur[0] : ur[1], k & 31);
      const double dbeta = __dsub_rn(beta[k], beta[k + 1]);
      const double delta = __dmul_rn(dbeta, (double)dE);
      const double x = __dmul_rn((double)uk, 0x1p-32);
      const double e = exp(delta);
      if (fabs(__dsub_rn(x, e)) < 1e-12) ++n_near;
      ++n_exact;
      accept = x < e;
    }
    const int placed = accept ? b : cur; // the replica that ends the pass at slot k
    if (!accept) {
      cur = b;
      ecur = eb;
    }
    if (lane == (k & 31)) {
      if (lo_k) np0 = placed;
      else np1 = placed;
    }
    if (accept) {
      if (lo_k) acc0 |= 1u << k;
      else acc1 |= 1u << (k - 32);
    }
  }
  if (T >= 1 && lane == ((T - 1) & 31)) {
    if (T - 1 < 32) np0 = cur;
    else np1 = cur;
  }
  __syncwarp();
  if (lane < T) {
    pm[lane] = np0;
    sl[np0] = lane;
  }
  if (lane + 32 < T) {
    pm[lane + 32] = np1;
    sl[np1] = lane + 32;
  }
  if ((acc0 >> lane) & 1u) pacc[lane] += 1u;
  if ((acc1 >> lane) & 1u) pacc[lane + 32] += 1u;
  if (lane == 0) {
    *pnear += n_near;
    *pexact += n_exact;
  }
  __syncwarp();
}

// The resident kernel.  Each CTA is one item of one job: WPC consecutive 32-replica word
// lattices of one sample (sample s, words w0 .. w0+WPC-1), staged in shared memory for
// n_mcs MCS.  When the job's `fuse` flag is set the item holds whole chains (a chain is
// Wc <= WPC words) and their exchange passes run between the MCS.  The job comes from a
// table in parameter space, so one launch can sweep many jobs of one lattice shape.
// FULLW: every word of every job of the launch is full (each chain a multiple of 32
// replicas), so the partial-word decision code is left out of the instantiation.
// HOUD (single-job launches whose CTAs hold both one-word chains of a sample): 1, after
// the last sweep write the Houdayer move's q bitmaps and M of every pair; 2 (energy
// only, right after the move's cluster phase), first apply the move's cluster flips;
// 3 (one MCS of sweeps between two moves), first the previous move's flips, the energies
// after it and that MCS's exchange, then the sweeps, then the next move's q bitmaps.
// PAIR (sweeps with the exchange fused, two chains whose last word holds at most 16
// replicas): a CTA holds one whole sample, the chains' full words (WPC = 3: one each)
// and ONE paired word whose lanes 0..15 are chain 0's last word and lanes 16..31 chain
// 1's (WPC = 1: chains of up to 16 replicas).  The paired word draws the same Philox
// words and takes the same decisions as the two partial words, with the per-site work of
// one word instead of two; it is assembled from and split back into them in global
// memory, so the layout there does not change.
template <int D, int NT, int WPC, bool ENERGY_ONLY, int MAXJ, bool MEAS = false, bool FULLW = false, int HOUD = 0,
          bool PAIR = false>
__global__ void __launch_bounds__(NT, SGMC_MIN_THREADS / NT)
    k_resident_packed(const __grid_constant__ ResidentParams<MAXJ> rp) {
  extern __shared__ __align__(128) unsigned char smem[];
  int jsel = 0;
  if (MAXJ > 1) {
    for (int q = 1; q < rp.n_jobs; ++q)
      if ((int)blockIdx.x >= rp.jobs[q].first_item) jsel = q;
  }
  const JobDesc &JD = rp.jobs[jsel];
  const Job &jb = JD.jb;
  const Dev &dv = JD.dv;
  const bool fuse = JD.fuse != 0;
  const int n_mcs = rp.n_mcs, n_metro = JD.n_metro;
  const Geo g = jb.g;
  static_assert(!PAIR || ((WPC == 1 || WPC == 3) && !ENERGY_ONLY && !MEAS && HOUD == 0), "paired words");
  const PackedSmem L = packed_smem(g.N, g.NW, D, NT, WPC, PAIR ? 2 : WPC);
  uint32_t *sp = reinterpret_cast<uint32_t *>(smem + L.spin);
  uint8_t *jbyte = smem + L.jbyte;
  uint32_t *jpl = reinterpret_cast<uint32_t *>(smem + L.jpl);
  uint2 *pair_tab = reinterpret_cast<uint2 *>(smem + L.thr); // [WPC][16 pairs][16 codes]
  int32_t *epart = reinterpret_cast<int32_t *>(smem + L.epart);
  int32_t *ptw = reinterpret_cast<int32_t *>(smem + L.pt);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);
  // per chain slot ci: pm, sl, el, pacc [64 each], near and exact-path counts, round-trip
  // direction and start [64 each], trips and their total
  auto PM = [&](int ci) { return ptw + ci * PT_WORDS; };
  auto SL = [&](int ci) { return ptw + ci * PT_WORDS + 64; };
  auto EL = [&](int ci) { return ptw + ci * PT_WORDS + 128; };
  auto PACC = [&](int ci) { return reinterpret_cast<unsigned int *>(ptw + ci * PT_WORDS + 192); };
  auto NEAR = [&](int ci) { return reinterpret_cast<unsigned int *>(ptw + ci * PT_WORDS + 256); };
  auto EXACT = [&](int ci) { return reinterpret_cast<unsigned int *>(ptw + ci * PT_WORDS + 257); };
  auto TD = [&](int ci) { return ptw + ci * PT_WORDS + 258; };
  auto T0 = [&](int ci) { return reinterpret_cast<uint32_t *>(ptw + ci * PT_WORDS + 322); };
  auto TN = [&](int ci) { return reinterpret_cast<uint32_t *>(ptw + ci * PT_WORDS + 386); };
  auto TSUM = [&](int ci) { return reinterpret_cast<unsigned long long *>(ptw + ci * PT_WORDS + 388); };
  const bool track = dv.trip_dir != nullptr;
  // energies after a Houdayer move (pad0 = 1): the move conserves E_a + E_b of the pair at
  // each slot, so only chain 0's words are counted and chain 1's energies follow
  const bool conserve = ENERGY_ONLY && MAXJ == 1 && WPC == 2 && rp.pad0 == 1 && JD.fuse && jb.C == 2 && jb.Wc == 1;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const uint32_t t_metro0 = (uint32_t)dv.ctr[CTR_TMETRO], t_pt0 = (uint32_t)dv.ctr[CTR_TPT];
  const unsigned long long adv_metro = ENERGY_ONLY ? 0ull : (unsigned long long)n_mcs * n_metro;
  const unsigned long long adv_pt = fuse ? (unsigned long long)n_mcs : 0ull;
  const int groups = PAIR ? 1 : jb.W / WPC; // items per sample
  const int li = (int)blockIdx.x - JD.first_item;
  const int s = li / groups;
  const int w0 = PAIR ? 0 : (li - s * groups) * WPC;
  const uint32_t s_glob = (uint32_t)(jb.s_off + s);
  const int c0 = w0 / jb.Wc;                           // first chain of the item
  const int nch = PAIR ? 2 : (fuse ? WPC / jb.Wc : 0); // whole chains held (fused exchange)
  const int tpair = PAIR ? jb.T - 32 * (jb.Wc - 1) : 0; // replicas per chain in the paired word
  int ngroups[WPC];
  uint32_t vmask[WPC], c3base[WPC];
#pragma unroll
  for (int w = 0; w < WPC; ++w) {
    if (PAIR) {
      if (w < WPC - 1) { // chain w's full first word
        vmask[w] = FULL;
        ngroups[w] = 8;
        c3base[w] = ((uint32_t)w << 20) | TAG_METRO;
      } else { // the paired last words (chain 1's counter bit is added per group)
        const uint32_t m = (1u << tpair) - 1u;
        vmask[w] = m | (m << 16);
        ngroups[w] = (tpair + 3) >> 2;
        c3base[w] = ((uint32_t)((jb.Wc - 1) * 8) << 8) | TAG_METRO;
      }
      continue;
    }
    const int cwv = (w0 + w) / jb.Wc;
    const int wcv = (w0 + w) - cwv * jb.Wc;
    const int nv = min(32, jb.T - wcv * 32);
    vmask[w] = nv >= 32 ? FULL : ((1u << nv) - 1u);
    ngroups[w] = (nv + 3) >> 2;
    c3base[w] = ((uint32_t)cwv << 20) | ((uint32_t)(wcv * 8) << 8) | TAG_METRO;
  }
  uint32_t *gsp = dv.spins + ((size_t)s * jb.W + w0) * g.N; // WPC consecutive word lattices
  const uint32_t *gj = dv.jbits + (size_t)s * D * g.NW;

  // two transactions: the coupling planes (bar[0]) are expanded and the threshold tables
  // filled while the larger spin lattices (bar[1]) are still in flight
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t sbytes = 4u * (uint32_t)(g.N * WPC), jbytes = 4u * (uint32_t)(D * g.NW);
    mbar_expect_tx(bar, jbytes);
    bulk_g2s(jpl, gj, jbytes, bar);
    if (PAIR) {
      // the chains' full first words (word 0 of chain 0 and of chain 1); none when WPC = 1
      const uint32_t wbytes = 4u * (uint32_t)g.N;
      mbar_expect_tx(bar + 1, (uint32_t)(WPC - 1) * wbytes);
      if (WPC == 3) {
        bulk_g2s(sp, gsp, wbytes, bar + 1);
        bulk_g2s(sp + g.N, gsp + (size_t)jb.Wc * g.N, wbytes, bar + 1);
      }
    } else {
      mbar_expect_tx(bar + 1, sbytes);
      bulk_g2s(sp, gsp, sbytes, bar + 1);
    }
  }
  if (PAIR) {
    // the paired word from the two chains' last words (lanes 0..15 each)
    const uint32_t *l0 = gsp + (size_t)(jb.Wc - 1) * g.N, *l1 = gsp + (size_t)(2 * jb.Wc - 1) * g.N;
    uint32_t *pw = sp + (WPC - 1) * g.N;
    for (int p = tid; p < g.N; p += NT) pw[p] = (l0[p] & 0xFFFFu) | (l1[p] << 16);
  }
  // warp w < WPC owns local word w: its chain slot, replica offset and valid lanes
  const int my_c = (w0 + warp) / jb.Wc;
  const int my_wc = (w0 + warp) - my_c * jb.Wc;
  const int my_ci = my_c - c0;
  const int my_j0 = my_wc * 32;
  const int my_nvalid = min(32, jb.T - my_j0);
  const size_t my_cb = ((size_t)s * jb.C + my_c) * jb.T;
  if (warp < nch) {
    // warp ci loads chain ci's maps
    const size_t cb = ((size_t)s * jb.C + c0 + warp) * jb.T;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      PM(warp)[j] = j < jb.T ? dv.perm[cb + j] : 0;
      SL(warp)[j] = j < jb.T ? dv.slot[cb + j] : 0;
      PACC(warp)[j] = 0u;
      if (track) {
        TD(warp)[j] = j < jb.T ? dv.trip_dir[cb + j] : 0;
        T0(warp)[j] = j < jb.T ? dv.trip_t0[cb + j] : 0u;
      }
    }
    if (lane == 0) {
      *NEAR(warp) = 0u;
      *EXACT(warp) = 0u;
      *TN(warp) = 0u;
      *TSUM(warp) = 0ull;
    }
  }
  // the paired word's table: lane l < 16 holds chain 0's replica 32 (Wc - 1) + l, lane
  // 16 + l chain 1's, valid for l < tpair
  auto fill_paired = [&]() {
    const int hl = lane & 15, jr = 32 * (jb.Wc - 1) + hl;
    const bool ok = hl < tpair;
    fill_pair_table<D>(pair_tab + (WPC - 1) * 256, lane, ok ? SL(lane >> 4)[jr] : 0, ok, dv.thr);
  };
  __syncthreads(); // the chains' maps
  const bool okj = mbar_wait(bar, 0, MBAR_MAX_TRIES);
  if (!ENERGY_ONLY && HOUD != 3 && warp < WPC) { // (HOUD 3: after its exchange)
    if (PAIR) {
      if (warp < WPC - 1) fill_pair_table<D>(pair_tab + warp * 256, lane, SL(warp)[lane], true, dv.thr);
      else fill_paired();
    } else {
      const int kslot = lane < my_nvalid ? (fuse ? SL(my_ci)[my_j0 + lane] : dv.slot[my_cb + my_j0 + lane]) : 0;
      fill_pair_table<D>(pair_tab + warp * 256, lane, kslot, lane < my_nvalid, dv.thr);
    }
  }
  expand_couplings<D, NT>(g, jpl, jbyte); // (read but unused if the copy timed out)
  const bool oks = mbar_wait(bar + 1, 0, MBAR_MAX_TRIES);
  if (__syncthreads_or(!(okj && oks))) {
    if (tid == 0) {
      atomicOr(&dv.ctr[CTR_ERROR], ERR_TMA_TIMEOUT);
      // let copies still in flight land before exiting
      mbar_wait(bar, 0, MBAR_MAX_TRIES);
      mbar_wait(bar + 1, 0, MBAR_MAX_TRIES);
    }
    job_done_advance(dv.ctr, JD.n_items, adv_metro, adv_pt, HOUD >= 2 ? 1ull : 0ull);
    return;
  }
  // warp ci < nch: chain ci's exchange pass number t_pt0 + m (Eq. 5), then its round trips
  auto exchange_step = [&](int m) {
    exchange_chain_smem(jb.T, dv.beta, PM(warp), SL(warp), EL(warp), PACC(warp), NEAR(warp), EXACT(warp), s_glob,
                        (uint32_t)(c0 + warp), t_pt0 + (uint32_t)m, jb);
    if (track) {
      uint32_t n_add = 0u;
      unsigned long long sum_add = 0ull;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        if (j < jb.T) {
          int32_t dir = TD(warp)[j];
          uint32_t t0 = T0(warp)[j];
          trip_step(jb.T, SL(warp)[j], dir, t0, t_pt0 + (uint32_t)m + 1u, n_add, sum_add);
          TD(warp)[j] = dir;
          T0(warp)[j] = t0;
        }
      }
      n_add = __reduce_add_sync(FULL, n_add);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum_add += __shfl_xor_sync(FULL, sum_add, o);
      if (lane == 0) {
        *TN(warp) += n_add;
        *TSUM(warp) += sum_add;
      }
    }
  };
  if constexpr (HOUD == 2 || HOUD == 3) {
    // Houdayer move, phase 3 (Eq. 10): on pair a's cluster (chain-0 lane a with the
    // chain-1 lane b = perm1[slot0[a]] of the same slot) both replicas flip.  A warp
    // transposes the pairs' cluster bitmap words of a 32-site block (lane l: bit a = site l
    // in pair a's cluster); the chain-0 word takes the mask as is, the chain-1 word its
    // permutation a -> b.  Pairs without a q = -1 site (M = 0) have no bitmap.
    uint32_t *sigi = reinterpret_cast<uint32_t *>(pair_tab); // 1024 words: byte tables a -> b
    const int T = jb.T, NBW = rp.hm.NBW, RW = rp.hm.RW;
    for (int e = tid; e < 1024; e += NT) {
      const int j = e >> 8, v = e & 255;
      uint32_t o = 0u;
#pragma unroll
      for (int bb = 0; bb < 8; ++bb) {
        const int a = 8 * j + bb;
        if (((v >> bb) & 1) && a < T) o |= 1u << PM(1)[SL(0)[a]];
      }
      sigi[e] = o;
    }
    const uint32_t skip = __ballot_sync(FULL, lane >= T || rp.hm.Mg[(size_t)s * 32 + lane] == 0u);
    const bool mine = lane < T && !((skip >> lane) & 1u);
    const uint32_t *Cb = rp.hm.Cg + (size_t)s * T * NBW + (size_t)lane * NBW;
    __syncthreads();
    // a warp takes 4 consecutive blocks at a time: lane a loads them as one 16-byte word
    // of pair a's bitmap (bitmaps of a multiple of 4 words; one block at a time otherwise),
    // and issues the loads of BQ such groups before it uses any
    const int G = NBW % 4 == 0 ? 4 : 1;
    const BlockMap bm = block_map(g, RW);
    constexpr int BQ = 4;
    const int gstep = (NT / 32) * G;
    for (int base = warp * G; base < NBW; base += BQ * gstep) {
      uint4 cv[BQ];
#pragma unroll
      for (int j = 0; j < BQ; ++j) {
        const int b0 = base + j * gstep;
        cv[j] = make_uint4(0u, 0u, 0u, 0u);
        if (mine && b0 < NBW) {
          if (G == 4) cv[j] = *reinterpret_cast<const uint4 *>(Cb + b0);
          else cv[j].x = Cb[b0];
        }
      }
#pragma unroll
      for (int j = 0; j < BQ; ++j) {
        const int b0 = base + j * gstep;
        if (b0 >= NBW) break; // warp-uniform
        const uint32_t cw[4] = {cv[j].x, cv[j].y, cv[j].z, cv[j].w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (u < G && __any_sync(FULL, cw[u] != 0u)) {
            const uint32_t f = transpose32(cw[u], lane);
            bool valid;
            const int p = block_site(g, bm, b0 + u, lane, valid);
            if (valid && f) {
              sp[p] ^= f;
              sp[g.N + p] ^= permute_word(sigi, f);
            }
          }
        }
      }
    }
    __syncthreads();
  }
  if constexpr (HOUD == 3) {
    // the energies after the previous MCS's move (chain 0's counted, chain 1's from the
    // pair sums E_a + E_b that the move conserves; the global energies are still those
    // before it), then that MCS's exchange and the threshold tables of the new slots
    {
      uint32_t V[WPC][NB];
#pragma unroll
      for (int w = 0; w < WPC; ++w)
#pragma unroll
        for (int b = 0; b < NB; ++b) V[w][b] = 0u;
      const PhiloxSweep P0 = {}; // (counting only: no draws)
      half_sweep<D, NT, WPC, true, false, false>(g, 1, true, sp, jbyte, pair_tab, vmask, ngroups, c3base, P0, jb, V,
                                                 1);
      epart[tid] = warp_lane_sum(V[0]);
      __syncthreads();
      if (warp == 0) {
        int32_t U = 0;
        for (int wq = 0; wq < NT / 32; ++wq) U += epart[wq * 32 + lane];
        EL(0)[lane] = 2 * U - D * g.N;
      }
      __syncthreads();
      if (warp == 1 && lane < jb.T) {
        const size_t cb0 = (size_t)s * 2 * jb.T, cb1 = cb0 + jb.T;
        const int a = PM(0)[lane], b = PM(1)[lane];
        EL(1)[b] = dv.E[cb0 + a] + dv.E[cb1 + b] - EL(0)[a];
      }
      __syncthreads();
    }
    if (warp < 2) {
      exchange_step(0);
      fill_pair_table<D>(pair_tab + warp * 256, lane, lane < jb.T ? SL(warp)[lane] : 0, lane < jb.T, dv.thr);
    }
  }
  // the sweeps start after a full barrier (which also keeps the prologue's values out of
  // the sweep loop's register allocation)
  __syncthreads();

  const bool warp_owned = !ENERGY_ONLY && !PAIR && (nch == 0 || (jb.Wc == 1 && nch == WPC));
  const int n_outer = ENERGY_ONLY ? 1 : n_mcs;
  const int n_inner = ENERGY_ONLY ? 1 : n_metro;
  for (int m = 0; m < n_outer; ++m) {
    for (int swp = 0; swp < n_inner; ++swp) {
      const uint32_t t = t_metro0 + (uint32_t)(m * n_metro + swp);
      const PhiloxSweep P = philox_sweep(s_glob, t, jb);
      uint32_t V[WPC][NB];
#pragma unroll
      for (int w = 0; w < WPC; ++w)
#pragma unroll
        for (int b = 0; b < NB; ++b) V[w][b] = 0u;
      if (!ENERGY_ONLY) {
        // colour 0, a barrier, colour 1 with the energy counts: one loop body, one copy of
        // the half-sweep's code
#pragma unroll 1
        for (int col = 0; col < 2; ++col) {
          half_sweep<D, NT, WPC, false, FULLW, PAIR>(g, col, col == 1, sp, jbyte, pair_tab, vmask, ngroups, c3base, P, jb,
                                                     V);
          if (col == 0) __syncthreads();
        }
      } else {
        half_sweep<D, NT, WPC, true, false, false>(g, 1, true, sp, jbyte, pair_tab, vmask, ngroups, c3base, P, jb, V,
                                                   conserve ? 1 : WPC);
      }
#pragma unroll
      for (int w = 0; w < WPC; ++w) epart[w * NT + tid] = warp_lane_sum(V[w]);
      __syncthreads();
      if (warp < WPC) {
        int32_t U = 0;
        for (int wq = 0; wq < NT / 32; ++wq) U += epart[warp * NT + wq * 32 + lane];
        // held chains (T <= 64) keep their energies for the exchange; otherwise the
        // energies go straight to global memory (the per-chain slots hold 64 replicas)
        if (PAIR) {
          if (warp < WPC - 1) EL(warp)[lane] = 2 * U - D * g.N;
          else if ((lane & 15) < tpair) EL(lane >> 4)[32 * (jb.Wc - 1) + (lane & 15)] = 2 * U - D * g.N;
        } else if (nch > 0) {
          EL(my_ci)[my_j0 + lane] = 2 * U - D * g.N;
        } else if (lane < my_nvalid) {
          dv.E[my_cb + my_j0 + lane] = 2 * U - D * g.N;
        }
      }
      // when each word is a whole chain, the warp that sums a word's energies is the one
      // that exchanges its chain, so only its own lanes need to see them; otherwise (a
      // chain of two words, or the energies after a cluster move) the whole CTA waits
      if (warp_owned) __syncwarp();
      else __syncthreads();
      if (conserve) {
        // slot k pairs chain-0 replica a = perm0[k] with chain-1 replica b = perm1[k]; the
        // global energies are still those before the move
        if (warp == 1 && lane < jb.T) {
          const size_t cb0 = (size_t)s * 2 * jb.T, cb1 = cb0 + jb.T;
          const int a = PM(0)[lane], b = PM(1)[lane];
          EL(1)[b] = dv.E[cb0 + a] + dv.E[cb1 + b] - EL(0)[a];
        }
        __syncthreads();
      }
    }
    if (nch > 0 && HOUD != 3) { // (HOUD 3: the exchange came before the sweeps)
      // warp ci exchanges chain ci, then refreshes the tables of the chain's words
      if (warp < nch) {
        exchange_step(m);
        // the tables follow the new slots, unless this was the launch's last MCS
        if (PAIR) {
          if (WPC == 3 && m + 1 < n_outer) fill_pair_table<D>(pair_tab + warp * 256, lane, SL(warp)[lane], true, dv.thr);
        } else if (!ENERGY_ONLY && m + 1 < n_outer) {
          for (int wc = 0; wc < jb.Wc; ++wc) {
            const int nv = min(32, jb.T - wc * 32);
            fill_pair_table<D>(pair_tab + (warp * jb.Wc + wc) * 256, lane,
                               lane < nv ? SL(warp)[wc * 32 + lane] : 0, lane < nv, dv.thr);
          }
        }
      }
      __syncthreads();
      if (PAIR && m + 1 < n_outer) { // the paired word's table needs both chains' new slots
        if (warp == WPC - 1) fill_paired();
        __syncthreads();
      }
    }
  }

  if constexpr (MEAS) {
    // fused measurement (the launcher checked: two one-word chains held, exchange fused):
    // E by slot from the held energies and maps, and N q of the 32 pairs from one xor
    // per site of chain 0's word with chain 1's word moved into chain-0 lane order (lane
    // b -> perm0[slot1[b]]) by byte tables, which take the no longer needed pair tables
    const int T = jb.T;
    for (int e = tid; e < 2 * T; e += NT) {
      const int ci = e >= T ? 1 : 0, k = e - ci * T;
      rp.mE[((size_t)s * 2 + ci) * T + k] = EL(ci)[PM(ci)[k]];
    }
    if (rp.mQ != nullptr) {
      uint32_t *sig = reinterpret_cast<uint32_t *>(pair_tab); // 1024 words = the 2 x 256 uint2 tables
      uint32_t *tot = reinterpret_cast<uint32_t *>(epart);    // [32] disagreeing sites per pair
      uint32_t *nib = tot + 32;                                // [8][16] the permutation by nibbles
      for (int e = tid; e < 128; e += NT) {
        const int j = e >> 4, v = e & 15;
        uint32_t o = 0u;
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) {
          const int b = 4 * j + bb;
          if (((v >> bb) & 1) && b < T) o |= 1u << PM(0)[SL(1)[b]];
        }
        nib[e] = o;
      }
      if (tid < 32) tot[tid] = 0u;
      __syncthreads();
      for (int e = tid; e < 1024; e += NT) {
        const int j = e >> 8, v = e & 255;
        sig[e] = nib[(2 * j) * 16 + (v & 15)] | nib[(2 * j + 1) * 16 + (v >> 4)];
      }
      __syncthreads();
      uint32_t Vq[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) Vq[b] = 0u;
      const int n4 = g.N >> 2; // every extent is even: N is a multiple of 4
      const int iters = (n4 + NT - 1) / NT;
      for (int it = 0; it < iters; ++it) {
        const int i = it * NT + tid;
        if (i < n4) {
          const uint4 a4 = reinterpret_cast<const uint4 *>(sp)[i];
          const uint4 b4 = reinterpret_cast<const uint4 *>(sp + g.N)[i];
          const uint32_t q0 = a4.x ^ permute_word(sig, b4.x), q1 = a4.y ^ permute_word(sig, b4.y);
          const uint32_t q2 = a4.z ^ permute_word(sig, b4.z), q3 = a4.w ^ permute_word(sig, b4.w);
          uint32_t s1, cy1;
          fadd(q0, q1, q2, s1, cy1);
          const uint32_t cc = s1 & q3;
          vcount_add(Vq, s1 ^ q3, cy1 ^ cc, cy1 & cc);
        }
        if ((it + 1) % 63 == 0 || it + 1 == iters) { // before 8 planes can overflow; warp-uniform
          const int32_t v = warp_lane_sum(Vq);
          if (v) atomicAdd(&tot[lane], (uint32_t)v);
#pragma unroll
          for (int b = 0; b < NB; ++b) Vq[b] = 0u;
        }
      }
      __syncthreads();
      if (tid < T) rp.mQ[(size_t)s * T + SL(0)[tid]] = g.N - 2 * (int32_t)tot[tid];
    }
  }
  if constexpr (HOUD == 1 || HOUD == 3) {
    // Houdayer move, phase 1 (Eq. 10) on the final configurations: per site the chain-1
    // word is permuted lane b -> lane a = perm0[slot1[b]] (byte tables), so that bit a of
    // w0 ^ sigma(w1) is q = -1 of pair a; a warp transposes 32 sites x 32 pairs, giving
    // each pair's bitmap word of the block, and M counts the q = -1 sites of each pair.
    // Only pairs at a slot below hK take part (the others get an empty bitmap).  The maps
    // are the global ones (HOUD 1, no exchange in the launch) or the held ones (HOUD 3,
    // after its exchange).
    __syncthreads(); // every warp is past its last half-sweep: the pair tables are free
    const int32_t *perm0, *slot0, *slot1;
    uint32_t *Mc;
    const int T = jb.T, NBW = rp.hm.NBW, RW = rp.hm.RW;
    if (HOUD == 1) {
      int32_t *maps = ptw; // perm0, perm1, slot0, slot1 [32 each], then M [32]
      if (warp < 2) {
        const size_t cb = ((size_t)s * 2 + warp) * T;
        maps[warp * 32 + lane] = lane < T ? dv.perm[cb + lane] : 0;
        maps[64 + warp * 32 + lane] = lane < T ? dv.slot[cb + lane] : 0;
      }
      perm0 = maps;
      slot0 = maps + 64;
      slot1 = maps + 96;
      Mc = reinterpret_cast<uint32_t *>(ptw + 128);
    } else {
      perm0 = PM(0);
      slot0 = SL(0);
      slot1 = SL(1);
      Mc = reinterpret_cast<uint32_t *>(epart);
    }
    if (tid < 32) Mc[tid] = 0u;
    __syncthreads();
    uint32_t *sig = reinterpret_cast<uint32_t *>(pair_tab); // 1024 words
    for (int e = tid; e < 1024; e += NT) {
      const int j = e >> 8, v = e & 255;
      uint32_t o = 0u;
#pragma unroll
      for (int bb = 0; bb < 8; ++bb) {
        const int b = 8 * j + bb;
        if (((v >> bb) & 1) && b < T) o |= 1u << perm0[slot1[b]];
      }
      sig[e] = o;
    }
    const uint32_t tmask = houd_pair_mask(jb, slot0);
    uint32_t *Qb = rp.hm.Qg + (size_t)s * T * NBW + (size_t)lane * NBW;
    uint32_t mpart = 0u;
    __syncthreads();
    // a warp takes 4 consecutive blocks at a time: lane a stores them as one 16-byte word
    // of pair a's bitmap (bitmaps of a multiple of 4 words; one block at a time otherwise)
    const int G = NBW % 4 == 0 ? 4 : 1;
    const BlockMap bm = block_map(g, RW);
    for (int b0 = warp * G; b0 < NBW; b0 += (NT / 32) * G) {
      uint32_t col[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        col[u] = 0u;
        if (u < G) {
          bool valid;
          const int p = block_site(g, bm, b0 + u, lane, valid);
          const uint32_t qa = valid ? (sp[p] ^ permute_word(sig, sp[g.N + p])) & tmask : 0u;
          col[u] = transpose32(qa, lane); // lane a: bit l = q of pair a at site l
        }
      }
      if (lane < T) {
        if (G == 4) *reinterpret_cast<uint4 *>(Qb + b0) = make_uint4(col[0], col[1], col[2], col[3]);
        else Qb[b0] = col[0];
        mpart += __popc(col[0]) + __popc(col[1]) + __popc(col[2]) + __popc(col[3]);
      }
    }
    if (lane < T && mpart) atomicAdd(&Mc[lane], mpart);
    __syncthreads();
    if (tid < 32) rp.hm.Mg[(size_t)s * 32 + tid] = Mc[tid]; // the CTA holds the whole sample
  }
  if (PAIR) {
    if (warp < 2) {
      const size_t cb = ((size_t)s * 2 + warp) * jb.T;
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (lane + 32 * h < jb.T) dv.E[cb + lane + 32 * h] = EL(warp)[lane + 32 * h];
    }
  } else if (nch > 0 && warp < WPC && lane < my_nvalid) {
    dv.E[my_cb + my_j0 + lane] = EL(my_ci)[my_j0 + lane];
  }
  if (warp < nch) {
    const size_t cb = ((size_t)s * jb.C + c0 + warp) * jb.T;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      if (j < jb.T) {
        dv.perm[cb + j] = PM(warp)[j];
        dv.slot[cb + j] = SL(warp)[j];
      }
      if (j + 1 < jb.T && PACC(warp)[j]) atomicAdd(&dv.ctr[CTR_PT + j], (unsigned long long)PACC(warp)[j]);
      if (track && j < jb.T) {
        dv.trip_dir[cb + j] = TD(warp)[j];
        dv.trip_t0[cb + j] = T0(warp)[j];
      }
    }
    if (lane == 0 && *NEAR(warp)) atomicAdd(&dv.ctr[CTR_NEAR], (unsigned long long)*NEAR(warp));
    if (lane == 0 && *EXACT(warp)) atomicAdd(&dv.ctr[CTR_XEXACT], (unsigned long long)*EXACT(warp));
    if (track && lane == 0) {
      const size_t chain = (size_t)s * jb.C + c0 + warp;
      dv.trip_n[chain] += *TN(warp);
      dv.trip_sum[chain] += *TSUM(warp);
    }
  }
  if (PAIR) {
    fence_proxy_async(); // this thread's shared-memory writes -> visible to the TMA store
    __syncthreads();
    // the full first words back by TMA, the paired word split into the two last words
    if (tid == 0 && WPC == 3) {
      bulk_s2g_and_release(gsp, sp, 4u * (uint32_t)g.N);
      bulk_s2g_and_release(gsp + (size_t)jb.Wc * g.N, sp + g.N, 4u * (uint32_t)g.N);
    }
    uint32_t *l0 = gsp + (size_t)(jb.Wc - 1) * g.N, *l1 = gsp + (size_t)(2 * jb.Wc - 1) * g.N;
    const uint32_t *pw = sp + (WPC - 1) * g.N;
    for (int p = tid; p < g.N; p += NT) {
      const uint32_t v = pw[p];
      l0[p] = v & 0xFFFFu;
      l1[p] = v >> 16;
    }
  } else if (!ENERGY_ONLY || HOUD == 2) {
    fence_proxy_async(); // this thread's shared-memory writes -> visible to the TMA store
    __syncthreads();
    if (tid == 0) bulk_s2g_and_release(gsp, sp, 4u * (uint32_t)(g.N * WPC));
  }
  job_done_advance(dv.ctr, JD.n_items, adv_metro, adv_pt, HOUD >= 2 ? 1ull : 0ull);
}

} // namespace sgmc
