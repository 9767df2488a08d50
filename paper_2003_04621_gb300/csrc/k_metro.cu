// k_metro.cu -- resident Metropolis kernels (Sec. 2.2 / 2.4 step 1) with the energy
// (Eq. 1) and, when a chain fits in one CTA, the replica exchange (Eq. 5) fused in.
//
// Packed kernel: one CTA owns one 32-replica word lattice (sample s, word w) for the
// whole launch.  TMA bulk-copies the N words and the sample's coupling bit planes into
// shared memory, runs n_mcs x n_metro checkerboard sweeps there (colour 0 then colour 1,
// each site updating its 32 replicas at once), keeps the energies exact, optionally
// performs the chain's exchange pass between MCS, and bulk-copies the lattice back.
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
#include "sgmc_houd.cuh"
#include "sgmc_internal.cuh"
#include "sgmc_sweep.cuh"
#include "sgmc_tma.cuh"

#include <vector>

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
template <int D, int NT, int WPC, bool NOFLIP, bool FULLW>
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
        F = decide_site<D, FULLW>(cnt, P, Q, c3base[w], ngroups[w], pair_tab + w * 256, jb) & vmask[w];
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
// only, right after the move's cluster phase), first apply the move's cluster flips.
template <int D, int NT, int WPC, bool ENERGY_ONLY, int MAXJ, bool MEAS = false, bool FULLW = false, int HOUD = 0>
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
  const PackedSmem L = packed_smem(g.N, g.NW, D, NT, WPC);
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
  const int groups = jb.W / WPC;
  const int li = (int)blockIdx.x - JD.first_item;
  const int s = li / groups;
  const int w0 = (li - s * groups) * WPC;
  const uint32_t s_glob = (uint32_t)(jb.s_off + s);
  const int c0 = w0 / jb.Wc;              // first chain of the item
  const int nch = fuse ? WPC / jb.Wc : 0; // whole chains held (fused exchange)
  int ngroups[WPC];
  uint32_t vmask[WPC], c3base[WPC];
#pragma unroll
  for (int w = 0; w < WPC; ++w) {
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
    mbar_expect_tx(bar + 1, sbytes);
    bulk_g2s(sp, gsp, sbytes, bar + 1);
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
  __syncthreads(); // the chains' maps
  const bool okj = mbar_wait(bar, 0, MBAR_MAX_TRIES);
  if (!ENERGY_ONLY && warp < WPC) {
    const int kslot = lane < my_nvalid ? (fuse ? SL(my_ci)[my_j0 + lane] : dv.slot[my_cb + my_j0 + lane]) : 0;
    fill_pair_table<D>(pair_tab + warp * 256, lane, kslot, my_nvalid, dv.thr);
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
    job_done_advance(dv.ctr, JD.n_items, adv_metro, adv_pt, HOUD == 2 ? 1ull : 0ull);
    return;
  }
  if constexpr (HOUD == 2) {
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
    // of pair a's bitmap (bitmaps of a multiple of 4 words; one block at a time otherwise)
    const int G = NBW % 4 == 0 ? 4 : 1;
    for (int b0 = warp * G; b0 < NBW; b0 += (NT / 32) * G) {
      uint32_t cw[4] = {0u, 0u, 0u, 0u};
      if (mine) {
        if (G == 4) {
          const uint4 v = *reinterpret_cast<const uint4 *>(Cb + b0);
          cw[0] = v.x, cw[1] = v.y, cw[2] = v.z, cw[3] = v.w;
        } else {
          cw[0] = Cb[b0];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (u < G && __any_sync(FULL, cw[u] != 0u)) {
          const uint32_t f = transpose32(cw[u], lane);
          bool valid;
          const int p = block_site(g, RW, b0 + u, lane, valid);
          if (valid && f) {
            sp[p] ^= f;
            sp[g.N + p] ^= permute_word(sigi, f);
          }
        }
      }
    }
    __syncthreads();
  }
  // the sweeps start after a full barrier (which also keeps the prologue's values out of
  // the sweep loop's register allocation)
  __syncthreads();

  const bool warp_owned = !ENERGY_ONLY && (nch == 0 || (jb.Wc == 1 && nch == WPC));
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
          half_sweep<D, NT, WPC, false, FULLW>(g, col, col == 1, sp, jbyte, pair_tab, vmask, ngroups, c3base, P, jb, V);
          if (col == 0) __syncthreads();
        }
      } else {
        half_sweep<D, NT, WPC, true, false>(g, 1, true, sp, jbyte, pair_tab, vmask, ngroups, c3base, P, jb, V,
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
        if (nch > 0) EL(my_ci)[my_j0 + lane] = 2 * U - D * g.N;
        else if (lane < my_nvalid) dv.E[my_cb + my_j0 + lane] = 2 * U - D * g.N;
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
    if (nch > 0) {
      // warp ci exchanges chain ci, then refreshes the tables of the chain's words
      if (warp < nch) {
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
        if (!ENERGY_ONLY) {
          for (int wc = 0; wc < jb.Wc; ++wc) {
            const int nv = min(32, jb.T - wc * 32);
            fill_pair_table<D>(pair_tab + (warp * jb.Wc + wc) * 256, lane,
                               lane < nv ? SL(warp)[wc * 32 + lane] : 0, nv, dv.thr);
          }
        }
      }
      __syncthreads();
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
  if constexpr (HOUD == 1) {
    // Houdayer move, phase 1 (Eq. 10) on the final configurations: per site the chain-1
    // word is permuted lane b -> lane a = perm0[slot1[b]] (byte tables), so that bit a of
    // w0 ^ sigma(w1) is q = -1 of pair a; a warp transposes 32 sites x 32 pairs, giving
    // each pair's bitmap word of the block, and M counts the q = -1 sites of each pair.
    // Only pairs at a slot below hK take part (the others get an empty bitmap).
    __syncthreads(); // every warp is past its last half-sweep: the pair tables are free
    int32_t *maps = ptw; // perm0, perm1, slot0, slot1 [32 each], then M [32]
    uint32_t *Mc = reinterpret_cast<uint32_t *>(ptw + 128);
    const int T = jb.T, NBW = rp.hm.NBW, RW = rp.hm.RW;
    if (warp < 2) {
      const size_t cb = ((size_t)s * 2 + warp) * T;
      maps[warp * 32 + lane] = lane < T ? dv.perm[cb + lane] : 0;
      maps[64 + warp * 32 + lane] = lane < T ? dv.slot[cb + lane] : 0;
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
        if (((v >> bb) & 1) && b < T) o |= 1u << maps[maps[96 + b]];
      }
      sig[e] = o;
    }
    const uint32_t tmask = houd_pair_mask(jb, maps + 64);
    uint32_t *Qb = rp.hm.Qg + (size_t)s * T * NBW + (size_t)lane * NBW;
    uint32_t mpart = 0u;
    __syncthreads();
    // a warp takes 4 consecutive blocks at a time: lane a stores them as one 16-byte word
    // of pair a's bitmap (bitmaps of a multiple of 4 words; one block at a time otherwise)
    const int G = NBW % 4 == 0 ? 4 : 1;
    for (int b0 = warp * G; b0 < NBW; b0 += (NT / 32) * G) {
      uint32_t col[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        col[u] = 0u;
        if (u < G) {
          bool valid;
          const int p = block_site(g, RW, b0 + u, lane, valid);
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
  if (nch > 0 && warp < WPC && lane < my_nvalid) dv.E[my_cb + my_j0 + lane] = EL(my_ci)[my_j0 + lane];
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
  if (!ENERGY_ONLY || HOUD == 2) {
    fence_proxy_async(); // this thread's shared-memory writes -> visible to the TMA store
    __syncthreads();
    if (tid == 0) bulk_s2g_and_release(gsp, sp, 4u * (uint32_t)(g.N * WPC));
  }
  job_done_advance(dv.ctr, JD.n_items, adv_metro, adv_pt, HOUD == 2 ? 1ull : 0ull);
}

// A colour-`col` site of the int8 kernel, from its offset q in the colour's half: its
// canonical index i and the colour-split indices of its 2d neighbours (+e_mu, -e_mu).
template <int D>
struct Int8SiteT {
  uint32_t i;
  int pn[2 * D];
};
template <int D>
__device__ __forceinline__ Int8SiteT<D> int8_site(const Geo &g, int col, int q) {
  Int8SiteT<D> r;
  SiteGeo sg;
  sg.c = col;
  sg.row = q / g.H;
  sg.k = q - sg.row * g.H;
  sg.y = D == 3 ? sg.row % g.L1 : sg.row;
  sg.z = D == 3 ? sg.row / g.L1 : 0;
  sg.xodd = col ^ ((sg.y + sg.z) & 1);
  r.i = (uint32_t)(g.L0 * sg.row + 2 * sg.k + sg.xodd);
#pragma unroll
  for (int mu = 0; mu < D; ++mu) {
    r.pn[2 * mu] = nbr_cs(g, sg, mu, 1);
    r.pn[2 * mu + 1] = nbr_cs(g, sg, mu, -1);
  }
  return r;
}

// ---------------------------------------------------------------------------------
// int8 resident kernel: one CTA owns one chain (sample s, chain c) with all its replicas,
// spins as int8 +-1 (the paper's layout, replicas of a site adjacent, Sec. 3).  A thread
// item is (site of the colour, group of four replicas) -- one Philox call.
// ---------------------------------------------------------------------------------
template <int D, int NT, bool FUSE_PT, bool ENERGY_ONLY>
__global__ void __launch_bounds__(NT) k_resident_int8(Job jb, Dev dv, int n_mcs, int n_metro) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Geo g = jb.g;
  const int T = jb.T, Tp = jb.Tp, G = Tp / 4;
  const Int8Smem L = int8_smem(g.N, g.NW, D, T, Tp);
  int8_t *sp8 = reinterpret_cast<int8_t *>(smem + L.spin);
  uint8_t *jbyte = smem + L.jbyte;
  uint32_t *jpl = reinterpret_cast<uint32_t *>(smem + L.jpl);
  uint32_t *thr = reinterpret_cast<uint32_t *>(smem + L.thr); // [Tp][4], entry m = 1..d, by replica
  uint32_t *thk = reinterpret_cast<uint32_t *>(smem + L.thk); // [T][4], by temperature slot
  int32_t *eacc = reinterpret_cast<int32_t *>(smem + L.eacc);
  int32_t *pm = reinterpret_cast<int32_t *>(smem + L.pm);
  int32_t *sl = reinterpret_cast<int32_t *>(smem + L.sl);
  unsigned int *pacc = reinterpret_cast<unsigned int *>(smem + L.pacc);
  unsigned int *pnear = reinterpret_cast<unsigned int *>(smem + L.near);
  int32_t *xch = reinterpret_cast<int32_t *>(smem + L.xch); // T <= 64: the warp exchange's exact-path count
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);

  const int tid = threadIdx.x;
  const uint32_t t_metro0 = (uint32_t)dv.ctr[CTR_TMETRO], t_pt0 = (uint32_t)dv.ctr[CTR_TPT];
  const unsigned long long adv_metro = ENERGY_ONLY ? 0ull : (unsigned long long)n_mcs * n_metro;
  const unsigned long long adv_pt = FUSE_PT ? (unsigned long long)n_mcs : 0ull;
  const int s = blockIdx.x / jb.C;
  const int c = blockIdx.x - s * jb.C;
  const uint32_t s_glob = (uint32_t)(jb.s_off + s);
  int8_t *gsp = reinterpret_cast<int8_t *>(dv.spins) + ((size_t)s * jb.C + c) * g.N * Tp;
  const uint32_t *gj = dv.jbits + (size_t)s * D * g.NW;
  const size_t chain_base = ((size_t)s * jb.C + c) * T;

  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  if (tid == 0) {
    const uint32_t sbytes = (uint32_t)(g.N * Tp), jbytes = 4u * (uint32_t)(D * g.NW);
    mbar_expect_tx(bar, sbytes + jbytes);
    bulk_g2s(sp8, gsp, sbytes, bar);
    bulk_g2s(jpl, gj, jbytes, bar);
  }
  for (int j = tid; j < T; j += NT) {
    pm[j] = dv.perm[chain_base + j];
    sl[j] = dv.slot[chain_base + j];
    pacc[j] = 0u;
  }
  if (tid == 0) {
    *pnear = 0u;
    if (T <= 64) xch[0] = 0;
  }
  __syncthreads();
  if (!ENERGY_ONLY) {
    if (T <= INT8_THK_MAX)
      for (int e = tid; e < 4 * T; e += NT) thk[e] = dv.thr[e];
    for (int j = tid; j < Tp; j += NT)
#pragma unroll
      for (int m = 0; m < 4; ++m) thr[j * 4 + m] = (j < T && m >= 1 && m <= D) ? dv.thr[sl[j] * 4 + m] : 0u;
  }
  const bool ok = mbar_wait(bar, 0, MBAR_MAX_TRIES);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      atomicOr(&dv.ctr[CTR_ERROR], ERR_TMA_TIMEOUT);
      mbar_wait(bar, 0, MBAR_MAX_TRIES);
    }
    grid_done_advance(dv.ctr, adv_metro, adv_pt, 0ull);
    return;
  }
  expand_couplings<D, NT>(g, jpl, jbyte);
  __syncthreads();

  const int Nh = g.Nh;
  const int n_chunks = G * ((Nh + 31) / 32); // (replica group, 32 sites) items per half-sweep
  // when every warp holds at most one item per colour (small chains), the items' site
  // geometry is computed once for the whole launch
  const bool one_item = n_chunks <= NT / 32;
  Int8SiteT<D> cache0 = {}, cache1 = {};
  if (one_item && (tid >> 5) < n_chunks) {
    const int q = ((tid >> 5) / G) * 32 + (tid & 31);
    if (q < Nh) {
      cache0 = int8_site<D>(g, 0, q);
      cache1 = int8_site<D>(g, 1, q);
    }
  }
  const int n_outer = ENERGY_ONLY ? 1 : n_mcs;
  const int n_inner = ENERGY_ONLY ? 1 : n_metro;
  for (int m = 0; m < n_outer; ++m) {
    for (int swp = 0; swp < n_inner; ++swp) {
      const uint32_t t = t_metro0 + (uint32_t)(m * n_metro + swp);
      const PhiloxSweep P = philox_sweep(s_glob, t, jb);
      for (int col = ENERGY_ONLY ? 1 : 0; col < 2; ++col) {
        if (col == 1) {
          for (int j = tid; j < Tp; j += NT) eacc[j] = 0;
          __syncthreads();
        }
        // a warp takes 32 consecutive sites of one replica group at a time, so that its
        // lanes' energy terms can be summed over the warp before one shared add each
        for (int ch = tid >> 5; ch < n_chunks; ch += NT / 32) {
          const int gi = ch % G;
          const int q = (ch / G) * 32 + (tid & 31);
          const bool valid = q < Nh;
          int sv[4] = {0, 0, 0, 0}, h[4] = {0, 0, 0, 0};
          if (valid) {
            const Int8SiteT<D> sn = one_item ? (col ? cache1 : cache0) : int8_site<D>(g, col, q);
            const int p = col * Nh + q;
            const uint32_t jbb = jbyte[p];
            char4 s4 = *reinterpret_cast<const char4 *>(sp8 + (size_t)p * Tp + 4 * gi);
#pragma unroll
            for (int mu = 0; mu < D; ++mu) {
#pragma unroll
              for (int dir = 0; dir < 2; ++dir) {
                const int pn = sn.pn[2 * mu + dir];
                const char4 n4 = *reinterpret_cast<const char4 *>(sp8 + (size_t)pn * Tp + 4 * gi);
                const int Jv = ((jbb >> (2 * mu + dir)) & 1u) ? -1 : 1;
                h[0] += Jv * n4.x;
                h[1] += Jv * n4.y;
                h[2] += Jv * n4.z;
                h[3] += Jv * n4.w;
              }
            }
            sv[0] = s4.x;
            sv[1] = s4.y;
            sv[2] = s4.z;
            sv[3] = s4.w;
            if (!ENERGY_ONLY) {
              int dE[4];
              bool need = false;
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                dE[r] = 2 * sv[r] * h[r];
                need |= (4 * gi + r < T) && dE[r] > 0;
              }
              uint4 rnd = make_uint4(0, 0, 0, 0);
              if (need) {
                // counter (i, t, s, c << 20 | gi << 8 | METRO), the rounds shared by the sweep
                // and by the site hoisted as in the packed kernel
                const PhiloxSite Q = philox_site(P, sn.i, jb);
                rnd = philox_finish(P, Q, ((uint32_t)c << 20) | ((uint32_t)gi << 8) | TAG_METRO, jb);
              }
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                const int j = 4 * gi + r;
                if (j < T) {
                  const bool acc = dE[r] <= 0 || word_of(rnd, r) < thr[j * 4 + (dE[r] >> 2)];
                  if (acc) sv[r] = -sv[r];
                }
              }
              s4 = make_char4((signed char)sv[0], (signed char)sv[1], (signed char)sv[2], (signed char)sv[3]);
              *reinterpret_cast<char4 *>(sp8 + (size_t)p * Tp + 4 * gi) = s4;
            }
          }
          if (col == 1) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const int e = __reduce_add_sync(FULL, -sv[r] * h[r]);
              if ((tid & 31) == 0 && 4 * gi + r < T && e) atomicAdd(&eacc[4 * gi + r], e);
            }
          }
        }
        __syncthreads();
      }
    }
    if (FUSE_PT) {
      if (T <= 64) { // one warp: integer bounds first, the exact fp64 test only near them
        if (tid < 32) {
          exchange_chain_smem(T, dv.beta, pm, sl, eacc, pacc, pnear, reinterpret_cast<unsigned int *>(xch), s_glob,
                              (uint32_t)c, t_pt0 + (uint32_t)m, jb);
          if (tid == 0) trip_chain(dv, (size_t)s * jb.C + c, T, sl, t_pt0 + (uint32_t)m + 1u);
        }
      } else if (tid == 0) {
        exchange_chain(T, dv.beta, pm, sl, eacc, s_glob, (uint32_t)c, t_pt0 + (uint32_t)m, jb.sk0, jb.sk1,
                       [&](int k) { pacc[k] += 1u; }, [&]() { *pnear += 1u; });
        trip_chain(dv, (size_t)s * jb.C + c, T, sl, t_pt0 + (uint32_t)m + 1u);
      }
      __syncthreads();
      if (!ENERGY_ONLY)
        for (int j = tid; j < T; j += NT)
#pragma unroll
          for (int mm = 1; mm <= D; ++mm)
            thr[j * 4 + mm] = T <= INT8_THK_MAX ? thk[sl[j] * 4 + mm] : dv.thr[sl[j] * 4 + mm];
      __syncthreads();
    }
  }

  for (int j = tid; j < T; j += NT) {
    dv.E[chain_base + j] = eacc[j];
    if (FUSE_PT) {
      dv.perm[chain_base + j] = pm[j];
      dv.slot[chain_base + j] = sl[j];
      if (j + 1 < T && pacc[j]) atomicAdd(&dv.ctr[CTR_PT + j], (unsigned long long)pacc[j]);
    }
  }
  if (FUSE_PT && tid == 0 && *pnear) atomicAdd(&dv.ctr[CTR_NEAR], (unsigned long long)*pnear);
  if (FUSE_PT && T <= 64 && tid == 0 && xch[0]) atomicAdd(&dv.ctr[CTR_XEXACT], (unsigned long long)xch[0]);
  if (!ENERGY_ONLY) {
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) bulk_s2g_and_release(gsp, sp8, (uint32_t)(g.N * Tp));
  }
  grid_done_advance(dv.ctr, adv_metro, adv_pt, 0ull);
}

// Standalone exchange pass: one thread per (sample, chain), state in global memory.
__global__ void k_exchange(Job jb, Dev dv) {
  const int chain = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t t_pt = (uint32_t)dv.ctr[CTR_TPT];
  if (chain < jb.S * jb.C) {
    const int s = chain / jb.C;
    const int c = chain - s * jb.C;
    const size_t base = (size_t)chain * jb.T;
    unsigned long long *ctr = dv.ctr;
    exchange_chain(jb.T, dv.beta, dv.perm + base, dv.slot + base, dv.E + base, (uint32_t)(jb.s_off + s),
                   (uint32_t)c, t_pt, jb.sk0, jb.sk1, [&](int k) { atomicAdd(&ctr[CTR_PT + k], 1ull); },
                   [&]() { atomicAdd(&ctr[CTR_NEAR], 1ull); });
    trip_chain(dv, (size_t)chain, jb.T, dv.slot + base, t_pt + 1u);
  }
  grid_done_advance(dv.ctr, 0ull, 1ull, 0ull);
}

namespace {
typedef void (*int8_fn)(Job, Dev, int, int);

template <bool FUSE, bool EONLY>
int8_fn pick_int8(int d, int nt) {
  if (nt == 512) return d == 2 ? k_resident_int8<2, 512, FUSE, EONLY> : k_resident_int8<3, 512, FUSE, EONLY>;
  return d == 2 ? k_resident_int8<2, 256, FUSE, EONLY> : k_resident_int8<3, 256, FUSE, EONLY>;
}

template <int MAXJ>
using packed_fn = void (*)(ResidentParams<MAXJ>);

template <int D, int WPC, bool EONLY, int MAXJ, bool MEAS = false, bool FULLW = false, int HOUD = 0>
packed_fn<MAXJ> pick_packed_nt(int nt) {
  switch (nt) {
  case 64: return k_resident_packed<D, 64, WPC, EONLY, MAXJ, MEAS, FULLW, HOUD>;
  case 128: return k_resident_packed<D, 128, WPC, EONLY, MAXJ, MEAS, FULLW, HOUD>;
  case 256: return k_resident_packed<D, 256, WPC, EONLY, MAXJ, MEAS, FULLW, HOUD>;
  case 512: return k_resident_packed<D, 512, WPC, EONLY, MAXJ, MEAS, FULLW, HOUD>;
  default: return k_resident_packed<D, 1024, WPC, EONLY, MAXJ, MEAS, FULLW, HOUD>;
  }
}
// the kernels that take a phase of the Houdayer move (two one-word chains per CTA):
// HOUD 1 the sweeps before it (q bitmaps out), HOUD 2 the energies after it (flips in)
template <int HOUD, bool FULLW = false>
packed_fn<1> pick_packed_houd(int d, int nt) {
  constexpr bool EONLY = HOUD == 2;
  return d == 2 ? pick_packed_nt<2, 2, EONLY, 1, false, FULLW, HOUD>(nt)
                : pick_packed_nt<3, 2, EONLY, 1, false, FULLW, HOUD>(nt);
}
// the sweep kernel that measures after its last MCS (two one-word chains per CTA)
template <bool FULLW>
packed_fn<1> pick_packed_meas(int d, int nt) {
  return d == 2 ? pick_packed_nt<2, 2, false, 1, true, FULLW>(nt) : pick_packed_nt<3, 2, false, 1, true, FULLW>(nt);
}

template <bool EONLY, int MAXJ, bool FULLW = false>
packed_fn<MAXJ> pick_packed(int d, int nt, int wpc) {
  if (d == 2)
    return wpc == 2 ? pick_packed_nt<2, 2, EONLY, MAXJ, false, FULLW>(nt) : pick_packed_nt<2, 1, EONLY, MAXJ, false, FULLW>(nt);
  return wpc == 2 ? pick_packed_nt<3, 2, EONLY, MAXJ, false, FULLW>(nt) : pick_packed_nt<3, 1, EONLY, MAXJ, false, FULLW>(nt);
}
} // namespace

cudaError_t launch_resident(const Job &jb, const Dev &dv, bool int8fmt, int nthreads, int wpc, bool fuse_pt,
                            bool energy_only, size_t smem, cudaStream_t st, int n_mcs, int n_metro,
                            int32_t *meas_E, int32_t *meas_Q, bool after_move, const HoudMaps *hm, int houd) {
  if (int8fmt) {
    // small chains: enough threads that a half-sweep is one pass of (group, 32 sites) items
    const int chunks = (jb.Tp / 4) * ((jb.g.Nh + 31) / 32);
    const int nt = chunks > 8 && chunks <= 16 ? 512 : 256;
    int8_fn fn;
    if (energy_only && fuse_pt) fn = pick_int8<true, true>(jb.g.d, nt);
    else if (energy_only) fn = pick_int8<false, true>(jb.g.d, nt);
    else if (fuse_pt) fn = pick_int8<true, false>(jb.g.d, nt);
    else fn = pick_int8<false, false>(jb.g.d, nt);
    fn<<<(unsigned)(jb.S * jb.C), (unsigned)nt, smem, st>>>(jb, dv, n_mcs, n_metro);
    return cudaGetLastError();
  }
  ResidentParams<1> rp;
  rp.n_jobs = 1;
  rp.n_mcs = n_mcs;
  rp.pad0 = energy_only && after_move ? 1 : 0;
  rp.pad1 = 0;
  // the fused measurement needs both one-word chains of a sample in every CTA
  const bool meas = meas_E && !energy_only && fuse_pt && jb.C == 2 && jb.Wc == 1 && wpc == 2;
  if (meas_E && !meas) return cudaErrorInvalidValue;
  rp.mE = meas ? meas_E : nullptr;
  rp.mQ = meas ? meas_Q : nullptr;
  rp.jobs[0].jb = jb;
  rp.jobs[0].dv = dv;
  rp.jobs[0].first_item = 0;
  rp.jobs[0].n_items = jb.S * (jb.W / wpc);
  rp.jobs[0].fuse = fuse_pt ? 1 : 0;
  rp.jobs[0].n_metro = n_metro;
  const bool full = jb.T % 32 == 0; // every word of the job is full
  if (houd != 0) {
    // a phase of the Houdayer move: the CTA must hold both one-word chains of its sample
    const bool ok = hm && !int8fmt && wpc == 2 && jb.C == 2 && jb.Wc == 1 && !meas &&
                    (houd == 1 ? !energy_only : (houd == 2 && energy_only && after_move && fuse_pt));
    if (!ok) return cudaErrorInvalidValue;
    rp.hm = *hm;
  } else {
    rp.hm = HoudMaps{};
  }
  const packed_fn<1> fn = houd == 1    ? (full ? pick_packed_houd<1, true>(jb.g.d, nthreads)
                                               : pick_packed_houd<1, false>(jb.g.d, nthreads))
                          : houd == 2  ? pick_packed_houd<2>(jb.g.d, nthreads)
                          : meas       ? (full ? pick_packed_meas<true>(jb.g.d, nthreads) : pick_packed_meas<false>(jb.g.d, nthreads))
                          : energy_only ? pick_packed<true, 1>(jb.g.d, nthreads, wpc)
                          : full        ? pick_packed<false, 1, true>(jb.g.d, nthreads, wpc)
                                        : pick_packed<false, 1>(jb.g.d, nthreads, wpc);
  fn<<<(unsigned)rp.jobs[0].n_items, nthreads, smem, st>>>(rp);
  return cudaGetLastError();
}

cudaError_t launch_resident_batch(JobDesc *jobs, int n_jobs, int nthreads, int wpc, size_t smem, cudaStream_t st,
                                  int n_mcs) {
  for (int base = 0; base < n_jobs; base += MAX_BATCH_JOBS) {
    const int n = n_jobs - base < MAX_BATCH_JOBS ? n_jobs - base : MAX_BATCH_JOBS;
    std::vector<char> raw(sizeof(ResidentParams<MAX_BATCH_JOBS>));
    ResidentParams<MAX_BATCH_JOBS> &rp = *reinterpret_cast<ResidentParams<MAX_BATCH_JOBS> *>(raw.data());
    rp.n_jobs = n;
    rp.n_mcs = n_mcs;
    rp.pad0 = rp.pad1 = 0;
    rp.mE = rp.mQ = nullptr;
    int items = 0;
    for (int i = 0; i < n; ++i) {
      rp.jobs[i] = jobs[base + i];
      rp.jobs[i].first_item = items;
      items += rp.jobs[i].n_items;
    }
    const packed_fn<MAX_BATCH_JOBS> fn = pick_packed<false, MAX_BATCH_JOBS>(jobs[base].jb.g.d, nthreads, wpc);
    fn<<<(unsigned)items, nthreads, smem, st>>>(rp);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Allow every resident kernel the device's full opt-in shared memory (the attribute only
// caps what a launch may request; it does not change occupancy).  Not a stream operation,
// so it is done once per device before any launch or capture.
cudaError_t prepare_resident_kernels(int max_smem) {
  std::vector<const void *> fns;
  for (int d = 2; d <= 3; ++d)
    for (int nt : {64, 128, 256, 512, 1024})
      for (int wpc = 1; wpc <= 2; ++wpc) {
        fns.push_back((const void *)pick_packed<false, 1>(d, nt, wpc));
        fns.push_back((const void *)pick_packed<false, 1, true>(d, nt, wpc));
        fns.push_back((const void *)pick_packed<true, 1>(d, nt, wpc));
        fns.push_back((const void *)pick_packed<false, MAX_BATCH_JOBS>(d, nt, wpc));
        if (wpc == 2) {
          fns.push_back((const void *)pick_packed_meas<false>(d, nt));
          fns.push_back((const void *)pick_packed_meas<true>(d, nt));
          fns.push_back((const void *)pick_packed_houd<1, false>(d, nt));
          fns.push_back((const void *)pick_packed_houd<1, true>(d, nt));
          fns.push_back((const void *)pick_packed_houd<2>(d, nt));
        }
      }
  for (int d = 2; d <= 3; ++d)
    for (int nt : {256, 512}) {
      fns.push_back((const void *)pick_int8<false, false>(d, nt));
      fns.push_back((const void *)pick_int8<true, false>(d, nt));
      fns.push_back((const void *)pick_int8<false, true>(d, nt));
      fns.push_back((const void *)pick_int8<true, true>(d, nt));
    }
  for (const void *fn : fns) {
    // what a launch may add to the kernel's static shared memory
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Exchange passes of many jobs in one launch: CTAs [first_item, first_item + n_items) of
// the grid belong to job j (128 chains per CTA), one thread per (sample, chain).
__global__ void k_exchange_batch(const __grid_constant__ ResidentParams<MAX_BATCH_JOBS> rp) {
  int jsel = 0;
  for (int q = 1; q < rp.n_jobs; ++q)
    if ((int)blockIdx.x >= rp.jobs[q].first_item) jsel = q;
  const JobDesc &JD = rp.jobs[jsel];
  const Job &jb = JD.jb;
  const Dev &dv = JD.dv;
  const int chain = ((int)blockIdx.x - JD.first_item) * blockDim.x + threadIdx.x;
  const uint32_t t_pt = (uint32_t)dv.ctr[CTR_TPT];
  if (chain < jb.S * jb.C) {
    const int s = chain / jb.C;
    const int c = chain - s * jb.C;
    const size_t base = (size_t)chain * jb.T;
    unsigned long long *ctr = dv.ctr;
    exchange_chain(jb.T, dv.beta, dv.perm + base, dv.slot + base, dv.E + base, (uint32_t)(jb.s_off + s),
                   (uint32_t)c, t_pt, jb.sk0, jb.sk1, [&](int k) { atomicAdd(&ctr[CTR_PT + k], 1ull); },
                   [&]() { atomicAdd(&ctr[CTR_NEAR], 1ull); });
    trip_chain(dv, (size_t)chain, jb.T, dv.slot + base, t_pt + 1u);
  }
  job_done_advance(dv.ctr, JD.n_items, 0ull, 1ull, 0ull);
}

cudaError_t launch_exchange_batch(JobDesc *jobs, int n_jobs, cudaStream_t st) {
  for (int base = 0; base < n_jobs; base += MAX_BATCH_JOBS) {
    const int n = n_jobs - base < MAX_BATCH_JOBS ? n_jobs - base : MAX_BATCH_JOBS;
    std::vector<char> raw(sizeof(ResidentParams<MAX_BATCH_JOBS>));
    ResidentParams<MAX_BATCH_JOBS> &rp = *reinterpret_cast<ResidentParams<MAX_BATCH_JOBS> *>(raw.data());
    rp.n_jobs = n;
    rp.n_mcs = 1;
    rp.pad0 = rp.pad1 = 0;
    rp.mE = rp.mQ = nullptr;
    int ctas = 0;
    for (int i = 0; i < n; ++i) {
      rp.jobs[i] = jobs[base + i];
      rp.jobs[i].first_item = ctas;
      rp.jobs[i].n_items = (jobs[base + i].jb.S * jobs[base + i].jb.C + 127) / 128;
      ctas += rp.jobs[i].n_items;
    }
    k_exchange_batch<<<(unsigned)ctas, 128, 0, st>>>(rp);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_exchange(const Job &jb, const Dev &dv, cudaStream_t st) {
  const long long chains = (long long)jb.S * jb.C;
  k_exchange<<<(unsigned)((chains + 127) / 128), 128, 0, st>>>(jb, dv);
  return cudaGetLastError();
}

} // namespace sgmc
