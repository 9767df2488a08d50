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
#include "sgmc_internal.cuh"
#include "sgmc_tma.cuh"

namespace sgmc {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr int NB = 8; // bit planes of the per-thread vertical counters (sum <= 255)

// Add the 3-plane value (v0, v1, v2) (weights 1, 2, 4) into the NB-plane counter V.
__device__ __forceinline__ void vcount_add(uint32_t (&V)[NB], uint32_t v0, uint32_t v1, uint32_t v2) {
  uint32_t c = V[0] & v0;
  V[0] ^= v0;
  uint32_t s, c2;
  fadd(V[1], v1, c, s, c2);
  V[1] = s;
  c = c2;
  fadd(V[2], v2, c, s, c2);
  V[2] = s;
  c = c2;
#pragma unroll
  for (int b = 3; b < NB; ++b) {
    s = V[b] ^ c;
    c = V[b] & c;
    V[b] = s;
  }
}

// Butterfly-add the warp's 32 vertical counters; return lane l's total for replica
// lane l (the value of bit l summed over the warp's counters, with weights).
__device__ __forceinline__ int32_t warp_lane_sum(const uint32_t (&V)[NB]) {
  uint32_t P[NB + 5];
#pragma unroll
  for (int b = 0; b < NB + 5; ++b) P[b] = b < NB ? V[b] : 0u;
#pragma unroll
  for (int lvl = 0; lvl < 5; ++lvl) {
    const int off = 16 >> lvl;
    uint32_t cy = 0;
#pragma unroll
    for (int b = 0; b < NB + 5; ++b) {
      if (b <= NB + lvl) {
        const uint32_t o = (b < NB + lvl) ? __shfl_xor_sync(FULL, P[b], off) : 0u;
        const uint32_t s = P[b] ^ o ^ cy;
        cy = (P[b] & o) | (cy & (P[b] ^ o));
        P[b] = s;
      }
    }
  }
  const int lane = threadIdx.x & 31;
  int32_t v = 0;
#pragma unroll
  for (int b = 0; b < NB + 5; ++b) v |= (int32_t)((P[b] >> lane) & 1u) << b;
  return v;
}

// One checkerboard half-sweep over the colour-`col` sites of a resident word lattice.
// ACCUM: add each site's post-update unsatisfied count to V.  NOFLIP: count only.
template <int D, int NT, bool ACCUM, bool NOFLIP>
__device__ __forceinline__ void half_sweep(const Geo &g, int col, uint32_t *__restrict__ sp,
                                           const uint8_t *__restrict__ jbyte,
                                           const uint32_t *__restrict__ thr_lane, uint32_t vmask,
                                           int ngroups, uint32_t t, uint32_t s_glob, uint32_t c3base,
                                           uint32_t k0, uint32_t k1, uint32_t (&V)[NB]) {
  const int H = g.H, L1 = g.L1, Nh = g.Nh;
  uint32_t *own = sp + col * Nh;
  const uint32_t *oth = sp + (1 - col) * Nh;
  const uint8_t *jown = jbyte + col * Nh;
  for (int q = threadIdx.x; q < Nh; q += NT) {
    const int row = q / H;
    const int k = q - row * H;
    int y, z;
    if (D == 3) {
      z = row / L1;
      y = row - z * L1;
    } else {
      y = row;
      z = 0;
    }
    const int xodd = col ^ ((y + z) & 1);
    const int rb = row * H;
    const int kxp = xodd ? (k + 1 == H ? 0 : k + 1) : k;
    const int kxm = xodd ? k : (k == 0 ? H - 1 : k - 1);
    const int ryp = (y + 1 == L1) ? row - (L1 - 1) : row + 1;
    const int rym = (y == 0) ? row + (L1 - 1) : row - 1;
    const uint32_t s0 = own[q];
    const uint32_t jb = jown[q];
    const uint32_t x0 = s0 ^ oth[rb + kxp] ^ (0u - (jb & 1u));
    const uint32_t x1 = s0 ^ oth[rb + kxm] ^ (0u - ((jb >> 1) & 1u));
    const uint32_t x2 = s0 ^ oth[ryp * H + k] ^ (0u - ((jb >> 2) & 1u));
    const uint32_t x3 = s0 ^ oth[rym * H + k] ^ (0u - ((jb >> 3) & 1u));
    uint32_t sA, cA, u0, u1, u2, aut;
    uint32_t sB = 0, cB = 0;
    fadd(x0, x1, x2, sA, cA);
    if (D == 3) {
      const int L2 = g.L2;
      const int rzp = (z + 1 == L2) ? row - (L2 - 1) * L1 : row + L1;
      const int rzm = (z == 0) ? row + (L2 - 1) * L1 : row - L1;
      const uint32_t x4 = s0 ^ oth[rzp * H + k] ^ (0u - ((jb >> 4) & 1u));
      const uint32_t x5 = s0 ^ oth[rzm * H + k] ^ (0u - ((jb >> 5) & 1u));
      fadd(x3, x4, x5, sB, cB);
      u0 = sA ^ sB;
      const uint32_t tt = sA & sB;
      fadd(cA, cB, tt, u1, u2);
      aut = u2 | (u1 & u0); // u >= 3
    } else {
      u0 = sA ^ x3;
      const uint32_t tt = sA & x3;
      u1 = cA ^ tt;
      u2 = cA & tt;
      aut = u1 | u2; // u >= 2
      sB = x3;       // kept for the post-flip count below
    }
    uint32_t F = 0;
    if (!NOFLIP) {
      uint32_t acc = aut;
      const uint32_t i = (uint32_t)(g.L0 * row + 2 * k + xodd);
#pragma unroll
      for (int gi = 0; gi < 8; ++gi) {
        if (gi < ngroups) {
          const uint4 r = philox10(i, t, s_glob, c3base | ((uint32_t)gi << 8), k0, k1);
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const int j = gi * 4 + qq;
            uint32_t idx;
            if (D == 3) idx = ((u0 >> j) & 1u) | (((u1 >> j) & 1u) << 1);
            else idx = (u0 >> j) & 1u;
            if (word_of(r, qq) < thr_lane[j * 4 + idx]) acc |= 1u << j;
          }
        }
      }
      F = acc & vmask;
      own[q] = s0 ^ F;
    }
    if (ACCUM) {
      // counts after the flip: flipping s_i toggles every bond of i, so each adder
      // input, sum and carry plane is toggled by F; the low bit of u is unchanged.
      uint32_t v1, v2;
      if (D == 3) {
        const uint32_t sA2 = sA ^ F, sB2 = sB ^ F, cA2 = cA ^ F, cB2 = cB ^ F;
        fadd(cA2, cB2, sA2 & sB2, v1, v2);
      } else {
        const uint32_t sA2 = sA ^ F, x32 = sB ^ F, cA2 = cA ^ F;
        const uint32_t tt2 = sA2 & x32;
        v1 = cA2 ^ tt2;
        v2 = cA2 & tt2;
      }
      vcount_add(V, u0, v1, v2);
    }
  }
}

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

template <int D, int NT, bool FUSE_PT, bool ENERGY_ONLY>
__global__ void __launch_bounds__(NT) k_resident_packed(Job jb, Dev dv, uint32_t t_metro0,
                                                        uint32_t t_pt0, int n_mcs, int n_metro) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Geo g = jb.g;
  const PackedSmem L = packed_smem(g.N, g.NW, D, NT);
  uint32_t *sp = reinterpret_cast<uint32_t *>(smem + L.spin);
  uint8_t *jbyte = smem + L.jbyte;
  uint32_t *jpl = reinterpret_cast<uint32_t *>(smem + L.jpl);
  uint32_t *thr_lane = reinterpret_cast<uint32_t *>(smem + L.thr);
  int32_t *epart = reinterpret_cast<int32_t *>(smem + L.epart);
  int32_t *pm = reinterpret_cast<int32_t *>(smem + L.pt);
  int32_t *sl = pm + 32;
  int32_t *el = sl + 32;
  unsigned int *pacc = reinterpret_cast<unsigned int *>(el + 32);
  unsigned int *pnear = pacc + 32;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);

  const int tid = threadIdx.x;
  const int item = blockIdx.x;
  const int s = item / jb.W;
  const int w = item - s * jb.W;
  const int c = w / jb.Wc;
  const int wc = w - c * jb.Wc;
  const uint32_t s_glob = (uint32_t)(jb.s_off + s);
  const int nvalid = min(32, jb.T - wc * 32);
  const uint32_t vmask = nvalid >= 32 ? FULL : ((1u << nvalid) - 1u);
  const int ngroups = (nvalid + 3) >> 2;
  uint32_t *gsp = dv.spins + ((size_t)s * jb.W + w) * g.N;
  const uint32_t *gj = dv.jbits + (size_t)s * D * g.NW;
  const size_t chain_base = ((size_t)s * jb.C + c) * jb.T;

  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  if (tid == 0) {
    const uint32_t sbytes = 4u * (uint32_t)g.N, jbytes = 4u * (uint32_t)(D * g.NW);
    mbar_expect_tx(bar, sbytes + jbytes);
    bulk_g2s(sp, gsp, sbytes, bar);
    bulk_g2s(jpl, gj, jbytes, bar);
  }
  if (tid < 32) {
    if (FUSE_PT) {
      pm[tid] = tid < jb.T ? dv.perm[chain_base + tid] : 0;
      sl[tid] = tid < jb.T ? dv.slot[chain_base + tid] : 0;
      pacc[tid] = 0u;
      if (tid == 0) *pnear = 0u;
    }
    if (!ENERGY_ONLY) {
      const int j = wc * 32 + tid;
      uint32_t tv[4] = {0u, 0u, 0u, 0u};
      if (tid < nvalid) {
        const int kslot = FUSE_PT ? sl[tid] : dv.slot[chain_base + j];
#pragma unroll
        for (int idx = 0; idx < D; ++idx) tv[idx] = dv.thr[kslot * 4 + (D - idx)];
      }
#pragma unroll
      for (int idx = 0; idx < 4; ++idx) thr_lane[tid * 4 + idx] = tv[idx];
    }
  }
  const bool ok = mbar_wait(bar, 0, MBAR_MAX_TRIES);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      atomicOr(&dv.ctr[CTR_ERROR], ERR_TMA_TIMEOUT);
      mbar_wait(bar, 0, MBAR_MAX_TRIES); // let copies still in flight land before exiting
    }
    return;
  }
  expand_couplings<D, NT>(g, jpl, jbyte);
  __syncthreads();

  const uint32_t c3base = ((uint32_t)c << 20) | ((uint32_t)(wc * 8) << 8) | TAG_METRO;
  const int n_outer = ENERGY_ONLY ? 1 : n_mcs;
  const int n_inner = ENERGY_ONLY ? 1 : n_metro;
  for (int m = 0; m < n_outer; ++m) {
    for (int swp = 0; swp < n_inner; ++swp) {
      const uint32_t t = t_metro0 + (uint32_t)(m * n_metro + swp);
      uint32_t V[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) V[b] = 0u;
      if (!ENERGY_ONLY) {
        half_sweep<D, NT, false, false>(g, 0, sp, jbyte, thr_lane, vmask, ngroups, t, s_glob, c3base,
                                        jb.sk0, jb.sk1, V);
        __syncthreads();
      }
      half_sweep<D, NT, true, ENERGY_ONLY>(g, 1, sp, jbyte, thr_lane, vmask, ngroups, t, s_glob, c3base,
                                           jb.sk0, jb.sk1, V);
      const int32_t part = warp_lane_sum(V);
      epart[tid] = part; // warp (tid / 32), lane (tid % 32)
      __syncthreads();
      if (tid < 32) {
        int32_t U = 0;
        for (int wq = 0; wq < NT / 32; ++wq) U += epart[wq * 32 + tid];
        el[tid] = 2 * U - D * g.N;
      }
      __syncthreads();
    }
    if (FUSE_PT) {
      if (tid == 0)
        exchange_chain(jb.T, dv.beta, pm, sl, el, s_glob, (uint32_t)c, t_pt0 + (uint32_t)m, jb.sk0, jb.sk1,
                       [&](int k) { pacc[k] += 1u; }, [&]() { *pnear += 1u; });
      __syncthreads();
      if (tid < nvalid) {
        const int kslot = sl[tid];
#pragma unroll
        for (int idx = 0; idx < D; ++idx) thr_lane[tid * 4 + idx] = dv.thr[kslot * 4 + (D - idx)];
      }
      __syncthreads();
    }
  }

  if (tid < nvalid) dv.E[chain_base + wc * 32 + tid] = el[tid];
  if (FUSE_PT && tid < 32) {
    if (tid < jb.T) {
      dv.perm[chain_base + tid] = pm[tid];
      dv.slot[chain_base + tid] = sl[tid];
    }
    if (tid + 1 < jb.T && pacc[tid]) atomicAdd(&dv.ctr[CTR_PT + tid], (unsigned long long)pacc[tid]);
    if (tid == 0 && *pnear) atomicAdd(&dv.ctr[CTR_NEAR], (unsigned long long)*pnear);
  }
  if (!ENERGY_ONLY) {
    fence_proxy_async(); // this thread's shared-memory writes -> visible to the TMA store
    __syncthreads();
    if (tid == 0) bulk_s2g_and_wait(gsp, sp, 4u * (uint32_t)g.N);
  }
}

// ---------------------------------------------------------------------------------
// int8 resident kernel: one CTA owns one chain (sample s, chain c) with all its replicas,
// spins as int8 +-1 (the paper's layout, replicas of a site adjacent, Sec. 3).  A thread
// item is (site of the colour, group of four replicas) -- one Philox call.
// ---------------------------------------------------------------------------------
template <int D, int NT, bool FUSE_PT, bool ENERGY_ONLY>
__global__ void __launch_bounds__(NT) k_resident_int8(Job jb, Dev dv, uint32_t t_metro0, uint32_t t_pt0,
                                                      int n_mcs, int n_metro) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Geo g = jb.g;
  const int T = jb.T, Tp = jb.Tp, G = Tp / 4;
  const Int8Smem L = int8_smem(g.N, g.NW, D, T, Tp);
  int8_t *sp8 = reinterpret_cast<int8_t *>(smem + L.spin);
  uint8_t *jbyte = smem + L.jbyte;
  uint32_t *jpl = reinterpret_cast<uint32_t *>(smem + L.jpl);
  uint32_t *thr = reinterpret_cast<uint32_t *>(smem + L.thr); // [Tp][4], entry m = 1..d
  int32_t *eacc = reinterpret_cast<int32_t *>(smem + L.eacc);
  int32_t *pm = reinterpret_cast<int32_t *>(smem + L.pm);
  int32_t *sl = reinterpret_cast<int32_t *>(smem + L.sl);
  unsigned int *pacc = reinterpret_cast<unsigned int *>(smem + L.pacc);
  unsigned int *pnear = reinterpret_cast<unsigned int *>(smem + L.near);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);

  const int tid = threadIdx.x;
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
  if (tid == 0) *pnear = 0u;
  __syncthreads();
  if (!ENERGY_ONLY)
    for (int j = tid; j < Tp; j += NT)
#pragma unroll
      for (int m = 0; m < 4; ++m) thr[j * 4 + m] = (j < T && m >= 1 && m <= D) ? dv.thr[sl[j] * 4 + m] : 0u;
  const bool ok = mbar_wait(bar, 0, MBAR_MAX_TRIES);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      atomicOr(&dv.ctr[CTR_ERROR], ERR_TMA_TIMEOUT);
      mbar_wait(bar, 0, MBAR_MAX_TRIES);
    }
    return;
  }
  expand_couplings<D, NT>(g, jpl, jbyte);
  __syncthreads();

  const int H = g.H, L1 = g.L1, Nh = g.Nh;
  const int n_outer = ENERGY_ONLY ? 1 : n_mcs;
  const int n_inner = ENERGY_ONLY ? 1 : n_metro;
  for (int m = 0; m < n_outer; ++m) {
    for (int swp = 0; swp < n_inner; ++swp) {
      const uint32_t t = t_metro0 + (uint32_t)(m * n_metro + swp);
      for (int col = ENERGY_ONLY ? 1 : 0; col < 2; ++col) {
        if (col == 1) {
          for (int j = tid; j < Tp; j += NT) eacc[j] = 0;
          __syncthreads();
        }
        for (int it = tid; it < Nh * G; it += NT) {
          const int q = it / G;
          const int gi = it - q * G;
          const int row = q / H;
          const int k = q - row * H;
          const int y = D == 3 ? row % L1 : row;
          const int z = D == 3 ? row / L1 : 0;
          const int xodd = col ^ ((y + z) & 1);
          SiteGeo sg;
          sg.c = col;
          sg.row = row;
          sg.k = k;
          sg.y = y;
          sg.z = z;
          sg.xodd = xodd;
          const int p = col * Nh + q;
          const uint32_t jbb = jbyte[p];
          char4 s4 = *reinterpret_cast<const char4 *>(sp8 + (size_t)p * Tp + 4 * gi);
          int h[4] = {0, 0, 0, 0};
#pragma unroll
          for (int mu = 0; mu < D; ++mu) {
#pragma unroll
            for (int dir = 0; dir < 2; ++dir) {
              const int pn = nbr_cs(g, sg, mu, dir == 0 ? 1 : -1);
              const char4 n4 = *reinterpret_cast<const char4 *>(sp8 + (size_t)pn * Tp + 4 * gi);
              const int Jv = ((jbb >> (2 * mu + dir)) & 1u) ? -1 : 1;
              h[0] += Jv * n4.x;
              h[1] += Jv * n4.y;
              h[2] += Jv * n4.z;
              h[3] += Jv * n4.w;
            }
          }
          int sv[4] = {s4.x, s4.y, s4.z, s4.w};
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
              const uint32_t i = (uint32_t)(g.L0 * row + 2 * k + xodd);
              rnd = philox10(i, t, s_glob, ((uint32_t)c << 20) | ((uint32_t)gi << 8) | TAG_METRO, jb.sk0,
                             jb.sk1);
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
          if (col == 1) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
              if (4 * gi + r < T) atomicAdd(&eacc[4 * gi + r], -sv[r] * h[r]);
          }
        }
        __syncthreads();
      }
    }
    if (FUSE_PT) {
      if (tid == 0)
        exchange_chain(T, dv.beta, pm, sl, eacc, s_glob, (uint32_t)c, t_pt0 + (uint32_t)m, jb.sk0, jb.sk1,
                       [&](int k) { pacc[k] += 1u; }, [&]() { *pnear += 1u; });
      __syncthreads();
      if (!ENERGY_ONLY)
        for (int j = tid; j < T; j += NT)
#pragma unroll
          for (int mm = 1; mm <= D; ++mm) thr[j * 4 + mm] = dv.thr[sl[j] * 4 + mm];
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
  if (!ENERGY_ONLY) {
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) bulk_s2g_and_wait(gsp, sp8, (uint32_t)(g.N * Tp));
  }
}

// Standalone exchange pass: one thread per (sample, chain), state in global memory.
__global__ void k_exchange(Job jb, Dev dv, uint32_t t_pt) {
  const int chain = blockIdx.x * blockDim.x + threadIdx.x;
  if (chain >= jb.S * jb.C) return;
  const int s = chain / jb.C;
  const int c = chain - s * jb.C;
  const size_t base = (size_t)chain * jb.T;
  unsigned long long *ctr = dv.ctr;
  exchange_chain(jb.T, dv.beta, dv.perm + base, dv.slot + base, dv.E + base, (uint32_t)(jb.s_off + s),
                 (uint32_t)c, t_pt, jb.sk0, jb.sk1, [&](int k) { atomicAdd(&ctr[CTR_PT + k], 1ull); },
                 [&]() { atomicAdd(&ctr[CTR_NEAR], 1ull); });
}

namespace {
typedef void (*resident_fn)(Job, Dev, uint32_t, uint32_t, int, int);

template <bool FUSE, bool EONLY>
resident_fn pick_packed(int d, int nt) {
  if (d == 2) {
    if (nt == 256) return k_resident_packed<2, 256, FUSE, EONLY>;
    if (nt == 512) return k_resident_packed<2, 512, FUSE, EONLY>;
    return k_resident_packed<2, 1024, FUSE, EONLY>;
  }
  if (nt == 256) return k_resident_packed<3, 256, FUSE, EONLY>;
  if (nt == 512) return k_resident_packed<3, 512, FUSE, EONLY>;
  return k_resident_packed<3, 1024, FUSE, EONLY>;
}

template <bool FUSE, bool EONLY>
resident_fn pick_int8(int d) {
  return d == 2 ? k_resident_int8<2, 256, FUSE, EONLY> : k_resident_int8<3, 256, FUSE, EONLY>;
}

template <bool FUSE, bool EONLY>
resident_fn pick(bool int8fmt, int d, int nt) {
  return int8fmt ? pick_int8<FUSE, EONLY>(d) : pick_packed<FUSE, EONLY>(d, nt);
}
} // namespace

cudaError_t launch_resident(const Job &jb, const Dev &dv, bool int8fmt, int nthreads, bool fuse_pt,
                            bool energy_only, size_t smem, cudaStream_t st, uint32_t t_metro0, uint32_t t_pt0,
                            int n_mcs, int n_metro) {
  resident_fn fn;
  if (energy_only) fn = pick<false, true>(int8fmt, jb.g.d, nthreads);
  else if (fuse_pt) fn = pick<true, false>(int8fmt, jb.g.d, nthreads);
  else fn = pick<false, false>(int8fmt, jb.g.d, nthreads);
  if (int8fmt) nthreads = 256;
  cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = int8fmt ? (unsigned)(jb.S * jb.C) : (unsigned)(jb.S * jb.W);
  fn<<<grid, nthreads, smem, st>>>(jb, dv, t_metro0, t_pt0, n_mcs, n_metro);
  return cudaGetLastError();
}

cudaError_t launch_exchange(const Job &jb, const Dev &dv, uint32_t t_pt, cudaStream_t st) {
  const long long chains = (long long)jb.S * jb.C;
  k_exchange<<<(unsigned)((chains + 127) / 128), 128, 0, st>>>(jb, dv, t_pt);
  return cudaGetLastError();
}

} // namespace sgmc
