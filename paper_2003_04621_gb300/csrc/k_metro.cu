// k_metro.cu -- the resident Metropolis kernels' instantiations and launchers (Sec. 2.2 /
// 2.4 step 1), the resident int8 kernel, and the standalone exchange kernels (Eq. 5).
// The packed kernel's template is in sgmc_resident.cuh; its instantiations that pair the
// two chains' partial words of a sample are in k_metro_pair.cu.
#include "sgmc_resident.cuh"

#include <vector>

namespace sgmc {

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
// HOUD 1 the sweeps before it (q bitmaps out), HOUD 2 the energies after it (flips in),
// HOUD 3 both around one MCS's sweeps (flips, energies and exchange in; q bitmaps out)
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

// the device's opt-in shared memory per CTA (prepare_resident_kernels)
static int g_max_smem = 0;

cudaError_t launch_resident(const Job &jb, const Dev &dv, bool int8fmt, int nthreads, int wpc, bool fuse_pt,
                            bool energy_only, size_t smem, cudaStream_t st, int n_mcs, int n_metro,
                            int32_t *meas_E, int32_t *meas_Q, bool after_move, const HoudMaps *hm, int houd,
                            bool allow_pair) {
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
  if (allow_pair && fuse_pt && !energy_only && !meas && houd == 0) {
    // chains whose last words hold at most 16 replicas: one CTA per sample, those words paired
    int pnt = nthreads;
    size_t psm = 0;
    const int pw = pair_words(jb, &pnt, g_max_smem, &psm);
    if (pw) {
      rp.jobs[0].n_items = jb.S;
      rp.hm = HoudMaps{};
      pair_kernel_1(jb.g.d, pnt, pw)<<<(unsigned)jb.S, (unsigned)pnt, psm, st>>>(rp);
      return cudaGetLastError();
    }
  }
  if (houd != 0) {
    // a phase of the Houdayer move: the CTA must hold both one-word chains of its sample
    const bool ok = hm && !int8fmt && wpc == 2 && jb.C == 2 && jb.Wc == 1 && !meas &&
                    (houd == 1   ? !energy_only
                     : houd == 2 ? energy_only && after_move && fuse_pt
                                 : houd == 3 && !energy_only && fuse_pt && n_mcs == 1);
    if (!ok) return cudaErrorInvalidValue;
    rp.hm = *hm;
  } else {
    rp.hm = HoudMaps{};
  }
  const packed_fn<1> fn = houd == 1    ? (full ? pick_packed_houd<1, true>(jb.g.d, nthreads)
                                               : pick_packed_houd<1, false>(jb.g.d, nthreads))
                          : houd == 3  ? (full ? pick_packed_houd<3, true>(jb.g.d, nthreads)
                                               : pick_packed_houd<3, false>(jb.g.d, nthreads))
                          : houd == 2  ? pick_packed_houd<2>(jb.g.d, nthreads)
                          : meas       ? (full ? pick_packed_meas<true>(jb.g.d, nthreads) : pick_packed_meas<false>(jb.g.d, nthreads))
                          : energy_only ? pick_packed<true, 1>(jb.g.d, nthreads, wpc)
                          : full        ? pick_packed<false, 1, true>(jb.g.d, nthreads, wpc)
                                        : pick_packed<false, 1>(jb.g.d, nthreads, wpc);
  fn<<<(unsigned)rp.jobs[0].n_items, nthreads, smem, st>>>(rp);
  return cudaGetLastError();
}

cudaError_t launch_resident_batch(JobDesc *jobs, int n_jobs, int nthreads, int wpc, size_t smem, cudaStream_t st,
                                  int n_mcs, bool pair) {
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
    const packed_fn<MAX_BATCH_JOBS> fn = pair ? pair_kernel_batch(jobs[base].jb.g.d, nthreads, wpc)
                                              : pick_packed<false, MAX_BATCH_JOBS>(jobs[base].jb.g.d, nthreads, wpc);
    if (!fn) return cudaErrorInvalidValue;
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
  g_max_smem = max_smem;
  if (const cudaError_t ep = prepare_pair_kernels(max_smem)) return ep;
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
          fns.push_back((const void *)pick_packed_houd<3, false>(d, nt));
          fns.push_back((const void *)pick_packed_houd<3, true>(d, nt));
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
