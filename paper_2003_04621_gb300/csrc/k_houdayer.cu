// k_houdayer.cu -- the Houdayer cluster move (Sec. 2.4, Eq. 10) for every (sample,
// temperature slot) pair of chain-0 / chain-1 replicas, one CTA per sample.
//
// Pair k joins chain-0 replica a = perm0[k] and chain-1 replica b = perm1[k]; both live
// in one 32-replica word each (n_temps <= 32), at lanes a and b.  The pair is named by
// its chain-0 lane a below.
//
// Phase 1 (q field).  For every site, the chain-1 word is permuted lane b -> lane a
// (byte tables), so qa = w0 ^ sigma(w1) has bit a set where the pair's spins differ
// (q_i = -1).  A warp transposes 32 sites x 32 lanes in registers, giving each pair's
// q field as a bitmap over the lattice in canonical site order (rows of L0 bits, each
// row padded to RW words), and counts M (the q = -1 sites) per pair.
// Phase 2 (cluster).  One warp per pair: u is the pair's Philox word, the seed is the
// floor(u M / 2^32)-th set bit of the bitmap in canonical order, and the connected q = -1
// cluster of the seed is grown over rows: a row's part of the cluster is always a union
// of whole runs of the q bitmap (filled with carry propagation, periodic in x); a row
// that gained sites is queued, and processing it adds the runs of each neighbouring row
// (y +- 1, z +- 1) that touch it.  The work is proportional to the cluster's rows.
// Phase 3 (flip).  The cluster bitmaps are transposed back per 32-site block; the
// chain-0 word is xor-ed with the block's flip mask and the chain-1 word with its
// permutation back (lane a -> lane b): on the cluster the two replicas differ, so
// flipping both is the exchange of the two configurations.
// Energies are recomputed afterwards by the resident kernel (exact, bit-sliced), which
// also runs the exchange pass when the MCS continues with it.
#include "sgmc_houd.cuh"
#include "sgmc_internal.cuh"

namespace sgmc {

namespace {

constexpr int HNT = 1024; // threads per CTA (32 warps)

// Phase 0: the two chains' slot maps of sample s and the byte tables of the lane
// permutations: sig maps chain-1 lane b -> chain-0 lane a = perm0[slot1[b]] (built when
// `sig` is given), sigi maps chain-0 lane a -> chain-1 lane b = perm1[slot0[a]] (when
// `sigi` is given).  Ends with a CTA barrier.
__device__ __forceinline__ void houd_tables(const Job &jb, const Dev &dv, int s, int32_t *perm0, int32_t *perm1,
                                            int32_t *slot0, int32_t *slot1, uint32_t *sig, uint32_t *sigi) {
  const int T = jb.T, tid = threadIdx.x;
  if (tid < 32) {
    const size_t c0 = ((size_t)s * jb.C + 0) * T, c1 = ((size_t)s * jb.C + 1) * T;
    perm0[tid] = tid < T ? dv.perm[c0 + tid] : 0;
    perm1[tid] = tid < T ? dv.perm[c1 + tid] : 0;
    slot0[tid] = tid < T ? dv.slot[c0 + tid] : 0;
    slot1[tid] = tid < T ? dv.slot[c1 + tid] : 0;
  }
  __syncthreads();
  for (int e = tid; e < 1024; e += blockDim.x) {
    const int j = e >> 8, v = e & 255;
    uint32_t o1 = 0u, o2 = 0u;
#pragma unroll
    for (int bb = 0; bb < 8; ++bb) {
      const int lanei = 8 * j + bb;
      if (((v >> bb) & 1) && lanei < T) {
        o1 |= 1u << perm0[slot1[lanei]];
        o2 |= 1u << perm1[slot0[lanei]];
      }
    }
    if (sig) sig[e] = o1;
    if (sigi) sigi[e] = o2;
  }
  __syncthreads();
}

// Phase 1: the q bitmap of every pair of sample s (pair a's bitmap at Qb + a * NBW) and
// its number M of q = -1 sites, added into Mc[a].  Warps stride over the 32-site blocks.
__device__ __forceinline__ void houd_qmaps(const Job &jb, int RW, const uint32_t *w0p, const uint32_t *w1p,
                                           const uint32_t *sig, const int32_t *slot0, uint32_t *Qb, int NBW,
                                           uint32_t *Mc) {
  const int T = jb.T, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t tmask = houd_pair_mask(jb, slot0);
  const BlockMap bm = block_map(jb.g, RW);
  uint32_t mpart = 0u;
  for (int b = warp; b < NBW; b += nwarps) {
    bool valid;
    const int p = block_site(jb.g, bm, b, lane, valid);
    uint32_t qa = 0u;
    if (valid) qa = (w0p[p] ^ permute_word(sig, w1p[p])) & tmask;
    const uint32_t col = transpose32(qa, lane); // lane a: bit l = q of pair a at site l
    if (lane < T) {
      Qb[(size_t)lane * NBW + b] = col;
      mpart += __popc(col);
    }
  }
  if (lane < T && mpart) atomicAdd(&Mc[lane], mpart);
}

// Phase 2 for one pair, by one warp: choose the seed (the floor(u M / 2^32)-th q = -1 site
// in canonical order) and grow its q = -1 cluster into C (zeroed here) over rows.  The
// worklist (stack of rows, in-list bits, size) is the warp's own.  Returns the cluster's
// size on every lane (0 when M = 0).
template <int D, int RW>
__device__ uint32_t houd_fill_pair(const Geo &g, const uint32_t *Q, uint32_t *C, int NBW, uint32_t M, uint32_t u,
                                   uint16_t *stack, uint32_t *inlist, int *ssize, unsigned long long *err) {
  const int lane = threadIdx.x & 31;
  const int L0 = g.L0, L1 = g.L1, R = g.R;
  for (int b = lane; b < NBW; b += 32) C[b] = 0u;
  __syncwarp();
  if (M == 0u) return 0u;
  const uint32_t n = (uint32_t)(((unsigned long long)u * M) >> 32);
  // the n-th set bit in canonical order: contiguous chunks per lane, then a warp scan
  const int chunk = (NBW + 31) / 32;
  const int b0 = lane * chunk, b1 = min(NBW, b0 + chunk);
  uint32_t cnt = 0u;
  for (int b = b0; b < b1; ++b) cnt += __popc(Q[b]);
  uint32_t pre = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(FULLM, pre, o);
    if (lane >= o) pre += v;
  }
  pre -= cnt; // exclusive
  int seed_b = -1, seed_bit = 0;
  if (n >= pre && n < pre + cnt) {
    uint32_t rem = n - pre;
    for (int b = b0; b < b1; ++b) {
      uint32_t w = Q[b];
      const uint32_t pc = __popc(w);
      if (rem < pc) {
        for (uint32_t i = 0; i < rem; ++i) w &= w - 1u; // drop the lowest `rem` set bits
        seed_b = b;
        seed_bit = __ffs(w) - 1;
        break;
      }
      rem -= pc;
    }
  }
  const unsigned owner = __ballot_sync(FULLM, seed_b >= 0);
  const int src = __ffs(owner) - 1;
  seed_b = __shfl_sync(FULLM, seed_b, src);
  seed_bit = __shfl_sync(FULLM, seed_bit, src);
  for (int i = lane; i < (R + 31) / 32; i += 32) inlist[i] = 0u;
  __syncwarp();
  if (lane == 0) {
    const int r0 = seed_b / RW;
    uint32_t q[RW], x[RW], f[RW];
#pragma unroll
    for (int m = 0; m < RW; ++m) {
      q[m] = Q[r0 * RW + m];
      x[m] = (r0 * RW + m == seed_b) ? (1u << seed_bit) : 0u;
    }
    close_row<RW>(q, x, f, L0);
#pragma unroll
    for (int m = 0; m < RW; ++m) C[r0 * RW + m] = f[m];
    stack[0] = (uint16_t)r0;
    inlist[r0 >> 5] |= 1u << (r0 & 31);
    *ssize = 1;
  }
  __syncwarp();
  // rows: each round pops up to 32 queued rows, one per lane
  const int max_rounds = 4 * g.N + 64; // never reached: every push adds at least one site
  for (int round = 0; round < max_rounds; ++round) {
    const int size = *ssize;
    if (size == 0) break;
    const int take = min(32, size);
    int r = -1;
    if (lane < take) {
      r = stack[size - 1 - lane];
      atomicAnd(&inlist[r >> 5], ~(1u << (r & 31)));
    }
    __syncwarp();
    if (lane == 0) *ssize = size - take;
    __syncwarp();
    if (r >= 0) {
      const int y = r % L1, z = r / L1;
      int nrow[2 * (D - 1)];
      nrow[0] = (y + 1 == L1) ? r - (L1 - 1) : r + 1;
      nrow[1] = (y == 0) ? r + (L1 - 1) : r - 1;
      if (D == 3) {
        const int L2 = g.L2;
        nrow[2] = (z + 1 == L2) ? r - (L2 - 1) * L1 : r + L1;
        nrow[3] = (z == 0) ? r + (L2 - 1) * L1 : r - L1;
      }
#pragma unroll
      for (int t = 0; t < 2 * (D - 1); ++t) {
        const int nr = nrow[t];
        uint32_t q[RW], x[RW], f[RW];
        bool any = false;
#pragma unroll
        for (int m = 0; m < RW; ++m) {
          q[m] = Q[nr * RW + m];
          x[m] = q[m] & C[r * RW + m] & ~C[nr * RW + m];
          any |= x[m] != 0u;
        }
        if (!any) continue;
        close_row<RW>(q, x, f, L0);
        bool changed = false;
#pragma unroll
        for (int m = 0; m < RW; ++m) {
          const uint32_t old = atomicOr(&C[nr * RW + m], f[m]);
          changed |= (f[m] & ~old) != 0u;
        }
        if (changed) {
          const uint32_t bit = 1u << (nr & 31);
          if (!(atomicOr(&inlist[nr >> 5], bit) & bit)) {
            const int pos = atomicAdd(ssize, 1);
            stack[pos] = (uint16_t)nr;
          }
        }
      }
    }
    __syncwarp();
  }
  if (lane == 0 && *ssize > 0) atomicOr(err, ERR_HOUD_ROUNDS);
  uint32_t sz = 0u;
  for (int b = lane; b < NBW; b += 32) sz += __popc(C[b]);
  return __reduce_add_sync(FULLM, sz);
}

// Phase 3: flip both replicas of every pair of sample s on its cluster (pair a's
// cluster bitmap at Cb + a * NBW; pairs whose bit in `skip` is set have no cluster).
__device__ __forceinline__ void houd_flips(const Job &jb, int RW, const uint32_t *Cb, int NBW, uint32_t skip,
                                           const uint32_t *sigi, uint32_t *w0w, uint32_t *w1w) {
  const int T = jb.T, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const bool mine = lane < T && !((skip >> lane) & 1u);
  const BlockMap bm = block_map(jb.g, RW);
  for (int b = warp; b < NBW; b += nwarps) {
    const uint32_t cw = mine ? Cb[(size_t)lane * NBW + b] : 0u;
    if (!__any_sync(FULLM, cw != 0u)) continue;
    const uint32_t f0 = transpose32(cw, lane); // lane l: bit a = site l in pair a's cluster
    bool valid;
    const int p = block_site(jb.g, bm, b, lane, valid);
    if (valid && f0) {
      w0w[p] ^= f0;
      w1w[p] ^= permute_word(sigi, f0);
    }
  }
}

} // namespace

struct HoudArgs {
  int RW;  // words per bitmap row
  int NBW; // words per bitmap (rows x RW)
};

// Shared-memory map of the single-CTA Houdayer kernel (bitmaps_smem = 0 leaves out the
// bitmaps, for sizing only).
__host__ __device__ inline int houd_smem_bytes(int T, int R, int NBW, int bitmaps_smem, int *off_q, int *off_wl) {
  int off = 0;
  off += 2 * 1024 * 4;      // sig, sigi tables
  off += 4 * 32 * 4;        // perm0, perm1, slot0, slot1
  off += 32 * 4 + 16;       // M per pair, counters
  *off_q = off;
  if (bitmaps_smem) off += 2 * T * NBW * 4;
  *off_wl = off;
  const int wl = ((2 * R + 3) & ~3) + 4 * ((R + 31) / 32) + 4; // stack (u16), in-list bits, size
  off += (HNT / 32) * wl;
  return (off + 15) & ~15;
}

__host__ __device__ inline int houd_worklist_bytes(int R) { return ((2 * R + 3) & ~3) + 4 * ((R + 31) / 32) + 4; }

// Single-CTA form: one CTA of 1024 threads per sample runs all three phases, the
// bitmaps in shared memory.
template <int D, int RW>
__global__ void __launch_bounds__(HNT) k_houdayer(Job jb, Dev dv, HoudArgs ha) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Geo g = jb.g;
  const int T = jb.T, N = g.N, R = g.R;
  const int NBW = ha.NBW;
  int off_q, off_wl;
  houd_smem_bytes(T, R, NBW, 1, &off_q, &off_wl);
  uint32_t *sig = reinterpret_cast<uint32_t *>(smem);
  uint32_t *sigi = sig + 1024;
  int32_t *perm0 = reinterpret_cast<int32_t *>(sigi + 1024);
  int32_t *perm1 = perm0 + 32, *slot0 = perm0 + 64, *slot1 = perm0 + 96;
  uint32_t *Mc = reinterpret_cast<uint32_t *>(perm0 + 128);
  unsigned long long *cnts = reinterpret_cast<unsigned long long *>(Mc + 32); // moves, sites

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t t_houd = (uint32_t)dv.ctr[CTR_THOUD];
  const int s = blockIdx.x;
  const uint32_t s_glob = (uint32_t)(jb.s_off + s);
  uint32_t *Qb = reinterpret_cast<uint32_t *>(smem + off_q);
  uint32_t *Cb = Qb + (size_t)T * NBW;
  const int wl_bytes = houd_worklist_bytes(R);
  unsigned char *wl = smem + off_wl + warp * wl_bytes;
  uint16_t *stack = reinterpret_cast<uint16_t *>(wl);
  uint32_t *inlist = reinterpret_cast<uint32_t *>(wl + ((2 * R + 3) & ~3));
  int *ssize = reinterpret_cast<int *>(inlist + (R + 31) / 32);

  uint32_t *w0w = dv.spins + ((size_t)s * jb.W + 0) * N; // chain 0 word (Wc = 1)
  uint32_t *w1w = dv.spins + ((size_t)s * jb.W + 1) * N; // chain 1 word

  if (tid < 32) Mc[tid] = 0u;
  if (tid < 2) cnts[tid] = 0ull;
  houd_tables(jb, dv, s, perm0, perm1, slot0, slot1, sig, sigi);
  houd_qmaps(jb, RW, w0w, w1w, sig, slot0, Qb, NBW, Mc);
  __syncthreads();
  for (int a = warp; a < T; a += HNT / 32) {
    const uint32_t M = Mc[a];
    const uint32_t u = M ? philox10((uint32_t)slot0[a], t_houd, s_glob, TAG_HOUD, jb.sk0, jb.sk1).x : 0u;
    const uint32_t sz = houd_fill_pair<D, RW>(g, Qb + (size_t)a * NBW, Cb + (size_t)a * NBW, NBW, M, u, stack,
                                              inlist, ssize, &dv.ctr[CTR_ERROR]);
    if (lane == 0 && M) {
      atomicAdd(&cnts[0], 1ull);
      atomicAdd(&cnts[1], (unsigned long long)sz);
    }
  }
  __syncthreads();
  houd_flips(jb, RW, Cb, NBW, 0u, sigi, w0w, w1w);
  __syncthreads();
  if (tid == 0) {
    if (cnts[0]) atomicAdd(&dv.ctr[CTR_HMOVES], cnts[0]);
    if (cnts[1]) atomicAdd(&dv.ctr[CTR_HSITES], cnts[1]);
  }
  grid_done_advance(dv.ctr, 0ull, 0ull, 1ull);
}

// ---------------------------------------------------------------------------------
// Split form, used when the handle holds bitmap scratch for every pair.  The single-CTA
// form runs a sample's pairs in one CTA, so the sample's largest cluster holds the whole
// CTA, and samples run in waves of one CTA per SM.  Here the q bitmaps are written to
// scratch by one CTA per sample, then every pair's cluster is grown by its own warp in
// CTAs of a few pairs, all pairs of all samples in flight together, and the flips are
// applied by one CTA per sample.
// ---------------------------------------------------------------------------------
constexpr int HSPLIT_NT = 512;     // threads of the per-sample kernels
constexpr int HFILL_MAX_WARPS = 8; // pairs per CTA of the fill kernel, at most

// The per-sample kernels move the bitmaps between registers and global scratch through a
// shared-memory tile of HQ_TB blocks for every pair (row stride HQ_TB + 1: the lanes of a
// warp, one pair each, fall in distinct banks), so the global accesses are contiguous runs
// of each pair's bitmap.
constexpr int HQ_TB = 64, HQ_U = 4;

__global__ void __launch_bounds__(HSPLIT_NT) k_houd_q(Job jb, Dev dv, HoudSplit hs) {
  __shared__ uint32_t sig[1024];
  __shared__ int32_t maps[4][32];
  __shared__ uint32_t Mc[32];
  __shared__ uint32_t stage[32][HQ_TB + 1];
  const int s = blockIdx.x, T = jb.T, NBW = hs.NBW, RW = hs.RW;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = HSPLIT_NT / 32;
  if (tid < 32) Mc[tid] = 0u;
  houd_tables(jb, dv, s, maps[0], maps[1], maps[2], maps[3], sig, nullptr);
  const uint32_t *w0p = dv.spins + ((size_t)s * jb.W + 0) * jb.g.N;
  const uint32_t *w1p = dv.spins + ((size_t)s * jb.W + 1) * jb.g.N;
  uint32_t *Qb = hs.Qg + (size_t)s * T * NBW;
  const uint32_t tmask = houd_pair_mask(jb, maps[2]);
  const BlockMap bm = block_map(jb.g, RW);
  uint32_t mpart = 0u;
  for (int tb = blockIdx.y * HQ_TB; tb < NBW; tb += gridDim.y * HQ_TB) {
    const int nb = min(HQ_TB, NBW - tb);
    // HQ_U blocks per warp at a time: their words are loaded before any is used
    for (int j0 = warp; j0 < nb; j0 += nwarps * HQ_U) {
      uint32_t x0[HQ_U], x1[HQ_U];
#pragma unroll
      for (int u = 0; u < HQ_U; ++u) {
        const int j = j0 + u * nwarps;
        x0[u] = x1[u] = 0u;
        if (j < nb) {
          bool valid;
          const int p = block_site(jb.g, bm, tb + j, lane, valid);
          if (valid) {
            x0[u] = w0p[p];
            x1[u] = w1p[p];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < HQ_U; ++u) {
        const int j = j0 + u * nwarps;
        if (j < nb) {
          const uint32_t qa = (x0[u] ^ permute_word(sig, x1[u])) & tmask;
          const uint32_t col = transpose32(qa, lane); // lane a: bit l = q of pair a at site l
          stage[lane][j] = col;
          mpart += lane < T ? __popc(col) : 0u;
        }
      }
    }
    __syncthreads();
    for (int e = tid; e < T * nb; e += HSPLIT_NT) {
      const int a = e / nb, j = e - a * nb;
      Qb[(size_t)a * NBW + tb + j] = stage[a][j];
    }
    __syncthreads();
  }
  if (lane < T && mpart) atomicAdd(&Mc[lane], mpart);
  __syncthreads();
  // the sample's CTAs (blockIdx.y = part of its blocks) add into M, cleared before launch
  if (tid < 32 && Mc[tid]) atomicAdd(&hs.Mg[(size_t)s * 32 + tid], Mc[tid]);
}

template <int D, int RW, bool SMEM>
__global__ void __launch_bounds__(HFILL_MAX_WARPS * 32, 4) k_houd_fill(Job jb, Dev dv, HoudSplit hs) {
  // dynamic shared memory only (its size attribute is the device's whole opt-in amount):
  // the CTA's two counters, then one region per warp (bitmaps if in_smem, worklist)
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long *cnts = reinterpret_cast<unsigned long long *>(smem);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int NBW = hs.NBW, R = jb.g.R;
  const long long gp = (long long)blockIdx.x * hs.wpb + warp; // pair: sample gp / T, chain-0 lane gp % T
  const bool active = gp < (long long)jb.S * jb.T;
  const int s = active ? (int)(gp / jb.T) : 0;
  const int a = active ? (int)(gp - (long long)s * jb.T) : 0;
  if (threadIdx.x < 2) cnts[threadIdx.x] = 0ull;
  const int wl_bytes = houd_worklist_bytes(R);
  const int per_warp = (SMEM ? 2 * NBW * 4 : 0) + wl_bytes;
  unsigned char *mine = smem + HFILL_HEAD + (size_t)warp * per_warp;
  uint32_t *Qs = reinterpret_cast<uint32_t *>(mine);
  uint32_t *Cs = Qs + NBW;
  unsigned char *wl = mine + (SMEM ? 2 * NBW * 4 : 0);
  uint16_t *stack = reinterpret_cast<uint16_t *>(wl);
  uint32_t *inlist = reinterpret_cast<uint32_t *>(wl + ((2 * R + 3) & ~3));
  int *ssize = reinterpret_cast<int *>(inlist + (R + 31) / 32);
  __syncthreads();
  if (active) {
    const uint32_t M = hs.Mg[(size_t)s * 32 + a];
    uint32_t *Qp = hs.Qg + ((size_t)s * jb.T + a) * NBW;
    uint32_t *Cp = hs.Cg + ((size_t)s * jb.T + a) * NBW;
    if (M) {
      const uint32_t t_houd = (uint32_t)dv.ctr[CTR_THOUD];
      const int k = dv.slot[((size_t)s * jb.C + 0) * jb.T + a];
      const uint32_t u = philox10((uint32_t)k, t_houd, (uint32_t)(jb.s_off + s), TAG_HOUD, jb.sk0, jb.sk1).x;
      const uint32_t *Q = Qp;
      uint32_t *C = Cp;
      if (SMEM) {
        for (int b = lane; b < NBW; b += 32) Qs[b] = Qp[b];
        __syncwarp();
        Q = Qs;
        C = Cs;
      }
      const uint32_t sz = houd_fill_pair<D, RW>(jb.g, Q, C, NBW, M, u, stack, inlist, ssize, &dv.ctr[CTR_ERROR]);
      if (SMEM) {
        __syncwarp();
        for (int b = lane; b < NBW; b += 32) Cp[b] = Cs[b];
      }
      if (lane == 0) {
        atomicAdd(&cnts[0], 1ull);
        atomicAdd(&cnts[1], (unsigned long long)sz);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (cnts[0]) atomicAdd(&dv.ctr[CTR_HMOVES], cnts[0]);
    if (cnts[1]) atomicAdd(&dv.ctr[CTR_HSITES], cnts[1]);
  }
}

__global__ void __launch_bounds__(HSPLIT_NT) k_houd_flip(Job jb, Dev dv, HoudSplit hs) {
  __shared__ uint32_t sigi[1024];
  __shared__ int32_t maps[4][32];
  __shared__ uint32_t stage[32][HQ_TB + 1];
  __shared__ uint32_t skip_s;
  const int s = blockIdx.x, T = jb.T, NBW = hs.NBW, RW = hs.RW;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = HSPLIT_NT / 32;
  houd_tables(jb, dv, s, maps[0], maps[1], maps[2], maps[3], nullptr, sigi);
  // pairs without a q = -1 site have no cluster (their bitmaps were not written)
  if (warp == 0) {
    const uint32_t skip = __ballot_sync(FULLM, lane >= T || hs.Mg[(size_t)s * 32 + lane] == 0u);
    if (lane == 0) skip_s = skip;
  }
  __syncthreads();
  const uint32_t skip = skip_s;
  uint32_t *w0w = dv.spins + ((size_t)s * jb.W + 0) * jb.g.N;
  uint32_t *w1w = dv.spins + ((size_t)s * jb.W + 1) * jb.g.N;
  const uint32_t *Cb = hs.Cg + (size_t)s * T * NBW;
  const BlockMap bm = block_map(jb.g, RW);
  for (int tb = blockIdx.y * HQ_TB; tb < NBW; tb += gridDim.y * HQ_TB) {
    const int nb = min(HQ_TB, NBW - tb);
    for (int e = tid; e < T * nb; e += HSPLIT_NT) {
      const int a = e / nb, j = e - a * nb;
      stage[a][j] = ((skip >> a) & 1u) ? 0u : Cb[(size_t)a * NBW + tb + j];
    }
    __syncthreads();
    for (int j0 = warp; j0 < nb; j0 += nwarps * HQ_U) {
      uint32_t f[HQ_U], x0[HQ_U], x1[HQ_U];
      int pp[HQ_U];
#pragma unroll
      for (int u = 0; u < HQ_U; ++u) {
        const int j = j0 + u * nwarps;
        f[u] = 0u;
        pp[u] = -1;
        if (j < nb) {
          const uint32_t cw = lane < T ? stage[lane][j] : 0u;
          if (__any_sync(FULLM, cw != 0u)) {
            f[u] = transpose32(cw, lane); // lane l: bit a = site l in pair a's cluster
            bool valid;
            const int p = block_site(jb.g, bm, tb + j, lane, valid);
            if (valid && f[u]) pp[u] = p;
          }
        }
        x0[u] = pp[u] >= 0 ? w0w[pp[u]] : 0u;
        x1[u] = pp[u] >= 0 ? w1w[pp[u]] : 0u;
      }
#pragma unroll
      for (int u = 0; u < HQ_U; ++u) {
        if (pp[u] >= 0) {
          w0w[pp[u]] = x0[u] ^ f[u];
          w1w[pp[u]] = x1[u] ^ permute_word(sigi, f[u]);
        }
      }
    }
    __syncthreads();
  }
  grid_done_advance(dv.ctr, 0ull, 0ull, 1ull);
}

// ---------------------------------------------------------------------------------
// Labelling form of phase 2: one CTA per pair labels every q = -1 cluster of the pair by
// union-find over the runs of its bitmap rows, then keeps the cluster of the seed.
//
// A run is a maximal row segment of q = -1 sites, cut at x = 0 (so no run wraps); runs
// are numbered in canonical order, and the run of site (row r, x) is the number of run
// starts at or before it minus one.  Edges: the runs at x = 0 and x = L0-1 of a row
// (periodic wrap), and for every pair of neighbouring rows (y+1, and z+1 in 3D) the two
// runs over each segment where both rows have q = -1.  Components come from rounds of
// hooking and pointer jumping over the edge list (every lane does the same work in a
// round), which converge in a few rounds on these graphs.  The work is proportional to
// the runs, and the CTA's threads share it, so no pair waits on a long serial fill.
// ---------------------------------------------------------------------------------
constexpr int HLAB_NT = 256;

// Parents are 16-bit run numbers (a pair has at most N/2 <= 65536 runs).

// Position of the j-th (from 0) set bit of w; w has more than j set bits.
__device__ __forceinline__ int nth_set_bit(uint32_t w, int j) {
  for (int q = 0; q < j; ++q) w &= w - 1u;
  return __ffs(w) - 1;
}

// Run number of site (row r, x) from the run-start bitmap and the per-word start counts.
template <int RW>
__device__ __forceinline__ int run_of(const uint32_t *St, const int32_t *pre, int r, int x) {
  const int i = r * RW + (x >> 5), b = x & 31;
  return pre[i] + __popc(St[i] & (0xFFFFFFFFu >> (31 - b))) - 1;
}

// Exclusive prefix sum over the CTA of one value per thread (HLAB_NT threads); the total
// goes to *total.  `ws` holds HLAB_NT / 32 ints.  Contains CTA barriers.
__device__ __forceinline__ int cta_exclusive_scan(int v, int *ws, int *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULLM, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int w = lane < HLAB_NT / 32 ? ws[lane] : 0;
    int iw = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(FULLM, iw, o);
      if (lane >= o) iw += t;
    }
    if (lane < HLAB_NT / 32) ws[lane] = iw - w;
    if (lane == HLAB_NT / 32 - 1) ws[HLAB_NT / 32] = iw;
  }
  __syncthreads();
  const int ex = ws[warp] + inc - v;
  *total = ws[HLAB_NT / 32];
  __syncthreads();
  return ex;
}

// Edges of a pair's run graph, at most: one wrap per row, and per next row at most 16
// overlap segments per word.
__host__ __device__ inline int label_max_edges(int NBW, int R, int D) { return R + 16 * NBW * (D - 1); }

// Edges kept in shared memory: up to N/4 + R (a random q field with half its sites at
// -1 has about N/7); a pair with more recomputes its edges from the bitmaps every round.
__host__ __device__ inline int label_edge_cap(int NBW, int N, int R, int D) {
  const int m = label_max_edges(NBW, R, D), c = N / 4 + R;
  return m < c ? m : c;
}

// Shared-memory bytes of the labelling kernel: Q, run starts, run counts per word, scan
// space, coin bits, the edges (two 16-bit runs each), 16-bit parents (at most N/2 runs),
// neighbour rows.
__host__ __device__ inline int label_smem_bytes(int NBW, int N, int R, int D) {
  return 4 * (3 * NBW + 32 + (N / 64 + 1)) + 4 * label_edge_cap(NBW, N, R, D) + ((2 * (N / 2) + 7) & ~7) +
         ((2 * (D - 1) * R + 7) & ~7);
}

// MULTI: the multi-cluster variant -- every cluster is exchanged by its own coin, the top
// bit of the Philox word with counter (i_min, t_houd, s, k << 8 | TAG_HMULTI), i_min the
// cluster's smallest canonical site: the start of its root run (roots are the smallest
// run of their tree, and a run's start is its smallest site).
template <int D, int RW, bool MULTI>
__global__ void __launch_bounds__(HLAB_NT) k_houd_label(Job jb, Dev dv, HoudSplit hs) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Geo g = jb.g;
  const int NBW = hs.NBW, L0 = g.L0, L1 = g.L1, R = g.R;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int s = (int)(blockIdx.x / (unsigned)jb.T), a = (int)(blockIdx.x - (unsigned)s * jb.T);
  const uint32_t M = hs.Mg[(size_t)s * 32 + a];
  if (M == 0u) return; // no q = -1 site: no move (the flip kernel skips the pair)
  uint32_t *Q = reinterpret_cast<uint32_t *>(smem);
  uint32_t *St = Q + NBW;
  int32_t *pre = reinterpret_cast<int32_t *>(St + NBW); // runs before each word
  int32_t *misc = pre + NBW; // [0..8] scan space, [16] seed root, [17] size
  uint32_t *coin = reinterpret_cast<uint32_t *>(misc + 32); // MULTI: coin bit per run
  ushort2 *edges = reinterpret_cast<ushort2 *>(coin + g.N / 64 + 1); // run graph edges
  const int ecap = label_edge_cap(NBW, g.N, R, D);
  uint16_t *par = reinterpret_cast<uint16_t *>(edges + ecap); // parents, by run
  uint16_t *nrow = par + ((g.N / 2 + 3) & ~3); // [D-1][R] next row along y (and z)
  const uint32_t *Qp = hs.Qg + ((size_t)s * jb.T + a) * NBW;
  uint32_t *Cp = hs.Cg + ((size_t)s * jb.T + a) * NBW;
  for (int i = tid; i < NBW; i += HLAB_NT) Q[i] = Qp[i];
  for (int r = tid; r < R; r += HLAB_NT) {
    const int y = r % L1, z = r / L1;
    nrow[r] = (uint16_t)((y + 1 == L1) ? r - (L1 - 1) : r + 1);
    if (D == 3) nrow[R + r] = (uint16_t)((z + 1 == g.L2) ? r - (g.L2 - 1) * L1 : r + L1);
  }
  if (tid == 0) misc[17] = 0;
  __syncthreads();

  // run starts (runs cut at x = 0) and the edges of the run graph, counted per word
  // (contiguous chunks of words per thread): the row's wrap (at its first word), and one
  // edge per overlap segment with each next row along y (and z), segments cut at the
  // word edge
  const int chunk = (NBW + HLAB_NT - 1) / HLAB_NT;
  const int i0 = min(NBW, tid * chunk), i1 = min(NBW, i0 + chunk);
  int nst = 0, ned = 0;
  for (int i = i0; i < i1; ++i) {
    const int r = i / RW, m = i - r * RW;
    const uint32_t w = Q[i];
    const uint32_t prev = m ? (Q[i - 1] >> 31) : 0u;
    const uint32_t st = w & ~((w << 1) | prev);
    St[i] = st;
    nst += __popc(st);
    pre[i] = nst; // inclusive, within the chunk (made global below)
    if (m == 0 && (w & 1u) && ((Q[r * RW + ((L0 - 1) >> 5)] >> ((L0 - 1) & 31)) & 1u)) ++ned;
#pragma unroll
    for (int t = 0; t < D - 1; ++t) {
      const uint32_t o = w & Q[nrow[t * R + r] * RW + m];
      ned += __popc(o & ~(o << 1));
    }
  }
  int nruns, nedges;
  const int run0 = cta_exclusive_scan(nst, misc, &nruns);
  const int ed0 = cta_exclusive_scan(ned, misc, &nedges);
  for (int i = i0; i < i1; ++i) pre[i] = run0 + pre[i] - __popc(St[i]); // runs before word i
  for (int i = tid; i < nruns; i += HLAB_NT) par[i] = (uint16_t)i;
  if (MULTI)
    for (int i = tid; i < g.N / 64 + 1; i += HLAB_NT) coin[i] = 0u;
  __syncthreads();
  const bool stored = nedges <= ecap; // the same on every thread
  if (stored) {
    int e = ed0;
    for (int i = i0; i < i1; ++i) {
      const int r = i / RW, m = i - r * RW;
      const uint32_t w = Q[i];
      if (m == 0 && (w & 1u) && ((Q[r * RW + ((L0 - 1) >> 5)] >> ((L0 - 1) & 31)) & 1u))
        edges[e++] = make_ushort2((unsigned short)run_of<RW>(St, pre, r, 0),
                                  (unsigned short)run_of<RW>(St, pre, r, L0 - 1));
#pragma unroll
      for (int t = 0; t < D - 1; ++t) {
        const int r2 = nrow[t * R + r];
        const uint32_t o = w & Q[r2 * RW + m];
        for (uint32_t sg = o & ~(o << 1); sg; sg &= sg - 1u) {
          const int x = 32 * m + __ffs(sg) - 1;
          edges[e++] = make_ushort2((unsigned short)run_of<RW>(St, pre, r, x),
                                    (unsigned short)run_of<RW>(St, pre, r2, x));
        }
      }
    }
  }
  __syncthreads();

  // components: rounds of hooking and pointer jumping.  At the start of a round every
  // run points at the root of its star; each edge whose ends have different roots hooks
  // the larger root under the smaller (a compare-and-swap minimum, so parents only
  // decrease and a root stays the smallest run of its tree); then every run jumps to
  // its root.  A round without a hook ends the labelling.  Each round merges at least
  // two trees, so at most nruns rounds are needed (a handful in practice).
  volatile uint16_t *vpar = par;
  auto hook = [&](int a_run, int b_run, int &hooked) {
    const int pa = vpar[a_run], pb = vpar[b_run];
    if (pa != pb) {
      const int hi = pa > pb ? pa : pb, lo = pa + pb - hi;
      int cur = vpar[hi];
      while (lo < cur) {
        const int old = atomicCAS(const_cast<unsigned short *>(par) + hi, (unsigned short)cur, (unsigned short)lo);
        if (old == cur) break;
        cur = old;
      }
      hooked = 1;
    }
  };
  for (int round = 0; round <= nruns; ++round) {
    int hooked = 0;
    if (stored) {
      for (int e = tid; e < nedges; e += HLAB_NT) {
        const ushort2 ab = edges[e];
        hook(ab.x, ab.y, hooked);
      }
    } else {
      for (int i = i0; i < i1; ++i) {
        const int r = i / RW, m = i - r * RW;
        const uint32_t w = Q[i];
        if (m == 0 && (w & 1u) && ((Q[r * RW + ((L0 - 1) >> 5)] >> ((L0 - 1) & 31)) & 1u))
          hook(run_of<RW>(St, pre, r, 0), run_of<RW>(St, pre, r, L0 - 1), hooked);
#pragma unroll
        for (int t = 0; t < D - 1; ++t) {
          const int r2 = nrow[t * R + r];
          const uint32_t o = w & Q[r2 * RW + m];
          for (uint32_t sg = o & ~(o << 1); sg; sg &= sg - 1u) {
            const int x = 32 * m + __ffs(sg) - 1;
            hook(run_of<RW>(St, pre, r, x), run_of<RW>(St, pre, r2, x), hooked);
          }
        }
      }
    }
    if (!__syncthreads_or(hooked)) break;
    // pointer jumping by doubling (every run to its grandparent, until nothing moves):
    // log(depth) uniform passes, where walking each run's whole path would cost the
    // square of a long chain's length
    for (int it = 0; it <= 16; ++it) {
      int moved = 0;
      for (int x = tid; x < nruns; x += HLAB_NT) {
        const int p = vpar[x], pp = vpar[p];
        if (pp != p) {
          vpar[x] = (uint16_t)pp;
          moved = 1;
        }
      }
      if (!__syncthreads_or(moved)) break;
    }
  }

  if (MULTI) {
    // a coin for every root run: locate its start (the last word whose run count before
    // it does not exceed the run's number, then the start bit within the word)
    const uint32_t t_houd = (uint32_t)dv.ctr[CTR_THOUD];
    const uint32_t c3 = ((uint32_t)dv.slot[((size_t)s * jb.C + 0) * jb.T + a] << 8) | TAG_HMULTI;
    const uint32_t s_glob = (uint32_t)(jb.s_off + s);
    for (int i = tid; i < nruns; i += HLAB_NT) {
      if ((int)par[i] != i) continue;
      int lo = 0, hi = NBW - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= i) lo = mid;
        else hi = mid - 1;
      }
      const int r = lo / RW, x = 32 * (lo - r * RW) + nth_set_bit(St[lo], i - pre[lo]);
      const uint32_t site = (uint32_t)(r * L0 + x);
      if (philox10(site, t_houd, s_glob, c3, jb.sk0, jb.sk1).x >> 31) atomicOr(&coin[i >> 5], 1u << (i & 31));
    }
  }
  // the seed: the floor(u M / 2^32)-th q = -1 site in canonical order (warp 0)
  if (!MULTI && warp == 0) {
    const uint32_t t_houd = (uint32_t)dv.ctr[CTR_THOUD];
    const int k = dv.slot[((size_t)s * jb.C + 0) * jb.T + a];
    const uint32_t uu = philox10((uint32_t)k, t_houd, (uint32_t)(jb.s_off + s), TAG_HOUD, jb.sk0, jb.sk1).x;
    const uint32_t n = (uint32_t)(((unsigned long long)uu * M) >> 32);
    const int ch = (NBW + 31) / 32;
    const int b0 = min(NBW, lane * ch), b1 = min(NBW, b0 + ch);
    uint32_t c = 0u;
    for (int b = b0; b < b1; ++b) c += __popc(Q[b]);
    uint32_t pre_c = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(FULLM, pre_c, o);
      if (lane >= o) pre_c += v;
    }
    pre_c -= c;
    if (n >= pre_c && n < pre_c + c) {
      uint32_t rem = n - pre_c;
      for (int b = b0; b < b1; ++b) {
        const uint32_t w = Q[b];
        const uint32_t pc = __popc(w);
        if (rem < pc) {
          const int r = b / RW, x = 32 * (b - r * RW) + nth_set_bit(w, (int)rem);
          misc[16] = (int)par[run_of<RW>(St, pre, r, x)];
          break;
        }
        rem -= pc;
      }
    }
  }
  __syncthreads();

  // the seed's cluster: the runs whose root is the seed's root (MULTI: whose root's coin
  // is 1)
  const int root0 = MULTI ? -1 : misc[16];
  uint32_t size = 0u;
  for (int i = tid; i < NBW; i += HLAB_NT) {
    const uint32_t w = Q[i];
    uint32_t seg = w & ~(w << 1), c = 0u;
    if (seg) {
      const int r = i / RW, x0 = 32 * (i - r * RW);
      // the run of the word's first segment; every later segment starts the next run
      int id = run_of<RW>(St, pre, r, x0 + __ffs(seg) - 1) - 1;
      while (seg) {
        const int b = __ffs(seg) - 1;
        seg &= seg - 1u;
        ++id;
        const int rt = (int)par[id];
        const bool take = MULTI ? ((coin[rt >> 5] >> (rt & 31)) & 1u) != 0u : rt == root0;
        if (take) c |= ((w + (1u << b)) ^ w) & w;
      }
    }
    Cp[i] = c;
    size += __popc(c);
  }
  size = __reduce_add_sync(FULLM, size);
  if (lane == 0 && size) atomicAdd(&misc[17], (int)size);
  __syncthreads();
  if (tid == 0) {
    atomicAdd(&dv.ctr[CTR_HMOVES], 1ull);
    atomicAdd(&dv.ctr[CTR_HSITES], (unsigned long long)misc[17]);
  }
}

int houdayer_smem(const Job &jb, int bitmaps_smem) {
  const int RW = (jb.g.L0 + 31) / 32;
  int oq, ow;
  return houd_smem_bytes(jb.T, jb.g.R, jb.g.R * RW, bitmaps_smem, &oq, &ow);
}

size_t houdayer_scratch_bytes(const Job &jb) {
  const int RW = (jb.g.L0 + 31) / 32;
  // q and cluster bitmaps of every pair, then M per (sample, lane), then the pair queue
  return (size_t)jb.S * 2 * jb.T * (size_t)(jb.g.R * RW) * 4 + (size_t)jb.S * 32 * 4 + 16;
}

namespace {
typedef void (*houd_fn)(Job, Dev, HoudArgs);
typedef void (*fill_fn)(Job, Dev, HoudSplit);
template <int D>
houd_fn pick_houd(int RW) {
  switch (RW) {
  case 1: return k_houdayer<D, 1>;
  case 2: return k_houdayer<D, 2>;
  case 3: return k_houdayer<D, 3>;
  case 4: return k_houdayer<D, 4>;
  case 5: return k_houdayer<D, 5>;
  case 6: return k_houdayer<D, 6>;
  case 7: return k_houdayer<D, 7>;
  default: return k_houdayer<D, 8>;
  }
}
template <int D, bool SMEM>
fill_fn pick_fill_rw(int RW) {
  switch (RW) {
  case 1: return k_houd_fill<D, 1, SMEM>;
  case 2: return k_houd_fill<D, 2, SMEM>;
  case 3: return k_houd_fill<D, 3, SMEM>;
  case 4: return k_houd_fill<D, 4, SMEM>;
  case 5: return k_houd_fill<D, 5, SMEM>;
  case 6: return k_houd_fill<D, 6, SMEM>;
  case 7: return k_houd_fill<D, 7, SMEM>;
  default: return k_houd_fill<D, 8, SMEM>;
  }
}
template <int D, bool MULTI>
fill_fn pick_label_rw(int RW) {
  switch (RW) {
  case 1: return k_houd_label<D, 1, MULTI>;
  case 2: return k_houd_label<D, 2, MULTI>;
  case 3: return k_houd_label<D, 3, MULTI>;
  case 4: return k_houd_label<D, 4, MULTI>;
  case 5: return k_houd_label<D, 5, MULTI>;
  case 6: return k_houd_label<D, 6, MULTI>;
  case 7: return k_houd_label<D, 7, MULTI>;
  default: return k_houd_label<D, 8, MULTI>;
  }
}
fill_fn pick_label(int d, int RW, bool multi) {
  if (d == 2) return multi ? pick_label_rw<2, true>(RW) : pick_label_rw<2, false>(RW);
  return multi ? pick_label_rw<3, true>(RW) : pick_label_rw<3, false>(RW);
}

fill_fn pick_fill(int d, int RW, bool in_smem) {
  if (d == 2) return in_smem ? pick_fill_rw<2, true>(RW) : pick_fill_rw<2, false>(RW);
  return in_smem ? pick_fill_rw<3, true>(RW) : pick_fill_rw<3, false>(RW);
}

// Fill-kernel shape: up to 8 pairs per CTA, fewer when their bitmaps would take more than
// 64 KB of shared memory; bitmaps stay in global scratch when even one pair's exceed the
// Houdayer shared-memory budget.
void fill_shape(const Job &jb, int NBW, int *wpb, int *in_smem, int *smem) {
  const int wl = houd_worklist_bytes(jb.g.R);
  const int per = 2 * NBW * 4 + wl;
  int w = HFILL_MAX_WARPS;
  while (w > 1 && w * per > 64 * 1024) w >>= 1;
  if (w * per <= HOUD_SMEM_BUDGET) {
    *wpb = w;
    *in_smem = 1;
    *smem = HFILL_HEAD + w * per;
  } else {
    *wpb = HFILL_MAX_WARPS;
    *in_smem = 0;
    *smem = HFILL_HEAD + HFILL_MAX_WARPS * wl;
  }
}
} // namespace

cudaError_t prepare_houdayer_kernels(int max_smem) {
  for (int rw = 1; rw <= 8; ++rw) {
    for (int d = 2; d <= 3; ++d) {
      const void *fns[5] = {(const void *)(d == 2 ? pick_houd<2>(rw) : pick_houd<3>(rw)),
                            (const void *)pick_fill(d, rw, true), (const void *)pick_fill(d, rw, false),
                            (const void *)pick_label(d, rw, false), (const void *)pick_label(d, rw, true)};
      for (const void *fn : fns) {
        const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
      }
    }
  }
  return prepare_houd_seed_kernels(max_smem);
}

bool houdayer_labels(const Job &jb) {
  const int RW = (jb.g.L0 + 31) / 32;
  return jb.g.N / 2 <= 65536 && label_smem_bytes(jb.g.R * RW, jb.g.N, jb.g.R, jb.g.d) <= HOUD_SMEM_BUDGET;
}

// With `scratch` (houdayer_scratch_bytes of the handle's buffer) the split form runs;
// without it the single-CTA form, whose bitmaps must then fit `smem_limit`.
HoudMaps houd_maps_of(const Job &jb, uint32_t *scratch) {
  HoudMaps hm;
  hm.RW = (jb.g.L0 + 31) / 32;
  hm.NBW = jb.g.R * hm.RW;
  hm.Qg = scratch;
  hm.Cg = scratch + (size_t)jb.S * jb.T * hm.NBW;
  hm.Mg = hm.Cg + (size_t)jb.S * jb.T * hm.NBW;
  return hm;
}

cudaError_t launch_houdayer(const Job &jb, const Dev &dv, uint32_t *scratch, int smem_limit, bool multi,
                            cudaStream_t st, bool fused) {
  const int RW = (jb.g.L0 + 31) / 32;
  const int NBW = jb.g.R * RW;
  if (scratch) {
    const HoudMaps hm = houd_maps_of(jb, scratch);
    HoudSplit hs;
    hs.RW = hm.RW;
    hs.NBW = hm.NBW;
    hs.Qg = hm.Qg;
    hs.Cg = hm.Cg;
    hs.Mg = hm.Mg;
    hs.queue = hs.Mg + (size_t)jb.S * 32;
    int smem = 0;
    fill_shape(jb, NBW, &hs.wpb, &hs.in_smem, &smem);
    const long long pairs = (long long)jb.S * jb.T;
    // per-sample kernels: about four CTAs per SM (parts of a sample's blocks)
    int dev = 0, n_sm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    int parts = (4 * n_sm + jb.S - 1) / jb.S;
    const int tiles = (NBW + HQ_TB - 1) / HQ_TB;
    parts = parts < 1 ? 1 : (parts > 8 ? 8 : parts);
    parts = parts > tiles ? tiles : parts;
    const dim3 pgrid((unsigned)jb.S, (unsigned)parts);
    if (fused) {
      // M was written whole by the sweep launch: only the pair queue is cleared
      const cudaError_t e0 = cudaMemsetAsync(hs.queue, 0, 16, st);
      if (e0 != cudaSuccess) return e0;
    } else {
      const cudaError_t e0 = cudaMemsetAsync(hs.Mg, 0, (size_t)jb.S * 32 * 4 + 16, st); // M and the pair queue
      if (e0 != cudaSuccess) return e0;
      k_houd_q<<<pgrid, HSPLIT_NT, 0, st>>>(jb, dv, hs);
    }
    const int lab = label_smem_bytes(NBW, jb.g.N, jb.g.R, jb.g.d);
    // the single-cluster move grows only the seed's cluster where a fill form applies
    bool seeded = false;
    if (!multi) {
      const cudaError_t es = launch_houd_seed(jb, dv, hs, n_sm, st, &seeded);
      if (es != cudaSuccess) return es;
    }
    if (seeded) {
    } else if (houdayer_labels(jb)) {
      pick_label(jb.g.d, RW, multi)<<<(unsigned)pairs, HLAB_NT, (size_t)lab, st>>>(jb, dv, hs);
    } else {
      if (multi) return cudaErrorNotSupported;
      // labels beyond the shared-memory budget: grow the seed's cluster row by row
      pick_fill(jb.g.d, RW, hs.in_smem != 0)<<<(unsigned)((pairs + hs.wpb - 1) / hs.wpb), 32 * hs.wpb,
                                                (size_t)smem, st>>>(jb, dv, hs);
    }
    if (!fused) k_houd_flip<<<pgrid, HSPLIT_NT, 0, st>>>(jb, dv, hs);
    return cudaGetLastError();
  }
  if (fused) return cudaErrorInvalidValue; // the fused phases need the split form's scratch
  if (multi) return cudaErrorNotSupported; // the multi-cluster variant labels in the split form only
  HoudArgs ha;
  ha.RW = RW;
  ha.NBW = NBW;
  const int smem = houdayer_smem(jb, 1);
  if (smem > smem_limit) return cudaErrorInvalidValue;
  const houd_fn fn = jb.g.d == 2 ? pick_houd<2>(RW) : pick_houd<3>(RW);
  fn<<<(unsigned)jb.S, HNT, (size_t)smem, st>>>(jb, dv, ha);
  return cudaGetLastError();
}

} // namespace sgmc
