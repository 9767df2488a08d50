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
#include "sgmc_internal.cuh"

namespace sgmc {

namespace {

constexpr uint32_t FULLM = 0xFFFFFFFFu;
constexpr int HNT = 1024; // threads per CTA (32 warps)

// In-warp 32x32 bit transpose: afterwards lane l holds bit i = (input of lane i, bit l).
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int j = 16 >> st;
    const uint32_t m = masks[st];
    const uint32_t y = __shfl_xor_sync(FULLM, x, j);
    if (lane & j) x = (x & ~m) | ((y & ~m) >> j);
    else x = (x & m) | ((y & m) << j);
  }
  return x;
}

// Byte-table permutation of a word: out = OR over bytes of tab[byte index][byte value].
__device__ __forceinline__ uint32_t permute_word(const uint32_t *tab, uint32_t w) {
  return tab[w & 255u] | tab[256 + ((w >> 8) & 255u)] | tab[512 + ((w >> 16) & 255u)] | tab[768 + (w >> 24)];
}

// Runs of an L0-bit row (RW words, bits >= L0 zero).
// fill_up: for every run of Q holding a bit of X (X subset of Q), the bits from its lowest
// X bit to the run's top (the carry of Q + X runs through the run and stops above it).
template <int RW>
__device__ __forceinline__ void fill_up(const uint32_t (&Q)[RW], const uint32_t (&X)[RW], uint32_t (&F)[RW]) {
  unsigned long long c = 0;
#pragma unroll
  for (int m = 0; m < RW; ++m) {
    const unsigned long long sum = (unsigned long long)Q[m] + X[m] + c;
    c = sum >> 32;
    F[m] = (((uint32_t)sum ^ Q[m]) & Q[m]) | X[m];
  }
}

// Reverse the L0-bit string held in RW words (bit x -> bit L0-1-x).
template <int RW>
__device__ __forceinline__ void reverse_row(const uint32_t (&A)[RW], uint32_t (&B)[RW], int L0) {
  uint32_t t[RW];
#pragma unroll
  for (int m = 0; m < RW; ++m) t[m] = __brev(A[RW - 1 - m]);
  const int sh = 32 * RW - L0; // 0..31
  if (sh == 0) {
#pragma unroll
    for (int m = 0; m < RW; ++m) B[m] = t[m];
  } else {
#pragma unroll
    for (int m = 0; m < RW; ++m) {
      const uint32_t hi = m + 1 < RW ? t[m + 1] : 0u;
      B[m] = (t[m] >> sh) | (hi << (32 - sh));
    }
  }
}

template <int RW>
__device__ __forceinline__ void fill_down(const uint32_t (&Q)[RW], const uint32_t (&X)[RW], uint32_t (&F)[RW],
                                          int L0) {
  uint32_t rq[RW], rx[RW], rf[RW];
  reverse_row<RW>(Q, rq, L0);
  reverse_row<RW>(X, rx, L0);
  fill_up<RW>(rq, rx, rf);
  reverse_row<RW>(rf, F, L0);
}

// F = the union of the runs of the periodic L0-bit row Q that contain a bit of X.
template <int RW>
__device__ __forceinline__ void close_row(const uint32_t (&Q)[RW], const uint32_t (&X)[RW], uint32_t (&F)[RW],
                                          int L0) {
  uint32_t a[RW], b[RW];
  fill_up<RW>(Q, X, a);
  fill_down<RW>(Q, X, b, L0);
#pragma unroll
  for (int m = 0; m < RW; ++m) F[m] = a[m] | b[m];
  // periodic wrap: a run through x = L0-1 continues at x = 0 and vice versa
  const int tw = (L0 - 1) >> 5, tb = (L0 - 1) & 31;
  uint32_t ftop = 0u, qtopw = 0u;
#pragma unroll
  for (int m = 0; m < RW; ++m)
    if (m == tw) {
      ftop = F[m];
      qtopw = Q[m];
    }
  const bool top_in = (ftop >> tb) & 1u, bot_in = F[0] & 1u;
  const bool qtop = (qtopw >> tb) & 1u, qbot = Q[0] & 1u;
  if (top_in && qbot && !bot_in) {
    uint32_t s[RW], g[RW];
#pragma unroll
    for (int m = 0; m < RW; ++m) s[m] = m == 0 ? 1u : 0u;
    fill_up<RW>(Q, s, g);
#pragma unroll
    for (int m = 0; m < RW; ++m) F[m] |= g[m];
  }
  uint32_t ftop2 = 0u;
#pragma unroll
  for (int m = 0; m < RW; ++m)
    if (m == tw) ftop2 = F[m];
  if (bot_in && qtop && !((ftop2 >> tb) & 1u)) {
    uint32_t s[RW], g[RW];
#pragma unroll
    for (int m = 0; m < RW; ++m) s[m] = m == tw ? (1u << tb) : 0u;
    fill_down<RW>(Q, s, g, L0);
#pragma unroll
    for (int m = 0; m < RW; ++m) F[m] |= g[m];
  }
}

} // namespace

struct HoudArgs {
  int RW;           // words per bitmap row
  int NBW;          // words per bitmap (rows x RW)
  int bitmaps_smem; // 1: q and cluster bitmaps in shared memory, 0: in `scratch`
  uint32_t *scratch; // [S][2][T][NBW] when not in shared memory
};

// Shared-memory map of the Houdayer kernel.
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

template <int D, int RW>
__global__ void __launch_bounds__(HNT) k_houdayer(Job jb, Dev dv, HoudArgs ha) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Geo g = jb.g;
  const int T = jb.T, N = g.N, L0 = g.L0, L1 = g.L1, R = g.R;
  const int NBW = ha.NBW;
  int off_q, off_wl;
  houd_smem_bytes(T, R, NBW, ha.bitmaps_smem, &off_q, &off_wl);
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
  uint32_t *Qb, *Cb;
  if (ha.bitmaps_smem) {
    Qb = reinterpret_cast<uint32_t *>(smem + off_q);
  } else {
    Qb = ha.scratch + (size_t)s * 2 * T * NBW;
  }
  Cb = Qb + (size_t)T * NBW;
  unsigned char *wlbase = smem + off_wl;
  const int wl_bytes = ((2 * R + 3) & ~3) + 4 * ((R + 31) / 32) + 4;
  uint16_t *stack = reinterpret_cast<uint16_t *>(wlbase + warp * wl_bytes);
  uint32_t *inlist = reinterpret_cast<uint32_t *>(wlbase + warp * wl_bytes + ((2 * R + 3) & ~3));
  int *ssize = reinterpret_cast<int *>(inlist + (R + 31) / 32);

  const uint32_t *w0p = dv.spins + ((size_t)s * jb.W + 0) * N; // chain 0 word (Wc = 1)
  const uint32_t *w1p = dv.spins + ((size_t)s * jb.W + 1) * N; // chain 1 word
  uint32_t *w0w = const_cast<uint32_t *>(w0p), *w1w = const_cast<uint32_t *>(w1p);

  // ---- phase 0: maps and lane-permutation tables --------------------------------
  if (tid < 32) {
    const size_t c0 = ((size_t)s * jb.C + 0) * T, c1 = ((size_t)s * jb.C + 1) * T;
    perm0[tid] = tid < T ? dv.perm[c0 + tid] : 0;
    perm1[tid] = tid < T ? dv.perm[c1 + tid] : 0;
    slot0[tid] = tid < T ? dv.slot[c0 + tid] : 0;
    slot1[tid] = tid < T ? dv.slot[c1 + tid] : 0;
    Mc[tid] = 0u;
    if (tid < 2) cnts[tid] = 0ull;
  }
  __syncthreads();
  {
    // entry e = (byte j, value v): sig maps chain-1 lane b -> chain-0 lane a = perm0[slot1[b]],
    // sigi maps chain-0 lane a -> chain-1 lane b = perm1[slot0[a]]
    const int j = tid >> 8, v = tid & 255;
    uint32_t o1 = 0u, o2 = 0u;
#pragma unroll
    for (int bb = 0; bb < 8; ++bb) {
      const int lanei = 8 * j + bb;
      if (((v >> bb) & 1) && lanei < T) {
        o1 |= 1u << perm0[slot1[lanei]];
        o2 |= 1u << perm1[slot0[lanei]];
      }
    }
    sig[tid] = o1;
    sigi[tid] = o2;
  }
  __syncthreads();

  const uint32_t tmask = T >= 32 ? FULLM : ((1u << T) - 1u);
  // canonical site of bitmap block b, lane l: row r = b / RW, x = 32 (b % RW) + l
  auto site_word = [&](int b, int l, int &p, bool &valid) {
    const int r = b / RW, x = 32 * (b - r * RW) + l;
    valid = x < L0;
    const int y = r % L1, z = r / L1;
    const int c = (x + y + z) & 1;
    p = c * g.Nh + r * g.H + (x >> 1);
  };

  // ---- phase 1: q bitmaps and M ----------------------------------------------------
  {
    uint32_t mpart = 0u;
    for (int b = warp; b < NBW; b += HNT / 32) {
      int p;
      bool valid;
      site_word(b, lane, p, valid);
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
  __syncthreads();

  // ---- phase 2: one cluster per pair -------------------------------------------------
  for (int a = warp; a < T; a += HNT / 32) {
    uint32_t *Q = Qb + (size_t)a * NBW;
    uint32_t *C = Cb + (size_t)a * NBW;
    for (int b = lane; b < NBW; b += 32) C[b] = 0u;
    const uint32_t M = Mc[a];
    if (M == 0u) continue;
    const int k = slot0[a];
    const uint32_t u = philox10((uint32_t)k, t_houd, s_glob, TAG_HOUD, jb.sk0, jb.sk1).x;
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
    // worklist reset
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
    const int max_rounds = 4 * N + 64; // never reached: every push adds at least one site
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
    if (lane == 0 && *ssize > 0) atomicOr(&dv.ctr[CTR_ERROR], ERR_HOUD_ROUNDS);
    uint32_t sz = 0u;
    for (int b = lane; b < NBW; b += 32) sz += __popc(C[b]);
    sz = __reduce_add_sync(FULLM, sz);
    if (lane == 0) {
      atomicAdd(&cnts[0], 1ull);
      atomicAdd(&cnts[1], (unsigned long long)sz);
    }
  }
  __syncthreads();

  // ---- phase 3: flip both replicas of every pair on its cluster ------------------------
  for (int b = warp; b < NBW; b += HNT / 32) {
    const uint32_t cw = lane < T ? Cb[(size_t)lane * NBW + b] : 0u;
    if (!__any_sync(FULLM, cw != 0u)) continue;
    const uint32_t f0 = transpose32(cw, lane); // lane l: bit a = site l in pair a's cluster
    int p;
    bool valid;
    site_word(b, lane, p, valid);
    if (valid && f0) {
      w0w[p] ^= f0;
      w1w[p] ^= permute_word(sigi, f0);
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (cnts[0]) atomicAdd(&dv.ctr[CTR_HMOVES], cnts[0]);
    if (cnts[1]) atomicAdd(&dv.ctr[CTR_HSITES], cnts[1]);
  }
  grid_done_advance(dv.ctr, 0ull, 0ull, 1ull);
}

int houdayer_smem(const Job &jb, int bitmaps_smem) {
  const int RW = (jb.g.L0 + 31) / 32;
  int oq, ow;
  return houd_smem_bytes(jb.T, jb.g.R, jb.g.R * RW, bitmaps_smem, &oq, &ow);
}

size_t houdayer_scratch_bytes(const Job &jb) {
  const int RW = (jb.g.L0 + 31) / 32;
  return (size_t)jb.S * 2 * jb.T * (size_t)(jb.g.R * RW) * 4;
}

namespace {
typedef void (*houd_fn)(Job, Dev, HoudArgs);
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
} // namespace

cudaError_t prepare_houdayer_kernels(int max_smem) {
  for (int rw = 1; rw <= 8; ++rw) {
    for (int d = 2; d <= 3; ++d) {
      const houd_fn fn = d == 2 ? pick_houd<2>(rw) : pick_houd<3>(rw);
      const cudaError_t e =
          cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_houdayer(const Job &jb, const Dev &dv, uint32_t *scratch, int smem_limit, cudaStream_t st) {
  HoudArgs ha;
  ha.RW = (jb.g.L0 + 31) / 32;
  ha.NBW = jb.g.R * ha.RW;
  const int in_smem = houdayer_smem(jb, 1);
  ha.bitmaps_smem = in_smem <= smem_limit ? 1 : 0;
  ha.scratch = scratch;
  if (!ha.bitmaps_smem && !scratch) return cudaErrorInvalidValue;
  const int smem = houdayer_smem(jb, ha.bitmaps_smem);
  const houd_fn fn = jb.g.d == 2 ? pick_houd<2>(ha.RW) : pick_houd<3>(ha.RW);
  fn<<<(unsigned)jb.S, HNT, (size_t)smem, st>>>(jb, dv, ha);
  return cudaGetLastError();
}

} // namespace sgmc
