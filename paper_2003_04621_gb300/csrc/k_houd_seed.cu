// k_houd_seed.cu -- phase 2 of the single-cluster Houdayer move (Sec. 2.4, Eq. 10) by
// growing only the seed's cluster.
//
// The move exchanges the two replicas of a pair on ONE q = -1 cluster, the one holding the
// seed (the floor(u M / 2^32)-th q = -1 site in canonical order, u the pair's Philox word).
// So only that cluster is needed, and it is grown by passes of a monotone fill over the
// pair's bitmap rows: a row's part of the cluster is always a union of whole runs of the
// q bitmap (close_row), so a pass visits each row, takes the q = -1 sites of the row that
// touch the cluster in a neighbouring row (y +- 1, and z +- 1 in 3D) and are not in it
// yet, and closes them along x.  One warp grows one pair; lane l owns the block of RPL
// consecutive rows l RPL .. l RPL + RPL - 1 and visits them downwards and then upwards in
// each pass, so the cluster crosses a whole block in one pass.  A lane may see a
// neighbouring lane's row before or after that lane's update in the same pass; as the
// cluster only grows and never leaves the seed's component, every such order reaches the
// same set, and a pass in which no lane adds a site proves the set complete (each row was
// then checked against the final values of its neighbours).
//
// Warps take pairs from a device queue (an atomic counter zeroed before the move), so a
// warp that finishes a small cluster goes on to the next pair instead of waiting for the
// largest cluster of a fixed group.
//
// Two forms: the register form keeps a lane's block of q and cluster rows in registers
// and fetches the neighbouring lanes' rows by warp shuffles (lattices whose rows per lane
// RPL divide the rows per plane L1, rows of at most 4 words and RW RPL <= 16 words per
// lane); the shared-memory form keeps both bitmaps in shared memory (3D lattices outside
// that).  Other 2D lattices are labelled instead (k_houdayer.cu).
#include "sgmc_houd.cuh"

namespace sgmc {

namespace {

constexpr int HSEED_NT = 256; // 8 warps (pairs in flight) per CTA

// Rows per lane: the smallest power of two with 32 RPL >= R.
__host__ __device__ inline int seed_rpl(int R) {
  int rpl = 1;
  while (32 * rpl < R) rpl <<= 1;
  return rpl;
}

// The next pair of the queue for this warp (lane 0 takes it), or -1 when none is left.
__device__ __forceinline__ long long next_pair(unsigned int *queue, long long pairs) {
  long long gp = 0;
  if ((threadIdx.x & 31) == 0) gp = (long long)atomicAdd(queue, 1u);
  gp = __shfl_sync(FULLM, gp, 0);
  return gp < pairs ? gp : -1;
}

// The pair's Philox seed index n = floor(u M / 2^32) (Sec. 2.4, reading H1).
__device__ __forceinline__ uint32_t seed_index(const Job &jb, const Dev &dv, int s, int a, uint32_t M,
                                               uint32_t t_houd) {
  const int k = dv.slot[((size_t)s * jb.C + 0) * jb.T + a];
  const uint32_t u = philox10((uint32_t)k, t_houd, (uint32_t)(jb.s_off + s), TAG_HOUD, jb.sk0, jb.sk1).x;
  return (uint32_t)(((unsigned long long)u * M) >> 32);
}

// ---------------------------------------------------------------------------------
// Register form.  Planes (rows of equal z) consist of whole blocks (L1 % RPL == 0), so the
// neighbours of a lane's row i are: along y, rows i -+ 1 of the same lane, or for the
// block's first and last row the last / first row of the lanes before / after it in the
// plane (periodic); along z, row i of the lanes bpp = L1 / RPL before / after it
// (periodic in z).  Every such fetch reads the same register index from another lane,
// which a warp shuffle does.
// ---------------------------------------------------------------------------------
template <int D, int RW, int RPL>
__global__ void __launch_bounds__(HSEED_NT) k_houd_seedreg(Job jb, Dev dv, HoudSplit hs) {
  const int lane = threadIdx.x & 31;
  const Geo g = jb.g;
  const int NBW = hs.NBW;
  const long long pairs = (long long)jb.S * jb.T;
  const int bpp = g.L1 / RPL;       // blocks per plane
  const bool owns = lane * RPL < g.R; // lanes past the last row hold empty rows
  const int b = lane % bpp, zb = lane / bpp;
  int src_yp = b == bpp - 1 ? lane - (bpp - 1) : lane + 1;
  int src_ym = b == 0 ? lane + (bpp - 1) : lane - 1;
  int src_zp = zb == g.L2 - 1 ? lane - (g.L2 - 1) * bpp : lane + bpp;
  int src_zm = zb == 0 ? lane + (g.L2 - 1) * bpp : lane - bpp;
  if (!owns) src_yp = src_ym = src_zp = src_zm = lane;
  const uint32_t t_houd = (uint32_t)dv.ctr[CTR_THOUD];
  unsigned long long n_moves = 0ull, n_sites = 0ull;
  for (long long gp = next_pair(hs.queue, pairs); gp >= 0; gp = next_pair(hs.queue, pairs)) {
    const int s = (int)(gp / jb.T), a = (int)(gp - (long long)s * jb.T);
    const uint32_t M = hs.Mg[(size_t)s * 32 + a];
    if (M == 0u) continue; // no q = -1 site: no move (the flip kernel skips the pair)
    const uint32_t *Qp = hs.Qg + ((size_t)s * jb.T + a) * NBW;
    uint32_t *Cp = hs.Cg + ((size_t)s * jb.T + a) * NBW;
    uint32_t q[RPL][RW], c[RPL][RW];
    uint32_t cnt = 0u;
#pragma unroll
    for (int i = 0; i < RPL; ++i)
#pragma unroll
      for (int m = 0; m < RW; ++m) {
        q[i][m] = owns ? Qp[(lane * RPL + i) * RW + m] : 0u;
        c[i][m] = 0u;
        cnt += __popc(q[i][m]);
      }
    // the seed: lane blocks are consecutive rows, so canonical order is lane order
    const uint32_t n = seed_index(jb, dv, s, a, M, t_houd);
    uint32_t pre = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(FULLM, pre, o);
      if (lane >= o) pre += v;
    }
    pre -= cnt;
    int srow = -1, sword = 0;
    uint32_t sbit = 0u;
    if (n >= pre && n < pre + cnt) {
      uint32_t rem = n - pre;
#pragma unroll
      for (int i = 0; i < RPL; ++i)
#pragma unroll
        for (int m = 0; m < RW; ++m) {
          const uint32_t pc = __popc(q[i][m]);
          if (srow < 0) {
            if (rem < pc) {
              uint32_t w = q[i][m];
              for (uint32_t j = 0; j < rem; ++j) w &= w - 1u;
              srow = i;
              sword = m;
              sbit = w & (0u - w);
            } else {
              rem -= pc;
            }
          }
        }
    }
#pragma unroll
    for (int i = 0; i < RPL; ++i)
      if (i == srow) {
        uint32_t x[RW], f[RW];
#pragma unroll
        for (int m = 0; m < RW; ++m) x[m] = m == sword ? sbit : 0u;
        close_row<RW>(q[i], x, f, g.L0);
#pragma unroll
        for (int m = 0; m < RW; ++m) c[i][m] = f[m];
      }
    const int max_passes = g.N + 2; // every pass that changes adds a site
    int pass = 0;
    for (; pass < max_passes; ++pass) {
      bool changed = false;
#pragma unroll
      for (int v = 0; v < 2 * RPL; ++v) {
        const int i = v < RPL ? v : 2 * RPL - 1 - v;
        uint32_t x[RW];
        bool any = false;
#pragma unroll
        for (int m = 0; m < RW; ++m) {
          const uint32_t up = i > 0 ? c[i > 0 ? i - 1 : 0][m] : __shfl_sync(FULLM, c[RPL - 1][m], src_ym);
          const uint32_t dn = i < RPL - 1 ? c[i < RPL - 1 ? i + 1 : 0][m] : __shfl_sync(FULLM, c[0][m], src_yp);
          uint32_t nb = up | dn;
          if (D == 3) nb |= __shfl_sync(FULLM, c[i][m], src_zp) | __shfl_sync(FULLM, c[i][m], src_zm);
          x[m] = q[i][m] & ~c[i][m] & nb;
          any |= x[m] != 0u;
        }
        if (any) {
          uint32_t f[RW];
          close_row<RW>(q[i], x, f, g.L0);
#pragma unroll
          for (int m = 0; m < RW; ++m) c[i][m] |= f[m];
          changed = true;
        }
      }
      if (!__any_sync(FULLM, changed)) break;
    }
    if (pass == max_passes && lane == 0) atomicOr(&dv.ctr[CTR_ERROR], ERR_HOUD_ROUNDS);
    uint32_t size = 0u;
    if (owns) {
#pragma unroll
      for (int i = 0; i < RPL; ++i)
#pragma unroll
        for (int m = 0; m < RW; ++m) {
          Cp[(lane * RPL + i) * RW + m] = c[i][m];
          size += __popc(c[i][m]);
        }
    }
    size = __reduce_add_sync(FULLM, size);
    n_moves += 1ull;
    n_sites += size;
  }
  // each warp reports on its own once the queue is empty (no wait for the CTA's others)
  if (lane == 0 && n_moves) {
    atomicAdd(&dv.ctr[CTR_HMOVES], n_moves);
    atomicAdd(&dv.ctr[CTR_HSITES], n_sites);
  }
}

// ---------------------------------------------------------------------------------
// Shared-memory form: the two bitmaps of the warp's pair in shared memory, word (row, m)
// of lane l's block at ((i RW + m) 32 + l), i = row - l RPL, so the lanes of a warp hit
// distinct banks; a row's neighbours are read wherever they lie.
// ---------------------------------------------------------------------------------
__host__ __device__ inline int seed_span_words(int R, int RW) { return 32 * seed_rpl(R) * RW; }

template <int D, int RW>
__global__ void __launch_bounds__(HSEED_NT) k_houd_seedfill(Job jb, Dev dv, HoudSplit hs) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long *cnts = reinterpret_cast<unsigned long long *>(smem);
  const Geo g = jb.g;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int R = g.R, L1 = g.L1, NBW = hs.NBW;
  const int RPL = seed_rpl(R);
  int lg = 0;
  while ((1 << lg) < RPL) ++lg;
  const int span = seed_span_words(R, RW);
  uint32_t *Qs = reinterpret_cast<uint32_t *>(smem + HFILL_HEAD) + (size_t)warp * 2 * span;
  volatile uint32_t *Cs = Qs + span;
  const long long pairs = (long long)jb.S * jb.T;
  if (threadIdx.x < 2) cnts[threadIdx.x] = 0ull;
  __syncthreads();
  auto at = [&](int row, int m) { return (((row & (RPL - 1)) * RW + m) << 5) + (row >> lg); };
  const uint32_t t_houd = (uint32_t)dv.ctr[CTR_THOUD];
  unsigned long long n_moves = 0ull, n_sites = 0ull;
  for (long long gp = next_pair(hs.queue, pairs); gp >= 0; gp = next_pair(hs.queue, pairs)) {
    const int s = (int)(gp / jb.T), a = (int)(gp - (long long)s * jb.T);
    const uint32_t M = hs.Mg[(size_t)s * 32 + a];
    if (M == 0u) continue;
    const uint32_t *Qp = hs.Qg + ((size_t)s * jb.T + a) * NBW;
    uint32_t *Cp = hs.Cg + ((size_t)s * jb.T + a) * NBW;
    // this lane's block: q words in, cluster words cleared, q = -1 sites counted
    uint32_t cnt = 0u;
    for (int i = 0; i < RPL; ++i) {
      const int row = lane * RPL + i;
#pragma unroll
      for (int m = 0; m < RW; ++m) {
        const uint32_t w = row < R ? Qp[row * RW + m] : 0u;
        Qs[at(row, m)] = w;
        Cs[at(row, m)] = 0u;
        cnt += __popc(w);
      }
    }
    const uint32_t n = seed_index(jb, dv, s, a, M, t_houd);
    uint32_t pre = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(FULLM, pre, o);
      if (lane >= o) pre += v;
    }
    pre -= cnt;
    __syncwarp();
    if (n >= pre && n < pre + cnt) {
      uint32_t rem = n - pre;
      bool found = false;
      for (int i = 0; i < RPL && !found; ++i) {
        const int row = lane * RPL + i;
        uint32_t qr[RW], x[RW], f[RW];
#pragma unroll
        for (int m = 0; m < RW; ++m) {
          qr[m] = Qs[at(row, m)];
          x[m] = 0u;
          const uint32_t pc = __popc(qr[m]);
          if (!found) {
            if (rem < pc) {
              uint32_t w = qr[m];
              for (uint32_t j = 0; j < rem; ++j) w &= w - 1u;
              x[m] = w & (0u - w);
              found = true;
            } else {
              rem -= pc;
            }
          }
        }
        if (found) {
          close_row<RW>(qr, x, f, g.L0);
#pragma unroll
          for (int m = 0; m < RW; ++m) Cs[at(row, m)] = f[m];
        }
      }
    }
    __syncwarp();
    const int max_passes = g.N + 2;
    int pass = 0;
    for (; pass < max_passes; ++pass) {
      bool changed = false;
      for (int v = 0; v < 2 * RPL; ++v) {
        const int i = v < RPL ? v : 2 * RPL - 1 - v;
        const int row = lane * RPL + i;
        if (row >= R) continue;
        const int y = row % L1, z = row / L1;
        int nr[2 * (D - 1)];
        nr[0] = (y + 1 == L1) ? row - (L1 - 1) : row + 1;
        nr[1] = (y == 0) ? row + (L1 - 1) : row - 1;
        if (D == 3) {
          nr[2] = (z + 1 == g.L2) ? row - (g.L2 - 1) * L1 : row + L1;
          nr[3] = (z == 0) ? row + (g.L2 - 1) * L1 : row - L1;
        }
        uint32_t qr[RW], cr[RW], x[RW];
        bool any = false;
#pragma unroll
        for (int m = 0; m < RW; ++m) {
          qr[m] = Qs[at(row, m)];
          cr[m] = Cs[at(row, m)];
          uint32_t nb = 0u;
#pragma unroll
          for (int t = 0; t < 2 * (D - 1); ++t) nb |= Cs[at(nr[t], m)];
          x[m] = qr[m] & ~cr[m] & nb;
          any |= x[m] != 0u;
        }
        if (any) {
          uint32_t f[RW];
          close_row<RW>(qr, x, f, g.L0);
#pragma unroll
          for (int m = 0; m < RW; ++m) Cs[at(row, m)] = cr[m] | f[m];
          changed = true;
        }
      }
      const bool more = __any_sync(FULLM, changed);
      __syncwarp();
      if (!more) break;
    }
    if (pass == max_passes && lane == 0) atomicOr(&dv.ctr[CTR_ERROR], ERR_HOUD_ROUNDS);
    uint32_t size = 0u;
    for (int i = 0; i < RPL; ++i) {
      const int row = lane * RPL + i;
      if (row >= R) break;
#pragma unroll
      for (int m = 0; m < RW; ++m) {
        const uint32_t w = Cs[at(row, m)];
        Cp[row * RW + m] = w;
        size += __popc(w);
      }
    }
    size = __reduce_add_sync(FULLM, size);
    n_moves += 1ull;
    n_sites += size;
    __syncwarp();
  }
  if (lane == 0 && n_moves) {
    atomicAdd(&cnts[0], n_moves);
    atomicAdd(&cnts[1], n_sites);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (cnts[0]) atomicAdd(&dv.ctr[CTR_HMOVES], cnts[0]);
    if (cnts[1]) atomicAdd(&dv.ctr[CTR_HSITES], cnts[1]);
  }
}

typedef void (*seed_fn)(Job, Dev, HoudSplit);

template <int D, int RPL>
seed_fn pick_reg_rw(int RW) {
  if (RPL <= 4) {
    switch (RW) {
    case 1: return k_houd_seedreg<D, 1, RPL>;
    case 2: return k_houd_seedreg<D, 2, RPL>;
    case 3: return k_houd_seedreg<D, 3, RPL>;
    case 4: return k_houd_seedreg<D, 4, RPL>;
    default: return nullptr;
    }
  }
  switch (RW) {
  case 1: return k_houd_seedreg<D, 1, 8>;
  case 2: return k_houd_seedreg<D, 2, 8>;
  default: return nullptr;
  }
}

// The register form for this lattice, or null where it does not apply.
seed_fn pick_reg(const Job &jb, int RW) {
  const int RPL = seed_rpl(jb.g.R);
  if (RPL > 8 || RW > 4 || RW * RPL > 16 || jb.g.L1 % RPL != 0) return nullptr;
  if (jb.g.d == 2) {
    switch (RPL) {
    case 1: return pick_reg_rw<2, 1>(RW);
    case 2: return pick_reg_rw<2, 2>(RW);
    case 4: return pick_reg_rw<2, 4>(RW);
    default: return pick_reg_rw<2, 8>(RW);
    }
  }
  switch (RPL) {
  case 1: return pick_reg_rw<3, 1>(RW);
  case 2: return pick_reg_rw<3, 2>(RW);
  case 4: return pick_reg_rw<3, 4>(RW);
  default: return pick_reg_rw<3, 8>(RW);
  }
}

template <int D>
seed_fn pick_smem_rw(int RW) {
  switch (RW) {
  case 1: return k_houd_seedfill<D, 1>;
  case 2: return k_houd_seedfill<D, 2>;
  case 3: return k_houd_seedfill<D, 3>;
  case 4: return k_houd_seedfill<D, 4>;
  case 5: return k_houd_seedfill<D, 5>;
  case 6: return k_houd_seedfill<D, 6>;
  case 7: return k_houd_seedfill<D, 7>;
  default: return k_houd_seedfill<D, 8>;
  }
}

// Grid of a queue-driven kernel: the CTAs that are resident at once, at most one warp per pair.
int seed_grid(seed_fn fn, size_t smem, long long pairs, int n_sm) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, HSEED_NT, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const long long need = (pairs + HSEED_NT / 32 - 1) / (HSEED_NT / 32);
  const long long grid = (long long)per_sm * n_sm;
  return (int)(grid < need ? grid : need);
}

} // namespace

cudaError_t launch_houd_seed(const Job &jb, const Dev &dv, const HoudSplit &hs, int n_sm, cudaStream_t st,
                             bool *launched) {
  *launched = false;
  const long long pairs = (long long)jb.S * jb.T;
  if (const seed_fn fn = pick_reg(jb, hs.RW)) {
    fn<<<(unsigned)seed_grid(fn, 0, pairs, n_sm), HSEED_NT, 0, st>>>(jb, dv, hs);
    *launched = true;
    return cudaGetLastError();
  }
  if (jb.g.d == 3) {
    // shared memory: 8 pairs' bitmaps per CTA, within the Houdayer shared-memory budget
    const size_t smem = HFILL_HEAD + (size_t)(HSEED_NT / 32) * 2 * seed_span_words(jb.g.R, hs.RW) * 4;
    if (smem <= (size_t)HOUD_SMEM_BUDGET) {
      const seed_fn fn = pick_smem_rw<3>(hs.RW);
      fn<<<(unsigned)seed_grid(fn, smem, pairs, n_sm), HSEED_NT, smem, st>>>(jb, dv, hs);
      *launched = true;
      return cudaGetLastError();
    }
  }
  return cudaSuccess;
}

cudaError_t prepare_houd_seed_kernels(int max_smem) {
  for (int rw = 1; rw <= 8; ++rw)
    for (const void *fn : {(const void *)pick_smem_rw<2>(rw), (const void *)pick_smem_rw<3>(rw)}) {
      const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

} // namespace sgmc
