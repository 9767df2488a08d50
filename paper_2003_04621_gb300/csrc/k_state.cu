// k_state.cu -- creation (Eq. 2 couplings, hot start), import/export of spins and
// couplings in plain layouts, and the measurement of E by slot and N q (Eqs. 3-4).
#include "sgmc_internal.cuh"
#include "sgmc_tma.cuh"
#include "sgmc_sweep.cuh"

namespace sgmc {

// Couplings (Eq. 2): thread per (sample, axis, plane word); each builds one 32-bit word
// of the bit plane, bit b = 1 iff J(i(p), mu) = -1 for p = 32 n + b.
__global__ void k_init_couplings(Job jb, Dev dv) {
  const Geo g = jb.g;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)jb.S * g.d * g.NW;
  if (idx >= total) return;
  const int n = (int)(idx % g.NW);
  const int mu = (int)((idx / g.NW) % g.d);
  const int s = (int)(idx / ((long long)g.NW * g.d));
  uint32_t word = 0;
  for (int b = 0; b < 32; ++b) {
    const int p = n * 32 + b;
    if (p >= g.N) break;
    const int i = canonical_of(g, site_geo(g, p));
    const uint32_t w = philox10((uint32_t)i, (uint32_t)mu, (uint32_t)(jb.s_off + s), TAG_J, jb.ck0, jb.ck1).x;
    if (!((unsigned long long)w < jb.jcut)) word |= 1u << b;
  }
  dv.jbits[idx] = word;
}

// Hot start, packed: thread per (sample, word, site).
__global__ void k_init_spins_packed(Job jb, Dev dv) {
  const Geo g = jb.g;
  const int p = blockIdx.x * blockDim.x + threadIdx.x; // site (colour-split order)
  if (p >= g.N) return;
  const uint32_t i = (uint32_t)canonical_of(g, site_geo(g, p));
  for (int plane = blockIdx.y; plane < jb.S * jb.W; plane += gridDim.y) { // (sample, word)
    const int s = plane / jb.W, w = plane - s * jb.W;
    const int c = w / jb.Wc, wc = w - c * jb.Wc;
    const int nvalid = min(32, jb.T - wc * 32);
    // the word's eight calls are independent: evaluate them together, keep the valid lanes
    uint4 r[8];
#pragma unroll
    for (int gi = 0; gi < 8; ++gi) {
      const uint32_t c3 = ((uint32_t)c << 20) | ((uint32_t)(wc * 8 + gi) << 8) | TAG_INIT;
      r[gi] = philox10(i, 0u, (uint32_t)(jb.s_off + s), c3, jb.sk0, jb.sk1);
    }
    uint32_t word = 0;
#pragma unroll
    for (int gi = 0; gi < 8; ++gi)
      word |= ((r[gi].x >> 31) | ((r[gi].y >> 31) << 1) | ((r[gi].z >> 31) << 2) | ((r[gi].w >> 31) << 3)) << (4 * gi);
    if (nvalid < 32) word &= (1u << nvalid) - 1u;
    dv.spins[(size_t)plane * g.N + p] = word;
  }
}

// Hot start, int8: thread per (sample, chain, site, group of four replicas).
__global__ void k_init_spins_int8(Job jb, Dev dv) {
  const Geo g = jb.g;
  const int G = jb.Tp / 4;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)jb.S * jb.C * g.N * G) return;
  const int gi = (int)(idx % G);
  const long long site_idx = idx / G; // (s, c, p)
  const int p = (int)(site_idx % g.N);
  const int c = (int)((site_idx / g.N) % jb.C);
  const int s = (int)(site_idx / ((long long)g.N * jb.C));
  const uint32_t i = (uint32_t)canonical_of(g, site_geo(g, p));
  const uint32_t c3 = ((uint32_t)c << 20) | ((uint32_t)gi << 8) | TAG_INIT;
  const uint4 r = philox10(i, 0u, (uint32_t)(jb.s_off + s), c3, jb.sk0, jb.sk1);
  int8_t v[4];
  for (int q = 0; q < 4; ++q) v[q] = (gi * 4 + q < jb.T && (word_of(r, q) >> 31)) ? -1 : 1;
  reinterpret_cast<char4 *>(dv.spins)[idx] = make_char4(v[0], v[1], v[2], v[3]);
}

__global__ void k_init_maps(Job jb, Dev dv) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)jb.S * jb.C * jb.T) return;
  const int j = (int)(idx % jb.T);
  dv.perm[idx] = j;
  dv.slot[idx] = j;
}

// Spins to the plain layout out[s][c][j][i] (1 iff s = -1): thread per output byte.
__global__ void k_export_spins(Job jb, Dev dv, int int8fmt, uint8_t *out) {
  const Geo g = jb.g;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)jb.S * jb.C * jb.T * g.N) return;
  const int i = (int)(idx % g.N);
  const long long r = idx / g.N; // (s, c, j)
  const int j = (int)(r % jb.T);
  const int c = (int)((r / jb.T) % jb.C);
  const int s = (int)(r / ((long long)jb.T * jb.C));
  const int p = cs_of_canonical(g, i);
  uint8_t bit;
  if (int8fmt) {
    const int8_t *sp = reinterpret_cast<const int8_t *>(dv.spins);
    bit = sp[(((size_t)s * jb.C + c) * g.N + p) * jb.Tp + j] < 0;
  } else {
    const int w = c * jb.Wc + j / 32;
    bit = (dv.spins[((size_t)s * jb.W + w) * g.N + p] >> (j & 31)) & 1u;
  }
  out[idx] = bit;
}

// Plain layout -> spins.  Packed: thread per (sample, word, site); int8: per spin.
__global__ void k_import_spins(Job jb, Dev dv, int int8fmt, const uint8_t *in) {
  const Geo g = jb.g;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (int8fmt) {
    if (idx >= (long long)jb.S * jb.C * g.N * jb.Tp) return;
    const int j = (int)(idx % jb.Tp);
    const long long r = idx / jb.Tp; // (s, c, p)
    const int p = (int)(r % g.N);
    const int c = (int)((r / g.N) % jb.C);
    const int s = (int)(r / ((long long)g.N * jb.C));
    int8_t v = 1;
    if (j < jb.T) {
      const int i = canonical_of(g, site_geo(g, p));
      v = in[(((size_t)s * jb.C + c) * jb.T + j) * g.N + i] ? -1 : 1;
    }
    reinterpret_cast<int8_t *>(dv.spins)[idx] = v;
    return;
  }
  if (idx >= (long long)jb.S * jb.W * g.N) return;
  const int p = (int)(idx % g.N);
  const int w = (int)((idx / g.N) % jb.W);
  const int s = (int)(idx / ((long long)g.N * jb.W));
  const int c = w / jb.Wc, wc = w - c * jb.Wc;
  const int nvalid = min(32, jb.T - wc * 32);
  const int i = canonical_of(g, site_geo(g, p));
  uint32_t word = 0;
  for (int l = 0; l < nvalid; ++l) {
    const int j = wc * 32 + l;
    word |= (uint32_t)(in[(((size_t)s * jb.C + c) * jb.T + j) * g.N + i] != 0) << l;
  }
  dv.spins[idx] = word;
}

// Couplings to the plain layout out[s][i][mu] = +-1: thread per entry.
__global__ void k_export_couplings(Job jb, Dev dv, int8_t *out) {
  const Geo g = jb.g;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)jb.S * g.N * g.d) return;
  const int mu = (int)(idx % g.d);
  const int i = (int)((idx / g.d) % g.N);
  const int s = (int)(idx / ((long long)g.d * g.N));
  const int p = cs_of_canonical(g, i);
  const uint32_t w = dv.jbits[((size_t)s * g.d + mu) * g.NW + (p >> 5)];
  out[idx] = ((w >> (p & 31)) & 1u) ? -1 : 1;
}

// Plain layout -> coupling bit planes: thread per plane word.
__global__ void k_import_couplings(Job jb, Dev dv, const int8_t *in) {
  const Geo g = jb.g;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)jb.S * g.d * g.NW) return;
  const int n = (int)(idx % g.NW);
  const int mu = (int)((idx / g.NW) % g.d);
  const int s = (int)(idx / ((long long)g.NW * g.d));
  uint32_t word = 0;
  for (int b = 0; b < 32; ++b) {
    const int p = n * 32 + b;
    if (p >= g.N) break;
    const int i = canonical_of(g, site_geo(g, p));
    if (in[((size_t)s * g.N + i) * g.d + mu] < 0) word |= 1u << b;
  }
  dv.jbits[idx] = word;
}

// E by temperature slot: thread per (sample, chain, slot).
__global__ void k_gather_energy(Job jb, Dev dv, int32_t *E_out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)jb.S * jb.C * jb.T) return;
  const long long base = idx - idx % jb.T;
  E_out[idx] = dv.E[base + dv.perm[idx]];
}

// N q (Eq. 4) per (sample, slot), int8 layout: CTA per (sample, slot); q = -1 sites are
// those where the chain-0 and chain-1 replicas at the slot differ.
__global__ void k_overlap_int8(Job jb, Dev dv, int32_t *Q_out) {
  const Geo g = jb.g;
  const int s = blockIdx.x / jb.T;
  const int k = blockIdx.x - s * jb.T;
  const int a = dv.perm[((size_t)s * jb.C + 0) * jb.T + k];
  const int b = dv.perm[((size_t)s * jb.C + 1) * jb.T + k];
  const int8_t *sp = reinterpret_cast<const int8_t *>(dv.spins);
  const int8_t *pa = sp + ((size_t)s * jb.C + 0) * g.N * jb.Tp + a;
  const int8_t *pb = sp + ((size_t)s * jb.C + 1) * g.N * jb.Tp + b;
  int cnt = 0;
  for (int p = threadIdx.x; p < g.N; p += blockDim.x) cnt += pa[(size_t)p * jb.Tp] != pb[(size_t)p * jb.Tp];
  __shared__ int red[32];
  cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0;
    v = __reduce_add_sync(0xFFFFFFFFu, v);
    if (threadIdx.x == 0) Q_out[blockIdx.x] = g.N - 2 * v;
  }
}

// N q per (sample, slot), packed layout: CTA per (sample, block of 32 slots).  The CTA
// stages the sample's W word planes through shared memory in tiles of `tl` sites
// (16-byte coalesced loads, several in flight per thread); then lane = slot, and each
// warp counts over its share of the tile's sites the q = -1 sites of the lane's pair,
// reading the two words it needs from shared memory (one broadcast per word).  N is a
// multiple of 4 (every extent even), so every word plane starts 16-byte aligned.
constexpr int OV_NT = 256, OV_TILE = 1024, OV_SMEM = 44 * 1024; // with the static 1 KB, under 48 KB

// Sites per tile: up to OV_TILE, fewer when the W planes would exceed OV_SMEM bytes; a
// multiple of 4.
inline int overlap_tile(int W) {
  int tl = OV_SMEM / (4 * W);
  tl = tl > OV_TILE ? OV_TILE : tl;
  return tl & ~3;
}

__global__ void __launch_bounds__(OV_NT) k_overlap_packed(Job jb, Dev dv, int tl, int32_t *Q_out) {
  extern __shared__ __align__(16) uint32_t tile[]; // [W][tl]
  __shared__ uint32_t red[OV_NT / 32][32];
  const Geo g = jb.g;
  const int nblk = (jb.T + 31) >> 5;
  const int s = blockIdx.x / nblk, blk = blockIdx.x - s * nblk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = blk * 32 + lane;
  const bool valid = k < jb.T;
  const int a = valid ? dv.perm[((size_t)s * jb.C + 0) * jb.T + k] : 0;
  const int b = valid ? dv.perm[((size_t)s * jb.C + 1) * jb.T + k] : 0;
  const uint32_t *ta = tile + (size_t)(a >> 5) * tl;
  const uint32_t *tb = tile + (size_t)(jb.Wc + (b >> 5)) * tl;
  const int la = a & 31, lb = b & 31;
  const int W = jb.W;
  const uint4 *src = reinterpret_cast<const uint4 *>(dv.spins + (size_t)s * W * g.N);
  const int n4 = g.N >> 2;
  uint32_t cnt = 0u;
  for (int base = 0; base < g.N; base += tl) {
    const int len = min(tl, g.N - base); // a multiple of 4
    const int len4 = len >> 2;
    __syncthreads();
    for (int e = threadIdx.x; e < W * len4; e += OV_NT) {
      const int w = e / len4, i = e - w * len4;
      reinterpret_cast<uint4 *>(tile + (size_t)w * tl)[i] = src[(size_t)w * n4 + (base >> 2) + i];
    }
    __syncthreads();
    const int per = (len + OV_NT / 32 - 1) / (OV_NT / 32);
    const int p0 = warp * per, p1 = min(len, p0 + per);
    for (int p = p0; p < p1; ++p) cnt += ((ta[p] >> la) ^ (tb[p] >> lb)) & 1u;
  }
  red[warp][lane] = cnt;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = 0u;
#pragma unroll
    for (int w = 0; w < OV_NT / 32; ++w) v += red[w][lane];
    if (valid) Q_out[(size_t)s * jb.T + k] = g.N - 2 * (int32_t)v;
  }
}

// Both observables of a two-chain packed job whose chains are one word each (T <= 32),
// in one pass per sample: E by slot and N q per slot (Eqs. 3-4).  One CTA per sample.
// The chain-1 word is permuted into chain-0 lane order (bit b moves to lane
// perm0[slot1[b]], the chain-0 replica at the same temperature), so bit a of
// w0 ^ sigma(w1) is 1 iff the pair of chain-0 replica a disagrees at that site.  Four
// sites' disagreement words are compressed to a 3-bit value and added into bit-sliced
// counters, 32 pairs per instruction; the warp sums its counters by butterfly before
// they can overflow (8 planes: at most 63 iterations of 4 sites).
constexpr int MP_NT = 128;

__global__ void __launch_bounds__(MP_NT) k_measure_pairs_w1(Job jb, Dev dv, int32_t *E_out, int32_t *Q_out) {
  __shared__ uint32_t sig[1024];
  __shared__ uint32_t nib[128];   // the same permutation by nibbles: [nibble][value]
  __shared__ int32_t maps[4][32]; // perm0, perm1, slot0, slot1
  __shared__ uint32_t tot[32];    // disagreeing sites of the pair of chain-0 replica a
  const int s = blockIdx.x, T = jb.T, tid = threadIdx.x, lane = tid & 31;
  const size_t c0 = (size_t)s * 2 * T;
  if (tid < 32) {
    maps[0][tid] = tid < T ? dv.perm[c0 + tid] : 0;
    maps[1][tid] = tid < T ? dv.perm[c0 + T + tid] : 0;
    maps[2][tid] = tid < T ? dv.slot[c0 + tid] : 0;
    maps[3][tid] = tid < T ? dv.slot[c0 + T + tid] : 0;
    tot[tid] = 0u;
  }
  __syncthreads();
  for (int e = tid; e < 128; e += MP_NT) {
    const int j = e >> 4, v = e & 15;
    uint32_t o = 0u;
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      const int b = 4 * j + bb;
      if (((v >> bb) & 1) && b < T) o |= 1u << maps[0][maps[3][b]];
    }
    nib[e] = o;
  }
  __syncthreads();
  for (int e = tid; e < 1024; e += MP_NT) {
    const int j = e >> 8, v = e & 255;
    sig[e] = nib[(2 * j) * 16 + (v & 15)] | nib[(2 * j + 1) * 16 + (v >> 4)];
  }
  if (E_out)
    for (int e = tid; e < 2 * T; e += MP_NT) {
      const int c = e >= T ? 1 : 0;
      E_out[c0 + e] = dv.E[c0 + (size_t)c * T + maps[c][e - c * T]];
    }
  __syncthreads();
  if (!Q_out) return;
  const int N = jb.g.N, n4 = N >> 2; // every extent is even, so N is a multiple of 4
  const uint4 *p0 = reinterpret_cast<const uint4 *>(dv.spins + (size_t)s * jb.W * N);
  const uint4 *p1 = p0 + n4;
  uint32_t V[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) V[b] = 0u;
  const int iters = (n4 + MP_NT - 1) / MP_NT;
  for (int it = 0; it < iters; ++it) {
    const int i = it * MP_NT + tid;
    if (i < n4) {
      const uint4 a = p0[i], b = p1[i];
      const uint32_t q0 = a.x ^ permute_word(sig, b.x), q1 = a.y ^ permute_word(sig, b.y);
      const uint32_t q2 = a.z ^ permute_word(sig, b.z), q3 = a.w ^ permute_word(sig, b.w);
      uint32_t s1, cy1;
      fadd(q0, q1, q2, s1, cy1);
      const uint32_t cc = s1 & q3;
      vcount_add(V, s1 ^ q3, cy1 ^ cc, cy1 & cc);
    }
    if ((it + 1) % 63 == 0 || it + 1 == iters) { // warp-uniform
      const int32_t v = warp_lane_sum(V);
      if (v) atomicAdd(&tot[lane], (uint32_t)v);
#pragma unroll
      for (int b = 0; b < NB; ++b) V[b] = 0u;
    }
  }
  __syncthreads();
  if (tid < T) Q_out[(size_t)s * T + maps[2][tid]] = N - 2 * (int32_t)tot[tid];
}

// ---------------------------------------------------------------------------------
// Overlap plane sums (the integer part of the Fourier modes of q behind chi_SG and the
// correlation length, two-replica measurements of Sec. 3): P[s][k][mu][x] = sum of
// q_i = s_i^(a) s_i^(b) over the sites with coordinate x along axis mu, a / b the
// chain-0 / chain-1 replicas at slot k.  Entries x >= L_mu are 0.
// ---------------------------------------------------------------------------------
constexpr int QM_NT = 256;

// Packed layout: CTA per (sample, block of 32 slots), lane = slot.  Rows are staged in
// shared memory a tile at a time (both colour halves of every word plane); warps take
// rows, walk them by half-column (two sites, one per colour, with known x), and each
// lane adds its slot's q into its slot's accumulators: x in acc[mu=0], the row sum into
// acc[1][y] and acc[2][z].  The warps share a slot's accumulators, so the adds are
// atomic; a slot's accumulators are d Lmax + 1 words apart, so the 32 lanes of a warp
// hit 32 banks.  With GACC they live in the global output instead.
template <int D, bool GACC>
__global__ void __launch_bounds__(QM_NT) k_qmodes_packed(Job jb, Dev dv, int Lmax, int nr, int32_t *P_out) {
  extern __shared__ __align__(16) uint32_t qm_smem[];
  const Geo g = jb.g;
  const int H = g.H, L1 = g.L1, R = g.R;
  const int nblk = (jb.T + 31) >> 5;
  const int s = blockIdx.x / nblk, blk = blockIdx.x - s * nblk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = blk * 32 + lane;
  const bool valid = k < jb.T;
  const int a = valid ? dv.perm[((size_t)s * jb.C + 0) * jb.T + k] : 0;
  const int b = valid ? dv.perm[((size_t)s * jb.C + 1) * jb.T + k] : 0;
  const int W = jb.W, la = a & 31, lb = b & 31;
  const int stride = D * Lmax + 1;
  uint32_t *tile = qm_smem;                 // [W][2][nr * H]
  const int tw = 2 * nr * H;                // words per plane in the tile
  int32_t *acc = GACC ? P_out + ((size_t)s * jb.T + (valid ? k : 0)) * D * Lmax
                      : reinterpret_cast<int32_t *>(qm_smem + (size_t)W * tw) + lane * stride;
  const uint32_t *ta0 = tile + (size_t)(a >> 5) * tw, *tb0 = tile + (size_t)(jb.Wc + (b >> 5)) * tw;
  // warp 0 clears every slot's accumulators (the tile loop's first barrier orders it
  // before any add)
  if (warp == 0 && (!GACC || valid))
    for (int i = 0; i < D * Lmax; ++i) acc[i] = 0;
  const uint32_t *src = dv.spins + (size_t)s * W * g.N;
  for (int r0 = 0; r0 < R; r0 += nr) {
    const int rows = min(nr, R - r0), n = rows * H;
    __syncthreads();
    // 2W contiguous segments (plane w, colour c) of n words; 16-byte copies when the
    // half-row length is a multiple of 4 words (then every segment starts 16-byte aligned)
    for (int seg = 0; seg < 2 * W; ++seg) {
      const int w = seg >> 1, c = seg & 1;
      uint32_t *dst = tile + (size_t)w * tw + c * nr * H;
      const uint32_t *from = src + (size_t)w * g.N + c * g.Nh + (size_t)r0 * H;
      if ((H & 3) == 0) {
        for (int i = threadIdx.x; i < (n >> 2); i += QM_NT)
          reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(from)[i];
      } else {
        for (int i = threadIdx.x; i < n; i += QM_NT) dst[i] = from[i];
      }
    }
    __syncthreads();
    for (int rr = warp; rr < rows; rr += QM_NT / 32) {
      const int r = r0 + rr, y = r % L1, z = r / L1, par = (y + z) & 1;
      int rowsum = 0;
      for (int kk = 0; kk < H; ++kk) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int i = c * nr * H + rr * H + kk;
          const int x = 2 * kk + (c ^ par);
          const int q = 1 - 2 * (int)(((ta0[i] >> la) ^ (tb0[i] >> lb)) & 1u);
          if (!GACC || valid) atomicAdd(&acc[x], q);
          rowsum += q;
        }
      }
      if (!GACC || valid) {
        atomicAdd(&acc[Lmax + y], rowsum);
        if (D == 3) atomicAdd(&acc[2 * Lmax + z], rowsum);
      }
    }
  }
  __syncthreads(); // every warp's adds are in before a lane copies its slot out
  if (!GACC) {
    if (valid) {
      int32_t *out = P_out + ((size_t)s * jb.T + k) * D * Lmax;
      for (int i = 0; i < D * Lmax; ++i) out[i] = acc[i];
    }
  }
}

// Two-chain packed jobs whose chains are one word each (T <= 32): one CTA per sample.
// The disagreement words d = w0 ^ sigma(w1) of 32 sites (sigma as in k_measure_pairs_w1)
// are transposed across the warp, so that lane a holds the disagreements of the pair of
// chain-0 replica a at the step's 32 sites, bit t for the site of lane t.  A step covers
// `rps` whole rows when L0 <= 32 (lane t: row t / L0, x = t % L0), else a 32-site chunk
// of one row, the warp's chunk fixed.  A row's popcount is its count, added to its y and
// z planes.  Bit-sliced counters over the steps hold the count of each bit position, i.e.
// of each x, until they are emptied (every 255 steps and at the end).
// P = (sites in the plane) - 2 (disagreements).
constexpr int QW_NT = 256;

// Empty a lane's bit-sliced x-plane counters into its pair's accumulators: bit t counts
// the site of lane t (x = t mod L0 for rows of at most 32 sites, else 32 chunk + t).
// The planes in use (those below the warp's highest nonzero one) are summed per x
// first, so each x takes one atomic add.
__device__ __forceinline__ void qw_flush(uint32_t (&V)[NB], bool narrow, int L0, uint32_t rep, int chunk,
                                         uint32_t *drow) {
  int nb = 0;
#pragma unroll
  for (int b = 0; b < NB; ++b) nb = __any_sync(0xFFFFFFFFu, V[b] != 0u) ? b + 1 : nb;
  if (narrow) {
    for (int xx = 0; xx < L0; ++xx) {
      uint32_t c = 0u;
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (b < nb) c += (uint32_t)__popc(V[b] & (rep << xx)) << b;
      if (c) atomicAdd(&drow[xx], c);
    }
  } else {
    for (int t = 0; t < 32 && 32 * chunk + t < L0; ++t) {
      uint32_t c = 0u;
#pragma unroll
      for (int b = 0; b < NB; ++b) c |= ((V[b] >> t) & 1u) << b;
      if (c) atomicAdd(&drow[32 * chunk + t], c);
    }
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) V[b] = 0u;
}

template <int D>
__global__ void __launch_bounds__(QW_NT, 4) k_qmodes_w1(Job jb, Dev dv, int Lmax, int32_t *P_out) {
  extern __shared__ __align__(16) uint32_t qw_smem[];
  uint32_t *sig = qw_smem;                                  // [1024]
  uint32_t *nib = sig + 1024;                               // [128]
  int32_t *maps = reinterpret_cast<int32_t *>(nib + 128);   // [4][32] perm0, perm1, slot0, slot1
  const int stride = D * Lmax + 1;                          // per pair; odd, so lanes hit 32 banks
  uint32_t *dis = reinterpret_cast<uint32_t *>(maps + 128); // [32][stride]
  const Geo g = jb.g;
  const int s = blockIdx.x, T = jb.T, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int L0 = g.L0, L1 = g.L1, H = g.H, R = g.R, Nh = g.Nh, N = g.N;
  const size_t c0 = (size_t)s * 2 * T;
  if (tid < 32) {
    maps[tid] = tid < T ? dv.perm[c0 + tid] : 0;
    maps[32 + tid] = tid < T ? dv.perm[c0 + T + tid] : 0;
    maps[64 + tid] = tid < T ? dv.slot[c0 + tid] : 0;
    maps[96 + tid] = tid < T ? dv.slot[c0 + T + tid] : 0;
  }
  for (int i = tid; i < 32 * stride; i += QW_NT) dis[i] = 0u;
  __syncthreads();
  for (int e = tid; e < 128; e += QW_NT) {
    const int j = e >> 4, v = e & 15;
    uint32_t o = 0u;
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      const int b = 4 * j + bb;
      if (((v >> bb) & 1) && b < T) o |= 1u << maps[maps[96 + b]];
    }
    nib[e] = o;
  }
  __syncthreads();
  for (int e = tid; e < 1024; e += QW_NT) {
    const int j = e >> 8, v = e & 255;
    sig[e] = nib[(2 * j) * 16 + (v & 15)] | nib[(2 * j + 1) * 16 + (v >> 4)];
  }
  __syncthreads();

  const uint32_t *w0 = dv.spins + (size_t)s * jb.W * N, *w1 = w0 + N;
  const bool narrow = L0 <= 32;
  const int rps = narrow ? 32 / L0 : 1;            // rows per step
  const int nch = narrow ? 1 : (L0 + 31) >> 5;     // chunks per row
  const int nw = QW_NT / 32;
  const int wpc = narrow ? nw : nw / nch;          // warps per chunk (launcher: nch <= nw)
  const bool active = narrow || warp < wpc * nch;
  const int chunk = narrow ? 0 : warp % nch;
  const int step0 = narrow ? warp : warp / nch;    // first row group of this warp
  const int sstride = narrow ? nw : wpc;
  const int nsteps = narrow ? (R + rps - 1) / rps : R;
  const uint32_t segmask = L0 >= 32 ? 0xFFFFFFFFu : ((1u << L0) - 1u);
  uint32_t rep = 0u; // one bit per row of a step, at the row's first lane
  for (int j = 0; j < rps; ++j) rep |= 1u << (j * L0);
  // this lane's site within a step
  const int jrow = narrow ? lane / L0 : 0;
  const int x = narrow ? lane - jrow * L0 : 32 * chunk + lane;
  const bool lane_ok = narrow ? jrow < rps : x < L0;
  const uint32_t mL1 = div_magic(L1);
  uint32_t V[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) V[b] = 0u;
  int since = 0;
  uint32_t *drow = dis + lane * stride; // this lane's pair
  constexpr int U = 4; // steps whose words are loaded before any is used
  if (active) {
    for (int st0 = step0; st0 < nsteps; st0 += U * sstride) {
      uint32_t a[U], bw[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int st = st0 + u * sstride;
        const int r = narrow ? st * rps + jrow : st;
        a[u] = bw[u] = 0u;
        if (st < nsteps && lane_ok && r < R) {
          const int z = div_by(r, L1, mL1), y = r - z * L1;
          const int p = ((x & 1) ^ ((y + z) & 1)) * Nh + r * H + (x >> 1);
          a[u] = w0[p];
          bw[u] = w1[p];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int st = st0 + u * sstride;
        if (st >= nsteps) break; // warp-uniform
        // empty words permute to 0, so lanes without a site give 0
        const uint32_t X = transpose32(a[u] ^ permute_word(sig, bw[u]), lane);
        // rows: y and z planes
        for (int j = 0; j < rps; ++j) {
          const int rr = narrow ? st * rps + j : st;
          if (rr >= R) break;
          const uint32_t cnt = __popc(narrow ? (X >> (j * L0)) & segmask : X);
          if (cnt) {
            const int z = div_by(rr, L1, mL1);
            atomicAdd(&drow[Lmax + rr - z * L1], cnt);
            if (D == 3) atomicAdd(&drow[2 * Lmax + z], cnt);
          }
        }
        // x planes: add X into the bit-sliced counters (one plane carries into the next)
        uint32_t cy = X;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const uint32_t t2 = V[b] & cy;
          V[b] ^= cy;
          cy = t2;
        }
        if (++since == 255) { // NB = 8 planes hold up to 255 per bit
          qw_flush(V, narrow, L0, rep, chunk, drow);
          since = 0;
        }
      }
    }
    qw_flush(V, narrow, L0, rep, chunk, drow);
  }
  __syncthreads();
  // slot k's pair is the one of chain-0 replica perm0[k]
  for (int e = tid; e < T * D * Lmax; e += QW_NT) {
    const int k = e / (D * Lmax), i = e - k * (D * Lmax);
    const int mu = i / Lmax, xx = i - mu * Lmax;
    const int Lmu = mu == 0 ? L0 : (mu == 1 ? L1 : g.L2);
    P_out[((size_t)s * T + k) * D * Lmax + i] =
        xx < Lmu ? N / Lmu - 2 * (int32_t)dis[maps[k] * stride + i] : 0;
  }
}

// int8 layout: CTA per (sample, slot); shared-memory accumulators, atomics per site.
__global__ void __launch_bounds__(256) k_qmodes_int8(Job jb, Dev dv, int Lmax, int32_t *P_out) {
  extern __shared__ __align__(16) uint32_t qm_smem[];
  int32_t *acc = reinterpret_cast<int32_t *>(qm_smem);
  const Geo g = jb.g;
  const int d = g.d;
  const int s = blockIdx.x / jb.T, k = blockIdx.x - s * jb.T;
  const int a = dv.perm[((size_t)s * jb.C + 0) * jb.T + k];
  const int b = dv.perm[((size_t)s * jb.C + 1) * jb.T + k];
  const int8_t *sp = reinterpret_cast<const int8_t *>(dv.spins);
  const int8_t *pa = sp + ((size_t)s * jb.C + 0) * g.N * jb.Tp + a;
  const int8_t *pb = sp + ((size_t)s * jb.C + 1) * g.N * jb.Tp + b;
  for (int i = threadIdx.x; i < d * Lmax; i += blockDim.x) acc[i] = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < g.N; p += blockDim.x) {
    const SiteGeo sg = site_geo(g, p);
    const int q = (int)pa[(size_t)p * jb.Tp] * (int)pb[(size_t)p * jb.Tp];
    atomicAdd(&acc[2 * sg.k + sg.xodd], q);
    atomicAdd(&acc[Lmax + sg.y], q);
    if (d == 3) atomicAdd(&acc[2 * Lmax + sg.z], q);
  }
  __syncthreads();
  int32_t *out = P_out + (size_t)blockIdx.x * d * Lmax;
  for (int i = threadIdx.x; i < d * Lmax; i += blockDim.x) out[i] = acc[i];
}

// Rows per staged tile (the tile holds every word plane, both colours, about 24 KB) and
// whether the accumulators fit shared memory (96 KB for 32 lanes).
void qmodes_shape(const Job &jb, int Lmax, int *nr, size_t *smem, bool *gacc) {
  const int per_row = jb.W * 2 * jb.g.H * 4;
  int n = 24 * 1024 / per_row;
  n = n < 1 ? 1 : (n > jb.g.R ? jb.g.R : n);
  const size_t accb = (size_t)32 * (jb.g.d * Lmax + 1) * 4;
  *gacc = accb > 96 * 1024;
  *nr = n;
  *smem = (size_t)n * per_row + (*gacc ? 0 : accb);
}

size_t qmodes_w1_smem(int d, int Lmax) { return (1024 + 128 + 128) * 4 + (size_t)32 * (d * Lmax + 1) * 4; }

int qmodes_lmax(const Job &jb) {
  int m = jb.g.L0;
  if (jb.g.L1 > m) m = jb.g.L1;
  if (jb.g.d == 3 && jb.g.L2 > m) m = jb.g.L2;
  return m;
}

cudaError_t launch_qmodes(const Job &jb, const Dev &dv, bool int8fmt, int32_t *P_out, cudaStream_t st) {
  if (jb.C < 2) return cudaErrorInvalidValue;
  const int Lmax = qmodes_lmax(jb);
  if (int8fmt) {
    k_qmodes_int8<<<(unsigned)(jb.S * jb.T), 256, (size_t)jb.g.d * Lmax * 4, st>>>(jb, dv, Lmax, P_out);
    return cudaGetLastError();
  }
  // chains of one word: the transposed single pass, while its counters fit shared memory
  // and a row has at most one 32-site chunk per warp
  const size_t wsm = qmodes_w1_smem(jb.g.d, Lmax);
  if (jb.C == 2 && jb.Wc == 1 && wsm <= 96 * 1024 && (jb.g.L0 + 31) / 32 <= QW_NT / 32) {
    if (jb.g.d == 2) k_qmodes_w1<2><<<(unsigned)jb.S, QW_NT, wsm, st>>>(jb, dv, Lmax, P_out);
    else k_qmodes_w1<3><<<(unsigned)jb.S, QW_NT, wsm, st>>>(jb, dv, Lmax, P_out);
    return cudaGetLastError();
  }
  int nr;
  size_t smem;
  bool gacc;
  qmodes_shape(jb, Lmax, &nr, &smem, &gacc);
  const unsigned grid = (unsigned)(jb.S * ((jb.T + 31) / 32));
  if (jb.g.d == 2) {
    if (gacc) k_qmodes_packed<2, true><<<grid, QM_NT, smem, st>>>(jb, dv, Lmax, nr, P_out);
    else k_qmodes_packed<2, false><<<grid, QM_NT, smem, st>>>(jb, dv, Lmax, nr, P_out);
  } else {
    if (gacc) k_qmodes_packed<3, true><<<grid, QM_NT, smem, st>>>(jb, dv, Lmax, nr, P_out);
    else k_qmodes_packed<3, false><<<grid, QM_NT, smem, st>>>(jb, dv, Lmax, nr, P_out);
  }
  return cudaGetLastError();
}

cudaError_t prepare_state_kernels(int max_smem) {
  const void *fns[7] = {(const void *)k_qmodes_packed<2, false>, (const void *)k_qmodes_packed<2, true>,
                        (const void *)k_qmodes_packed<3, false>, (const void *)k_qmodes_packed<3, true>,
                        (const void *)k_qmodes_int8, (const void *)k_qmodes_w1<2>, (const void *)k_qmodes_w1<3>};
  for (const void *fn : fns) {
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Failure detection without a fault: one thread waits, bounded, on an mbarrier that no
// arrival or copy will ever complete; when the bound runs out it records the same error
// flag a lost TMA copy would, and returns.  The host then reads SG_ETIMEOUT.
__global__ void k_wait_selftest(unsigned long long *ctr, uint32_t max_tries) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, max_tries)) atomicOr(&ctr[CTR_ERROR], ERR_TMA_TIMEOUT);
}

cudaError_t launch_wait_selftest(const Dev &dv, uint32_t max_tries, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(dv.ctr, max_tries);
  return cudaGetLastError();
}

namespace {
unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }
} // namespace

cudaError_t launch_init(const Job &jb, const Dev &dv, bool int8fmt, cudaStream_t st) {
  const long long nplane = (long long)jb.S * jb.g.d * jb.g.NW;
  k_init_couplings<<<blocks_for(nplane, 128), 128, 0, st>>>(jb, dv);
  if (int8fmt) {
    const long long n = (long long)jb.S * jb.C * jb.g.N * (jb.Tp / 4);
    k_init_spins_int8<<<blocks_for(n, 128), 128, 0, st>>>(jb, dv);
  } else {
    const unsigned planes = (unsigned)min(jb.S * jb.W, 65535);
    k_init_spins_packed<<<dim3((unsigned)((jb.g.N + 127) / 128), planes), 128, 0, st>>>(jb, dv);
  }
  k_init_maps<<<blocks_for((long long)jb.S * jb.C * jb.T, 256), 256, 0, st>>>(jb, dv);
  return cudaGetLastError();
}

cudaError_t launch_export_spins(const Job &jb, const Dev &dv, bool int8fmt, uint8_t *out, cudaStream_t st) {
  const long long n = (long long)jb.S * jb.C * jb.T * jb.g.N;
  k_export_spins<<<blocks_for(n, 256), 256, 0, st>>>(jb, dv, int8fmt ? 1 : 0, out);
  return cudaGetLastError();
}

cudaError_t launch_import_spins(const Job &jb, const Dev &dv, bool int8fmt, const uint8_t *in, cudaStream_t st) {
  const long long n = int8fmt ? (long long)jb.S * jb.C * jb.g.N * jb.Tp : (long long)jb.S * jb.W * jb.g.N;
  k_import_spins<<<blocks_for(n, 256), 256, 0, st>>>(jb, dv, int8fmt ? 1 : 0, in);
  return cudaGetLastError();
}

cudaError_t launch_export_couplings(const Job &jb, const Dev &dv, int8_t *out, cudaStream_t st) {
  const long long n = (long long)jb.S * jb.g.N * jb.g.d;
  k_export_couplings<<<blocks_for(n, 256), 256, 0, st>>>(jb, dv, out);
  return cudaGetLastError();
}

cudaError_t launch_import_couplings(const Job &jb, const Dev &dv, const int8_t *in, cudaStream_t st) {
  const long long n = (long long)jb.S * jb.g.d * jb.g.NW;
  k_import_couplings<<<blocks_for(n, 128), 128, 0, st>>>(jb, dv, in);
  return cudaGetLastError();
}

cudaError_t launch_measure(const Job &jb, const Dev &dv, bool int8fmt, int32_t *E_out, int32_t *Q_out,
                           cudaStream_t st) {
  if (!int8fmt && jb.C == 2 && jb.Wc == 1 && Q_out) {
    k_measure_pairs_w1<<<(unsigned)jb.S, MP_NT, 0, st>>>(jb, dv, E_out, Q_out);
    return cudaGetLastError();
  }
  k_gather_energy<<<blocks_for((long long)jb.S * jb.C * jb.T, 256), 256, 0, st>>>(jb, dv, E_out);
  if (Q_out && jb.C >= 2) {
    if (int8fmt) k_overlap_int8<<<(unsigned)(jb.S * jb.T), 256, 0, st>>>(jb, dv, Q_out);
    else {
      const int tl = overlap_tile(jb.W);
      k_overlap_packed<<<(unsigned)(jb.S * ((jb.T + 31) / 32)), OV_NT, (size_t)jb.W * tl * 4, st>>>(jb, dv, tl,
                                                                                                Q_out);
    }
  }
  return cudaGetLastError();
}

} // namespace sgmc
