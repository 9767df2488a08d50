// k_global.cu -- the streaming sweep path, for lattices whose word planes do not fit a
// CTA's shared memory.  Same dynamics and decisions as the resident kernel (same Philox
// counters, lane-pair threshold tables and bit-sliced counts), with the lattice read
// from global memory (L2) instead of staged in shared memory:
//   k_pair_tables    one lane-pair threshold table per (sample, word) from the slots
//   k_half_global    one checkerboard half-sweep, a thread per (site of the colour, word);
//                    on colour 1 it also adds each site's post-update unsatisfied-bond
//                    count per replica into a per-(sample, word) scratch sum
//   k_energy_global  E = 2U - dN for every replica, clears the sums, advances t_metro
#include "sgmc_internal.cuh"
#include "sgmc_sweep.cuh"

#include <mutex>

namespace sgmc {

// Scratch of the allocation-free streaming sweep (sg_sweep_streaming_static): the
// lane-pair tables, then the per-replica bond sums, of at most STATIC_SWEEP_ITEMS
// (sample, word) pairs.  A file-scope device array: every GPU that loads the library
// holds it until the process exits, and every call shares it.
static __device__ __align__(256) unsigned char g_sweep_scratch[STATIC_SWEEP_BYTES];

namespace {
std::mutex g_scratch_mutex;
void *g_scratch_ptr[64] = {nullptr};
} // namespace

// Device address of g_sweep_scratch on the current device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress, once per device with that device current, and cached.
cudaError_t static_sweep_scratch(void **ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sweep_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *ptr = g_scratch_ptr[dev];
  return cudaSuccess;
}

__global__ void k_pair_tables(Job jb, Dev dv, uint2 *tables) {
  // one warp per (sample, word): the table of the word's 32 lanes
  const int warp_id = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp_id >= jb.S * jb.W) return;
  const int s = warp_id / jb.W, w = warp_id - s * jb.W;
  const int c = w / jb.Wc, wc = w - c * jb.Wc;
  const int nvalid = min(32, jb.T - wc * 32);
  const size_t cb = ((size_t)s * jb.C + c) * jb.T;
  const int kslot = lane < nvalid ? dv.slot[cb + wc * 32 + lane] : 0;
  if (jb.g.d == 3) fill_pair_table<3>(tables + (size_t)warp_id * 256, lane, kslot, lane < nvalid, dv.thr);
  else fill_pair_table<2>(tables + (size_t)warp_id * 256, lane, kslot, lane < nvalid, dv.thr);
}

template <int D, bool ACCUM, bool NOFLIP>
__global__ void __launch_bounds__(256) k_half_global(Job jb, Dev dv, int col, const uint2 *tables,
                                                     uint32_t *esum) {
  __shared__ int32_t red[8][32];
  const Geo g = jb.g;
  const int sw = blockIdx.y; // (sample, word)
  const int s = sw / jb.W, w = sw - (sw / jb.W) * jb.W;
  const int c = w / jb.Wc, wc = w - c * jb.Wc;
  const int nvalid = min(32, jb.T - wc * 32);
  const uint32_t vmask = nvalid >= 32 ? 0xFFFFFFFFu : ((1u << nvalid) - 1u);
  const int ngroups = (nvalid + 3) >> 2;
  const uint32_t c3base = ((uint32_t)c << 20) | ((uint32_t)(wc * 8) << 8) | TAG_METRO;
  const uint32_t s_glob = (uint32_t)(jb.s_off + s);
  const uint32_t t = (uint32_t)dv.ctr[CTR_TMETRO];
  uint32_t *sp = dv.spins + ((size_t)s * jb.W + w) * g.N;
  const uint32_t *jpl = dv.jbits + (size_t)s * D * g.NW;
  const uint2 *tab = tables + (size_t)sw * 256;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t V[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) V[b] = 0u;
  if (q < g.Nh) {
    const int H = g.H, L1 = g.L1;
    const int row = q / H, k = q - row * H;
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
    const uint32_t *oth = sp + (1 - col) * g.Nh;
    const int p = col * g.Nh + q;
    uint32_t jm[2 * D], nb[2 * D];
#pragma unroll
    for (int mu = 0; mu < D; ++mu) {
      // forward bond (i, mu) at this site; backward bond (i - e_mu, mu) at the neighbour
      const uint32_t *pl = jpl + mu * g.NW;
      const int pb = (1 - col) * g.Nh + nidx[2 * mu + 1];
      jm[2 * mu] = 0u - ((pl[p >> 5] >> (p & 31)) & 1u);
      jm[2 * mu + 1] = 0u - ((pl[pb >> 5] >> (pb & 31)) & 1u);
    }
#pragma unroll
    for (int b = 0; b < 2 * D; ++b) nb[b] = oth[nidx[b]];
    const uint32_t s0 = sp[p];
    const SiteCount<D> cnt = count_site<D>(s0, nb, jm);
    uint32_t F = 0u;
    if (!NOFLIP) {
      const PhiloxSweep P = philox_sweep(s_glob, t, jb);
      const PhiloxSite Q = philox_site(P, (uint32_t)(g.L0 * row + 2 * k + xodd), jb);
      F = decide_site<D>(cnt, P, Q, c3base, ngroups, tab, jb) & vmask;
      sp[p] = s0 ^ F;
    }
    if (ACCUM) {
      uint32_t v1, v2;
      recount<D>(cnt, F, v1, v2);
      vcount_add(V, cnt.u0, v1, v2);
    }
  }
  if (ACCUM) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    red[warp][lane] = warp_lane_sum(V);
    __syncthreads();
    if (warp == 0) {
      int32_t sum = 0;
#pragma unroll
      for (int wq = 0; wq < 8; ++wq) sum += red[wq][lane];
      if (sum) atomicAdd(&esum[(size_t)sw * 32 + lane], (uint32_t)sum);
    }
  }
}

__global__ void k_energy_global(Job jb, Dev dv, uint32_t *esum, unsigned long long adv_metro) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < (long long)jb.S * jb.W * 32) {
    const int lane = (int)(idx & 31);
    const long long sw = idx >> 5;
    const int s = (int)(sw / jb.W), w = (int)(sw % jb.W);
    const int c = w / jb.Wc, wc = w - c * jb.Wc;
    const int j = wc * 32 + lane;
    if (j < jb.T) dv.E[((size_t)s * jb.C + c) * jb.T + j] = 2 * (int32_t)esum[idx] - jb.g.d * jb.g.N;
    esum[idx] = 0u;
  }
  grid_done_advance(dv.ctr, adv_metro, 0ull, 0ull);
}

cudaError_t launch_global_sweep(const Job &jb, const Dev &dv, uint2 *tables, uint32_t *esum, cudaStream_t st) {
  const int warps = jb.S * jb.W;
  k_pair_tables<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(jb, dv, tables);
  const dim3 grid((unsigned)((jb.g.Nh + 255) / 256), (unsigned)(jb.S * jb.W));
  if (jb.g.d == 3) {
    k_half_global<3, false, false><<<grid, 256, 0, st>>>(jb, dv, 0, tables, esum);
    k_half_global<3, true, false><<<grid, 256, 0, st>>>(jb, dv, 1, tables, esum);
  } else {
    k_half_global<2, false, false><<<grid, 256, 0, st>>>(jb, dv, 0, tables, esum);
    k_half_global<2, true, false><<<grid, 256, 0, st>>>(jb, dv, 1, tables, esum);
  }
  const long long n = (long long)jb.S * jb.W * 32;
  k_energy_global<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(jb, dv, esum, 1ull);
  return cudaGetLastError();
}

cudaError_t launch_global_energy(const Job &jb, const Dev &dv, uint2 *tables, uint32_t *esum, cudaStream_t st) {
  const dim3 grid((unsigned)((jb.g.Nh + 255) / 256), (unsigned)(jb.S * jb.W));
  if (jb.g.d == 3) k_half_global<3, true, true><<<grid, 256, 0, st>>>(jb, dv, 1, tables, esum);
  else k_half_global<2, true, true><<<grid, 256, 0, st>>>(jb, dv, 1, tables, esum);
  const long long n = (long long)jb.S * jb.W * 32;
  k_energy_global<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(jb, dv, esum, 0ull);
  return cudaGetLastError();
}

} // namespace sgmc
