// k_state.cu -- creation (Eq. 2 couplings, hot start), import/export of spins and
// couplings in plain layouts, and the measurement of E by slot and N q (Eqs. 3-4).
#include "sgmc_internal.cuh"

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
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)jb.S * jb.W * g.N) return;
  const int p = (int)(idx % g.N);
  const int w = (int)((idx / g.N) % jb.W);
  const int s = (int)(idx / ((long long)g.N * jb.W));
  const int c = w / jb.Wc, wc = w - c * jb.Wc;
  const int nvalid = min(32, jb.T - wc * 32);
  const uint32_t i = (uint32_t)canonical_of(g, site_geo(g, p));
  uint32_t word = 0;
  for (int gi = 0; gi * 4 < nvalid; ++gi) {
    const uint32_t c3 = ((uint32_t)c << 20) | ((uint32_t)(wc * 8 + gi) << 8) | TAG_INIT;
    const uint4 r = philox10(i, 0u, (uint32_t)(jb.s_off + s), c3, jb.sk0, jb.sk1);
    for (int q = 0; q < 4; ++q)
      if (gi * 4 + q < nvalid) word |= (word_of(r, q) >> 31) << (gi * 4 + q);
  }
  dv.spins[idx] = word;
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

// N q (Eq. 4) per (sample, slot): CTA per (sample, slot); q = -1 sites are those where
// the chain-0 and chain-1 replicas at the slot differ.
__global__ void k_overlap(Job jb, Dev dv, int int8fmt, int32_t *Q_out) {
  const Geo g = jb.g;
  const int s = blockIdx.x / jb.T;
  const int k = blockIdx.x - s * jb.T;
  const int a = dv.perm[((size_t)s * jb.C + 0) * jb.T + k];
  const int b = dv.perm[((size_t)s * jb.C + 1) * jb.T + k];
  int cnt = 0;
  if (int8fmt) {
    const int8_t *sp = reinterpret_cast<const int8_t *>(dv.spins);
    const int8_t *pa = sp + ((size_t)s * jb.C + 0) * g.N * jb.Tp + a;
    const int8_t *pb = sp + ((size_t)s * jb.C + 1) * g.N * jb.Tp + b;
    for (int p = threadIdx.x; p < g.N; p += blockDim.x) cnt += pa[(size_t)p * jb.Tp] != pb[(size_t)p * jb.Tp];
  } else {
    const uint32_t *wa = dv.spins + ((size_t)s * jb.W + 0 * jb.Wc + a / 32) * g.N;
    const uint32_t *wb = dv.spins + ((size_t)s * jb.W + 1 * jb.Wc + b / 32) * g.N;
    const int la = a & 31, lb = b & 31;
    for (int p = threadIdx.x; p < g.N; p += blockDim.x) cnt += ((wa[p] >> la) ^ (wb[p] >> lb)) & 1u;
  }
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
    const long long n = (long long)jb.S * jb.W * jb.g.N;
    k_init_spins_packed<<<blocks_for(n, 128), 128, 0, st>>>(jb, dv);
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
  k_gather_energy<<<blocks_for((long long)jb.S * jb.C * jb.T, 256), 256, 0, st>>>(jb, dv, E_out);
  if (Q_out && jb.C >= 2) k_overlap<<<(unsigned)(jb.S * jb.T), 256, 0, st>>>(jb, dv, int8fmt ? 1 : 0, Q_out);
  return cudaGetLastError();
}

} // namespace sgmc
