// k_probe.cu -- the sweep's Philox ceiling, measured.
//
// The packed sweep draws one Philox4x32-10 word per attempt (Sec. 3: counter-based
// generators), and those draws are the bulk of its integer work.  This probe runs the
// same Philox work a sweep thread does -- per sweep the rounds shared by every call,
// per site the rounds shared by the site's calls, then for each of two 32-replica words
// the eight calls of the word interleaved round by round -- and nothing else: no lattice,
// no couplings, no counts, no decisions.  Its words per ns therefore bound the sweep's
// attempts per ns from above, on the same launch shape (256 threads, three CTAs per SM).
// Every word is folded into one register and a thread stores it only if it equals a
// value passed in, so no call is optimised away.
#include "sgmc.h"
#include "sgmc_internal.cuh"
#include "sgmc_sweep.cuh"

namespace sgmc {

namespace {

constexpr int PROBE_NT = 256;
constexpr int PROBE_WPC = 2;

__global__ void __launch_bounds__(PROBE_NT, SGMC_MIN_THREADS / PROBE_NT)
    k_probe_philox(const __grid_constant__ Job jb, int n_sites, int n_sweeps, uint32_t sentinel, uint32_t *out) {
  uint32_t acc = 0u;
  const int stride = (int)gridDim.x * PROBE_NT;
  for (int swp = 0; swp < n_sweeps; ++swp) {
    const PhiloxSweep P = philox_sweep((uint32_t)blockIdx.x, (uint32_t)swp, jb);
    for (int i = (int)blockIdx.x * PROBE_NT + (int)threadIdx.x; i < n_sites; i += stride) {
      const PhiloxSite Q = philox_site(P, (uint32_t)i, jb);
#pragma unroll
      for (int w = 0; w < PROBE_WPC; ++w) {
        uint4 rr[8];
        philox_finishK<8>(P, Q, ((uint32_t)w << 20) | TAG_METRO, 0, jb, rr);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc ^= rr[u].x ^ rr[u].y ^ rr[u].z ^ rr[u].w;
      }
    }
  }
  if (acc == sentinel) out[blockIdx.x * PROBE_NT + threadIdx.x] = acc;
}

} // namespace

} // namespace sgmc

extern "C" sg_status sg_probe_philox(int32_t n_sites, int32_t n_sweeps, int32_t n_blocks, uint64_t sim_seed,
                                     uint32_t *out, uintptr_t stream) {
  using namespace sgmc;
  if (n_sites < 1 || n_sweeps < 1 || n_blocks < 1 || !out) return SG_EINVAL;
  Job jb = {};
  jb.sk0 = (uint32_t)(sim_seed & 0xFFFFFFFFu);
  jb.sk1 = (uint32_t)(sim_seed >> 32);
  for (int r = 0; r < 10; ++r) {
    jb.rk0[r] = jb.sk0 + (uint32_t)r * PH_W0;
    jb.rk1[r] = jb.sk1 + (uint32_t)r * PH_W1;
  }
  k_probe_philox<<<(unsigned)n_blocks, PROBE_NT, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      jb, n_sites, n_sweeps, 0x9E3779B9u, out);
  return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ECUDA;
}
