// sgmc_houd.cuh -- pieces shared by the Houdayer move's kernels (Sec. 2.4, Eq. 10): bit
// operations on one bitmap row of the q = -1 field, the split form's scratch layout, and
// the launcher of the seed-cluster forms (k_houd_seed.cu).
#pragma once
#include "sgmc_internal.cuh"

namespace sgmc {

constexpr uint32_t FULLM = 0xFFFFFFFFu;
constexpr int HFILL_HEAD = 16; // fill kernels' shared-memory header (two counters)

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

// Bitmap block b of a pair (row r = b / RW, x = 32 (b % RW) + l for lane l) as a site:
// the divisions by RW and L1 are multiply-highs with ceil(2^32 / divisor) (division by an
// invariant integer, Granlund and Montgomery), exact while dividend x divisor < 2^32:
// the move is limited to L0 <= 256 (RW <= 8) and R <= 65535 rows, so b RW < 2^22 and
// r L1 <= R^2 < 2^32.
struct BlockMap {
  int RW;
  uint32_t mRW, mL1;
};
__device__ __forceinline__ BlockMap block_map(const Geo &g, int RW) {
  BlockMap bm;
  bm.RW = RW;
  bm.mRW = RW > 1 ? 0xFFFFFFFFu / (uint32_t)RW + 1u : 0u;
  bm.mL1 = g.L1 > 1 ? 0xFFFFFFFFu / (uint32_t)g.L1 + 1u : 0u;
  return bm;
}
// The colour-split index p of block b, lane l; `valid` is false for the padding bits
// past L0.
__device__ __forceinline__ int block_site(const Geo &g, const BlockMap &bm, int b, int l, bool &valid) {
  const int r = bm.RW > 1 ? (int)__umulhi((uint32_t)b, bm.mRW) : b;
  const int x = 32 * (b - r * bm.RW) + l;
  valid = x < g.L0;
  const int z = g.L1 > 1 ? (int)__umulhi((uint32_t)r, bm.mL1) : r;
  const int y = r - z * g.L1;
  const int c = (x + y + z) & 1;
  return c * g.Nh + r * g.H + (x >> 1);
}

// The chain-0 lanes whose pair takes part in the move: a < T at a slot below hK.  A pair
// outside it gets an empty q bitmap, hence M = 0 and no move.  Needs slot0 (phase 0).
__device__ __forceinline__ uint32_t houd_pair_mask(const Job &jb, const int32_t *slot0) {
  const int lane = threadIdx.x & 31;
  return __ballot_sync(FULLM, lane < jb.T && slot0[lane] < jb.hK);
}

struct HoudSplit {
  int RW;        // words per bitmap row
  int NBW;       // words per bitmap
  uint32_t *Qg;  // [S][T][NBW] q bitmaps
  uint32_t *Cg;  // [S][T][NBW] cluster bitmaps
  uint32_t *Mg;  // [S][32] q = -1 sites per pair (by chain-0 lane)
  int wpb;       // pairs (warps) per CTA of the fill kernel
  int in_smem;   // 1: a fill warp copies its bitmaps into shared memory
  unsigned int *queue; // next pair to take (seed-cluster forms), zeroed before each move
};
// The single-cluster move's phase 2 by a seed-cluster fill (k_houd_seed.cu): grows only
// the cluster of each pair's seed into hs.Cg, with the move counters.  *launched is false
// when no fill form applies to this lattice (the caller labels instead).
cudaError_t launch_houd_seed(const Job &jb, const Dev &dv, const HoudSplit &hs, int n_sm, cudaStream_t st,
                             bool *launched);
cudaError_t prepare_houd_seed_kernels(int max_smem);

} // namespace sgmc
