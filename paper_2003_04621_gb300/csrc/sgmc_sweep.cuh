// sgmc_sweep.cuh -- the per-site Metropolis machinery shared by the resident and the
// streaming sweep kernels: the bit-sliced unsatisfied-bond count of one site for 32
// replicas, the Philox work shared by a sweep and by a site, the threshold decisions
// through lane-pair tables, and the bit-sliced energy counters.
#pragma once
#include "sgmc_internal.cuh"

#ifndef SGMC_MIN_THREADS
#define SGMC_MIN_THREADS 768 // resident threads per SM the register budget must allow
#endif

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

// Reject-mask accumulation: rej = 2 rej + [r >= thr].  The carry of r - thr is 1 iff
// r >= thr (for thr = 0 always), so the Metropolis test r < thr costs one subtract and
// one add-with-carry, and walking the lanes from high to low leaves lane j's reject bit
// at bit j.
__device__ __forceinline__ uint32_t push_reject(uint32_t rej, uint32_t r, uint32_t thr) {
  uint32_t out;
  asm("{\n\t.reg .u32 t;\n\tsub.cc.u32 t, %1, %2;\n\taddc.u32 %0, %3, %3;\n\t}"
      : "=r"(out)
      : "r"(r), "r"(thr), "r"(rej));
  return out;
}

// 32x32 -> 64-bit product as one wide multiply: (hi, lo).
__device__ __forceinline__ void mulwide(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo) {
  unsigned long long p;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
  lo = (uint32_t)p;
  hi = (uint32_t)(p >> 32);
}

// Per-sweep part of the site counters' Philox calls.  Every call of a sweep has counter
// (i, t, s, c3) with s and t fixed, so round 1's product M1 * s and round 2's product
// M0 * (round-1 word 0) are the same for every site and are computed once.
struct PhiloxSweep {
  uint32_t B;        // round 1 output word 1: lo(M1 s)
  uint32_t hiA, loA; // round 2 product M0 * A, A = hi(M1 s) ^ t ^ k0[0]
};

__device__ __forceinline__ PhiloxSweep philox_sweep(uint32_t s_glob, uint32_t t, const Job &jb) {
  PhiloxSweep P;
  const uint32_t hi1 = __umulhi(PH_M1, s_glob);
  P.B = PH_M1 * s_glob;
  const uint32_t A = hi1 ^ t ^ jb.rk0[0];
  P.hiA = __umulhi(PH_M0, A);
  P.loA = PH_M0 * A;
  return P;
}

// Per-site part: round 1's product M0 * i and round 3's product M1 * (round-2 word 2).
struct PhiloxSite {
  uint32_t X;        // hi(M0 i) ^ k1[0]: round-1 word 2 before the counter's c3 is mixed in
  uint32_t z3;       // round 2 output word 3
  uint32_t hiZ, loZ; // round 3 product M1 * z2
};

__device__ __forceinline__ PhiloxSite philox_site(const PhiloxSweep &P, uint32_t i, const Job &jb) {
  PhiloxSite Q;
  const uint32_t hi0 = __umulhi(PH_M0, i), lo0 = PH_M0 * i;
  Q.X = hi0 ^ jb.rk1[0];
  const uint32_t z2 = P.hiA ^ lo0 ^ jb.rk1[1];
  Q.z3 = P.loA;
  Q.hiZ = __umulhi(PH_M1, z2);
  Q.loZ = PH_M1 * z2;
  return Q;
}

// The rest of one Philox4x32-10 call with counter (i, t, s, c3): rounds 2..10.
__device__ __forceinline__ uint4 philox_finish(const PhiloxSweep &P, const PhiloxSite &Q, uint32_t c3,
                                               const Job &jb) {
  const uint32_t y2 = Q.X ^ c3; // round 1 word 2
  // round 2: products M0 * A (per sweep) and M1 * y2
  uint32_t r2hi, r2lo;
  mulwide(PH_M1, y2, r2hi, r2lo);
  const uint32_t z0 = r2hi ^ P.B ^ jb.rk0[1];
  const uint32_t z1 = r2lo;
  // round 3: products M0 * z0 and M1 * z2 (per site)
  uint32_t p3hi, p3lo;
  mulwide(PH_M0, z0, p3hi, p3lo);
  uint32_t x0 = Q.hiZ ^ z1 ^ jb.rk0[2];
  uint32_t x1 = Q.loZ;
  uint32_t x2 = p3hi ^ Q.z3 ^ jb.rk1[2];
  uint32_t x3 = p3lo;
#pragma unroll
  for (int r = 3; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mulwide(PH_M0, x0, hi0, lo0);
    mulwide(PH_M1, x2, hi1, lo1);
    const uint32_t y0 = hi1 ^ x1 ^ jb.rk0[r];
    const uint32_t yy2 = hi0 ^ x3 ^ jb.rk1[r];
    x0 = y0;
    x1 = lo1;
    x2 = yy2;
    x3 = lo0;
  }
  return make_uint4(x0, x1, x2, x3);
}

// K calls of philox_finish for the groups g0 .. g0 + K - 1 (counters (i, t, s,
// c3base | g << 8)), written round by round so that the K independent chains interleave.
template <int K>
__device__ __forceinline__ void philox_finishK(const PhiloxSweep &P, const PhiloxSite &Q, uint32_t c3base, int g0,
                                               const Job &jb, uint4 (&out)[K]) {
  uint32_t a0[K], a1[K], a2[K], a3[K];
#pragma unroll
  for (int u = 0; u < K; ++u) {
    const uint32_t y = Q.X ^ (c3base | ((uint32_t)(g0 + u) << 8));
    uint32_t h, l;
    mulwide(PH_M1, y, h, l);
    const uint32_t z0 = h ^ P.B ^ jb.rk0[1];
    uint32_t ph, pl;
    mulwide(PH_M0, z0, ph, pl);
    a0[u] = Q.hiZ ^ l ^ jb.rk0[2];
    a1[u] = Q.loZ;
    a2[u] = ph ^ Q.z3 ^ jb.rk1[2];
    a3[u] = pl;
  }
#pragma unroll
  for (int r = 3; r < 10; ++r) {
#pragma unroll
    for (int u = 0; u < K; ++u) {
      uint32_t h0, l0, h1, l1;
      mulwide(PH_M0, a0[u], h0, l0);
      mulwide(PH_M1, a2[u], h1, l1);
      const uint32_t n0 = h1 ^ a1[u] ^ jb.rk0[r], n2 = h0 ^ a3[u] ^ jb.rk1[r];
      a0[u] = n0; a1[u] = l1; a2[u] = n2; a3[u] = l0;
    }
  }
#pragma unroll
  for (int u = 0; u < K; ++u) out[u] = make_uint4(a0[u], a1[u], a2[u], a3[u]);
}

// Bit-sliced unsatisfied-bond count of one site for 32 replicas: the adder planes.
template <int D>
struct SiteCount {
  uint32_t u0, u1, aut;    // u = count (low two bits) and the auto-accept mask (u >= d)
  uint32_t sA, cA, sB, cB; // adder planes, kept to recount after the flip
  uint32_t u2;
};

template <int D>
__device__ __forceinline__ SiteCount<D> count_site(uint32_t s0, const uint32_t *nb, const uint32_t *jm) {
  SiteCount<D> r;
  const uint32_t x0 = s0 ^ nb[0] ^ jm[0];
  const uint32_t x1 = s0 ^ nb[1] ^ jm[1];
  const uint32_t x2 = s0 ^ nb[2] ^ jm[2];
  const uint32_t x3 = s0 ^ nb[3] ^ jm[3];
  fadd(x0, x1, x2, r.sA, r.cA);
  if (D == 3) {
    const uint32_t x4 = s0 ^ nb[4] ^ jm[4];
    const uint32_t x5 = s0 ^ nb[5] ^ jm[5];
    fadd(x3, x4, x5, r.sB, r.cB);
    r.u0 = r.sA ^ r.sB;
    const uint32_t tt = r.sA & r.sB;
    fadd(r.cA, r.cB, tt, r.u1, r.u2);
    r.aut = r.u2 | (r.u1 & r.u0); // u >= 3
  } else {
    r.sB = x3;
    r.cB = 0u;
    r.u0 = r.sA ^ x3;
    const uint32_t tt = r.sA & x3;
    r.u1 = r.cA ^ tt;
    r.u2 = r.cA & tt;
    r.aut = r.u1 | r.u2; // u >= 2
  }
  return r;
}

// Post-flip count planes (v1, v2) of the site: flipping s_i toggles all its bonds, so
// every adder input, sum and carry plane is toggled by F; the low bit is unchanged.
template <int D>
__device__ __forceinline__ void recount(const SiteCount<D> &c, uint32_t F, uint32_t &v1, uint32_t &v2) {
  if (D == 3) {
    fadd(c.cA ^ F, c.cB ^ F, (c.sA ^ F) & (c.sB ^ F), v1, v2);
  } else {
    const uint32_t tt2 = (c.sA ^ F) & (c.sB ^ F);
    v1 = (c.cA ^ F) ^ tt2;
    v2 = (c.cA ^ F) & tt2;
  }
}

// The reject bits of one group of four lanes (4 gi .. 4 gi + 3) pushed onto rej, highest
// lane first: their thresholds come from the lane-pair tables (see decide_site).
template <int D>
__device__ __forceinline__ uint32_t decide_group(uint32_t rej, const uint4 &r, int gi, const SiteCount<D> &cnt,
                                                 const uint2 *__restrict__ pair_tab) {
  uint2 th[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int pp = 2 * gi + h; // lanes 2pp, 2pp+1
    // byte offset = 8 * code, code = (u0 >> 2pp) & 3 | ((u1 >> 2pp) & 3) << 2
    const int s0 = 2 * pp - 3, s1 = 2 * pp - 5;
    const uint32_t a0 = s0 >= 0 ? (cnt.u0 >> s0) : (cnt.u0 << (-s0));
    const uint32_t a1 = s1 >= 0 ? (cnt.u1 >> s1) : (cnt.u1 << (-s1));
    const uint32_t off = (a0 & 0x18u) | (a1 & 0x60u);
    th[h] = *reinterpret_cast<const uint2 *>(reinterpret_cast<const char *>(pair_tab) + pp * 128 + off);
  }
  rej = push_reject(rej, r.w, th[1].y);
  rej = push_reject(rej, r.z, th[1].x);
  rej = push_reject(rej, r.y, th[0].y);
  rej = push_reject(rej, r.x, th[0].x);
  return rej;
}

// Metropolis decisions of one site's 32 replicas: returns the accepted-flip mask.  The
// groups of 4 replicas draw their words in interleaved Philox evaluations: a full word's
// eight in one, a partial word's (ngroups of 8 in use, the rest masked) in blocks of four,
// two or one, so that a partial word costs about its share of a full one (the block of
// groups 0..3 drops the word of group 3 when only three are in use).  The reject bits are pushed
// highest group first; the masked groups at the top leave zeros, excluded by vmask.
// pair_tab holds, for each pair of lanes (2p, 2p+1) and each 4-bit code
// (u0_2p, u0_2p+1, u1_2p, u1_2p+1), the two lanes' thresholds for their counts u
// (m = d - u), 8 bytes per entry: one 64-bit load serves two lanes, and the code is
// cut from the count planes with two shifts and one three-input logic op.
// FULLW: the caller guarantees full words (every chain a multiple of 32 replicas), so the
// partial-word code is left out and cannot take registers from the full-word path.
template <int D, bool FULLW = false>
__device__ __forceinline__ uint32_t decide_site(const SiteCount<D> &cnt, const PhiloxSweep &P,
                                                const PhiloxSite &Q, uint32_t c3base, int ngroups,
                                                const uint2 *__restrict__ pair_tab, const Job &jb) {
  uint32_t rej = 0;
  if (FULLW || ngroups == 8) { // a full word: all eight groups in one interleaved evaluation
    uint4 rr[8];
    philox_finishK<8>(P, Q, c3base, 0, jb, rr);
#pragma unroll
    for (int u = 7; u >= 0; --u) rej = decide_group<D>(rej, rr[u], u, cnt, pair_tab);
    return cnt.aut | ~rej;
  }
  if (ngroups > 4) { // groups 4 .. ngroups - 1 first (the higher ones)
    if (ngroups == 7) {
      uint4 rc[1];
      philox_finishK<1>(P, Q, c3base, 6, jb, rc);
      rej = decide_group<D>(rej, rc[0], 6, cnt, pair_tab);
    }
    if (ngroups >= 6) {
      uint4 rb[2];
      philox_finishK<2>(P, Q, c3base, 4, jb, rb);
      rej = decide_group<D>(rej, rb[1], 5, cnt, pair_tab);
      rej = decide_group<D>(rej, rb[0], 4, cnt, pair_tab);
    } else {
      uint4 rb[1];
      philox_finishK<1>(P, Q, c3base, 4, jb, rb);
      rej = decide_group<D>(rej, rb[0], 4, cnt, pair_tab);
    }
  }
  if (ngroups >= 3) { // groups 0..3 (group 3 dropped when only three are in use)
    uint4 ra[4];
    philox_finishK<4>(P, Q, c3base, 0, jb, ra);
    if (ngroups >= 4) rej = decide_group<D>(rej, ra[3], 3, cnt, pair_tab);
    rej = decide_group<D>(rej, ra[2], 2, cnt, pair_tab);
    rej = decide_group<D>(rej, ra[1], 1, cnt, pair_tab);
    rej = decide_group<D>(rej, ra[0], 0, cnt, pair_tab);
  } else if (ngroups == 2) {
    uint4 ra[2];
    philox_finishK<2>(P, Q, c3base, 0, jb, ra);
    rej = decide_group<D>(rej, ra[1], 1, cnt, pair_tab);
    rej = decide_group<D>(rej, ra[0], 0, cnt, pair_tab);
  } else {
    uint4 ra[1];
    philox_finishK<1>(P, Q, c3base, 0, jb, ra);
    rej = decide_group<D>(rej, ra[0], 0, cnt, pair_tab);
  }
  return cnt.aut | ~rej;
}

// K calls for each of two counter bases, interleaved round by round (2K chains): out[u] is
// the call with c3 = c3lo | u << 8 and out[K + u] the one with c3hi | u << 8, u < K.
template <int K>
__device__ __forceinline__ void philox_finish2K(const PhiloxSweep &P, const PhiloxSite &Q, uint32_t c3lo,
                                                uint32_t c3hi, const Job &jb, uint4 (&out)[2 * K]) {
  uint32_t a0[2 * K], a1[2 * K], a2[2 * K], a3[2 * K];
#pragma unroll
  for (int u = 0; u < 2 * K; ++u) {
    const uint32_t c3 = (u < K ? c3lo : c3hi) | ((uint32_t)(u < K ? u : u - K) << 8);
    const uint32_t y = Q.X ^ c3;
    uint32_t h, l;
    mulwide(PH_M1, y, h, l);
    const uint32_t z0 = h ^ P.B ^ jb.rk0[1];
    uint32_t ph, pl;
    mulwide(PH_M0, z0, ph, pl);
    a0[u] = Q.hiZ ^ l ^ jb.rk0[2];
    a1[u] = Q.loZ;
    a2[u] = ph ^ Q.z3 ^ jb.rk1[2];
    a3[u] = pl;
  }
#pragma unroll
  for (int r = 3; r < 10; ++r) {
#pragma unroll
    for (int u = 0; u < 2 * K; ++u) {
      uint32_t h0, l0, h1, l1;
      mulwide(PH_M0, a0[u], h0, l0);
      mulwide(PH_M1, a2[u], h1, l1);
      const uint32_t n0 = h1 ^ a1[u] ^ jb.rk0[r], n2 = h0 ^ a3[u] ^ jb.rk1[r];
      a0[u] = n0; a1[u] = l1; a2[u] = n2; a3[u] = l0;
    }
  }
#pragma unroll
  for (int u = 0; u < 2 * K; ++u) out[u] = make_uint4(a0[u], a1[u], a2[u], a3[u]);
}

// Metropolis decisions of a paired word: lanes 0..15 hold replicas of chain 0 and lanes
// 16..31 the same replicas of chain 1 (the two chains' last, partial words), each half
// with K groups of 4 in use.  Group u < 4 draws chain 0's word with c3 = c3lo | u << 8,
// group 4 + u chain 1's with c3lo | 1 << 20 | u << 8: exactly the words the two
// unpaired partial words would draw.  Returns the accepted-flip mask.
template <int D, int K>
__device__ __forceinline__ uint32_t decide_pair_k(const SiteCount<D> &cnt, const PhiloxSweep &P,
                                                  const PhiloxSite &Q, uint32_t c3lo,
                                                  const uint2 *__restrict__ pair_tab, const Job &jb) {
  uint4 rr[2 * K];
  philox_finish2K<K>(P, Q, c3lo, c3lo | (1u << 20), jb, rr);
  uint32_t rej = 0;
#pragma unroll
  for (int u = 7; u >= 4; --u) {
    if (u - 4 < K) rej = decide_group<D>(rej, rr[K + u - 4], u, cnt, pair_tab);
    else rej <<= 4;
  }
#pragma unroll
  for (int u = 3; u >= 0; --u) {
    if (u < K) rej = decide_group<D>(rej, rr[u], u, cnt, pair_tab);
    else rej <<= 4;
  }
  return cnt.aut | ~rej;
}

template <int D>
__device__ __forceinline__ uint32_t decide_pair(const SiteCount<D> &cnt, const PhiloxSweep &P,
                                                const PhiloxSite &Q, uint32_t c3lo, int ngroups,
                                                const uint2 *__restrict__ pair_tab, const Job &jb) {
  switch (ngroups) {
  case 1: return decide_pair_k<D, 1>(cnt, P, Q, c3lo, pair_tab, jb);
  case 2: return decide_pair_k<D, 2>(cnt, P, Q, c3lo, pair_tab, jb);
  case 3: return decide_pair_k<D, 3>(cnt, P, Q, c3lo, pair_tab, jb);
  default: return decide_pair_k<D, 4>(cnt, P, Q, c3lo, pair_tab, jb);
  }
}

// Fill the pair tables of one word from its lanes' temperature slots (one warp; lane
// j's slot in kslot).  Entry (pair p, code) = (thr of lane 2p for u = u0a + 2 u1a,
// thr of lane 2p+1 for u = u0b + 2 u1b), code = u0a | u0b << 1 | u1a << 2 | u1b << 3.
// In 2D only the low bit of u selects (u >= 2 is auto-accepted).
template <int D>
__device__ __forceinline__ void fill_pair_table(uint2 *pair_tab, int lane, int kslot, bool valid,
                                                const uint32_t *thr) {
  // this lane's four thresholds by u = 0..3 (m = d - u for u < d; 0 otherwise or for a
  // lane that holds no replica)
  uint32_t mine[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) mine[u] = (valid && u < D) ? thr[kslot * 4 + (D - u)] : 0u;
  // 256 entries: lane handles pair (lane / 2) ... every (pair, code) via shuffles
#pragma unroll
  for (int rep = 0; rep < 8; ++rep) {
    const int e = rep * 32 + lane;  // entry index 0..255
    const int pp = e >> 4, code = e & 15;
    const int ua = D == 3 ? ((code & 1) | ((code >> 1) & 2)) : (code & 1);
    const int ub = D == 3 ? (((code >> 1) & 1) | ((code >> 2) & 2)) : ((code >> 1) & 1);
    uint32_t ta = 0, tb = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t va = __shfl_sync(FULL, mine[u], 2 * pp);
      const uint32_t vb = __shfl_sync(FULL, mine[u], 2 * pp + 1);
      if (ua == u) ta = va;
      if (ub == u) tb = vb;
    }
    pair_tab[pp * 16 + code] = make_uint2(ta, tb);
  }
}

} // namespace sgmc
