// k_metro_pair.cu -- the resident sweep kernel's instantiations that hold a whole sample
// per CTA with the two chains' partial last words paired in one word (PAIR in
// sgmc_resident.cuh), and the host-side rule for when they apply.  Each chain's replicas
// draw the same Philox words and take the same decisions as in the unpaired kernel
// (Sec. 2.2 / 2.4 step 1, Eq. 5 for the fused exchange); only the per-site work of one
// word is saved.
#include "sgmc_resident.cuh"

namespace sgmc {

namespace {

template <int D, int WPC, int MAXJ>
void (*pick_pair_nt(int nt))(ResidentParams<MAXJ>) {
  switch (nt) {
  case 64: return WPC == 1 ? k_resident_packed<D, 64, 1, false, MAXJ, false, false, 0, true> : nullptr;
  case 128: return k_resident_packed<D, 128, WPC, false, MAXJ, false, false, 0, true>;
  case 256: return k_resident_packed<D, 256, WPC, false, MAXJ, false, false, 0, true>;
  case 512: return k_resident_packed<D, 512, WPC, false, MAXJ, false, false, 0, true>;
  case 1024: return k_resident_packed<D, 1024, WPC, false, MAXJ, false, false, 0, true>;
  default: return nullptr;
  }
}

template <int MAXJ>
void (*pick_pair(int d, int nt, int wpc))(ResidentParams<MAXJ>) {
  if (d == 2) return wpc == 1 ? pick_pair_nt<2, 1, MAXJ>(nt) : pick_pair_nt<2, 3, MAXJ>(nt);
  return wpc == 1 ? pick_pair_nt<3, 1, MAXJ>(nt) : pick_pair_nt<3, 3, MAXJ>(nt);
}

} // namespace

int pair_words(const Job &jb, int *nthreads, int smem_limit, size_t *smem) {
  if (jb.C != 2) return 0;
  int wpc = 0;
  if (jb.Wc == 1 && jb.T <= 16) wpc = 1;
  else if (jb.Wc == 2 && jb.T <= 48) wpc = 3;
  if (!wpc) return 0;
  int nt = *nthreads;
  if (wpc == 3 && nt < 128) nt = 128; // a warp per word
  if (nt != 64 && nt != 128 && nt != 256 && nt != 512 && nt != 1024) return 0;
  const int per_thread = (jb.g.Nh + nt - 1) / nt; // the energy counters hold 8 bit planes
  if (per_thread * 2 * jb.g.d > 255) return 0;
  const PackedSmem L = packed_smem(jb.g.N, jb.g.NW, jb.g.d, nt, wpc, 2);
  if (L.total > smem_limit) return 0;
  *nthreads = nt;
  *smem = (size_t)L.total;
  return wpc;
}

resident_fn1 pair_kernel_1(int d, int nthreads, int wpc) { return pick_pair<1>(d, nthreads, wpc); }
resident_fnB pair_kernel_batch(int d, int nthreads, int wpc) { return pick_pair<MAX_BATCH_JOBS>(d, nthreads, wpc); }

cudaError_t prepare_pair_kernels(int max_smem) {
  for (int d = 2; d <= 3; ++d)
    for (int nt : {64, 128, 256, 512, 1024})
      for (int wpc : {1, 3})
        for (const void *fn : {(const void *)pick_pair<1>(d, nt, wpc), (const void *)pick_pair<MAX_BATCH_JOBS>(d, nt, wpc)}) {
          if (!fn) continue;
          cudaFuncAttributes fa;
          cudaError_t e = cudaFuncGetAttributes(&fa, fn);
          if (e != cudaSuccess) return e;
          e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - (int)fa.sharedSizeBytes);
          if (e != cudaSuccess) return e;
        }
  return cudaSuccess;
}

} // namespace sgmc
