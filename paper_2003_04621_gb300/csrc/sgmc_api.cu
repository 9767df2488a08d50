// sgmc_api.cu -- host side of the C-ABI declared in include/sgmc.h: parameter checks,
// the device-memory layout inside the caller's buffer, the host-computed tables
// (Metropolis thresholds, inverse temperatures) and the kernel launches.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "sgmc.h"
#include "sgmc_internal.cuh"

using namespace sgmc;

namespace {

struct Layout {
  size_t spins, jbits, E, perm, slot, thr, beta, ctr, meas_E, meas_Q, meas_P, gtab, esum, houd, houd_bytes;
  size_t trip_dir, trip_t0, trip_n, trip_sum, jfix, E64, meas_E64, jstage, total;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int MAX_TEMPS = 4096;
constexpr long long MAX_SITES = 1ll << 26;

} // namespace

struct sg_handle {
  sg_params p;
  std::vector<double> temps, beta;
  std::vector<uint32_t> thr; // [T][4]
  Job job;
  Dev dev;
  Layout lay;
  char *buf;
  size_t bytes;
  uint64_t t_metro, t_pt, t_houd;
  sg_status sticky;
  int int8fmt;
  int nt;          // threads of the resident kernel
  int wpc;         // 32-replica words per CTA of the packed resident kernel
  size_t smem;     // its dynamic shared memory
  bool fuse_pt;    // the exchange can run inside the resident kernel
  bool pair_on;    // fused MCS may pair the chains' partial last words (sg_set_pairing)
  bool global;     // sweeps stream the lattice from global memory (no resident kernel)
  bool gauss;      // general fixed-point couplings (k_gauss.cu)
  int n_ctr;       // counters in the device array
  // sg_measure_async: device-to-host copies on a copy stream of the handle, from two
  // alternating staging slots (created at the first asynchronous measurement)
  cudaStream_t cst = nullptr;
  cudaEvent_t ev_ready[2] = {nullptr, nullptr}; // slot's observables written (caller's stream)
  cudaEvent_t ev_done[2] = {nullptr, nullptr};  // slot's copies finished (copy stream)
  bool slot_used[2] = {false, false};
  int mslot = 0;
  ~sg_handle() {
    if (cst) { // copies still in flight read the caller's buffer: let them finish first
      cudaStreamSynchronize(cst);
      cudaStreamDestroy(cst);
    }
    for (int i = 0; i < 2; ++i) {
      if (ev_ready[i]) cudaEventDestroy(ev_ready[i]);
      if (ev_done[i]) cudaEventDestroy(ev_done[i]);
    }
  }
};

namespace {

sg_status validate(const sg_params *p) {
  if (!p) return SG_EINVAL;
  if (p->ndim != 2 && p->ndim != 3) return SG_EINVAL;
  long long N = 1;
  for (int a = 0; a < p->ndim; ++a) {
    if (p->dims[a] < 2) return SG_EINVAL;
    N *= p->dims[a];
    if (N > MAX_SITES) return SG_EUNSUPPORTED;
  }
  if (p->n_samples < 1 || p->sample_offset < 0) return SG_EINVAL;
  if (p->n_chains != 1 && p->n_chains != 2) return SG_EINVAL;
  if (p->n_temps < 1 || p->n_temps > MAX_TEMPS || !p->temps) return SG_EINVAL;
  for (int k = 0; k < p->n_temps; ++k) {
    if (!(p->temps[k] > 0.0) || !std::isfinite(p->temps[k])) return SG_EINVAL;
    if (k > 0 && !(p->temps[k] > p->temps[k - 1])) return SG_EINVAL;
  }
  if (!(p->p_plus >= 0.0 && p->p_plus <= 1.0)) return SG_EINVAL;
  if (p->spin_format != SG_PACKED32 && p->spin_format != SG_INT8) return SG_EINVAL;
  if (p->houdayer < 0 || p->houdayer > 2) return SG_EINVAL;
  if (p->houdayer && p->n_chains != 2) return SG_EINVAL;
  if (p->n_metro < 1 || (p->track_trips != 0 && p->track_trips != 1)) return SG_EINVAL;
  if (p->coupling_kind != SG_COUPLINGS_PM && p->coupling_kind != SG_COUPLINGS_FIXED) return SG_EINVAL;
  if (p->houdayer_slots < 0 || p->houdayer_slots > p->n_temps) return SG_EINVAL;
  // general couplings: int8 spins (one replica per byte), no cluster move
  if (p->coupling_kind == SG_COUPLINGS_FIXED && (p->spin_format != SG_INT8 || p->houdayer != 0))
    return SG_EUNSUPPORTED;
  for (int a = 0; a < p->ndim; ++a)
    if (p->dims[a] % 2) return SG_EUNSUPPORTED; // checkerboard needs even extents
  return SG_OK;
}

void build_job(const sg_params *p, Job *jb) {
  Geo &g = jb->g;
  g.d = p->ndim;
  g.L0 = p->dims[0];
  g.L1 = p->dims[1];
  g.L2 = p->ndim == 3 ? p->dims[2] : 1;
  g.N = g.L0 * g.L1 * g.L2;
  g.H = g.L0 / 2;
  g.R = g.L1 * g.L2;
  g.Nh = g.N / 2;
  g.NW = (((g.N + 31) / 32) + 3) & ~3; // multiple of 4 words: 16-byte aligned planes
  jb->S = p->n_samples;
  jb->s_off = p->sample_offset;
  jb->C = p->n_chains;
  jb->T = p->n_temps;
  jb->Wc = (p->n_temps + 31) / 32;
  jb->W = jb->C * jb->Wc;
  jb->Tp = (p->n_temps + 3) & ~3;
  jb->hK = p->houdayer_slots > 0 ? p->houdayer_slots : p->n_temps;
  jb->sk0 = (uint32_t)(p->sim_seed & 0xFFFFFFFFu);
  jb->sk1 = (uint32_t)(p->sim_seed >> 32);
  jb->ck0 = (uint32_t)(p->coupling_seed & 0xFFFFFFFFu);
  jb->ck1 = (uint32_t)(p->coupling_seed >> 32);
  for (int r = 0; r < 10; ++r) {
    jb->rk0[r] = jb->sk0 + (uint32_t)r * PH_W0;
    jb->rk1[r] = jb->sk1 + (uint32_t)r * PH_W1;
  }
  double cut = std::floor(std::ldexp(p->p_plus, 32));
  if (cut < 0.0) cut = 0.0;
  if (cut > 4294967296.0) cut = 4294967296.0;
  jb->jcut = (unsigned long long)cut;
}

// The Houdayer kernel pairs lanes of one chain-0 and one chain-1 word: packed spins, two
// chains, at most 32 temperatures, rows of at most 256 sites.
bool houdayer_possible(const sg_params *p, const Job &jb) {
  return p->spin_format == SG_PACKED32 && jb.C == 2 && jb.Wc == 1 && jb.g.L0 <= 256 && jb.g.R <= 65535;
}

Layout layout_of(const sg_params *p, const Job &jb) {
  const Geo &g = jb.g;
  const size_t S = (size_t)jb.S, C = (size_t)jb.C, T = (size_t)jb.T, N = (size_t)g.N;
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  const size_t spin_bytes = p->spin_format == SG_INT8 ? S * C * N * (size_t)jb.Tp : S * (size_t)jb.W * N * 4;
  L.spins = take(spin_bytes);
  L.jbits = take(S * (size_t)g.d * (size_t)g.NW * 4);
  L.E = take(S * C * T * 4);
  L.perm = take(S * C * T * 4);
  L.slot = take(S * C * T * 4);
  L.thr = take(T * 4 * 4);
  L.beta = take(T * 8);
  L.ctr = take((size_t)(CTR_PT + T) * 8);
  L.meas_E = take(2 * S * C * T * 4); // two staging slots (asynchronous measurements)
  L.meas_Q = take(2 * S * T * 4);
  L.meas_P = take(C >= 2 ? S * T * (size_t)g.d * (size_t)qmodes_lmax(jb) * 4 : 0);
  // streaming sweep path: lane-pair threshold tables and per-replica bond sums
  L.gtab = take(S * (size_t)jb.W * 256 * 8);
  L.esum = take(S * (size_t)jb.W * 32 * 4);
  // Houdayer bitmap scratch of the split move: for jobs that make the move every MCS, and
  // for lattices whose bitmaps exceed the single-CTA kernel's shared-memory budget
  L.houd_bytes = 0;
  if (houdayer_possible(p, jb) && (p->houdayer || houdayer_smem(jb, 1) > HOUD_SMEM_BUDGET))
    L.houd_bytes = houdayer_scratch_bytes(jb);
  L.houd = take(L.houd_bytes);
  // round trips in temperature, when tracked
  const size_t tr = p->track_trips ? 1 : 0;
  L.trip_dir = take(tr * S * C * T * 4);
  L.trip_t0 = take(tr * S * C * T * 4);
  L.trip_n = take(tr * S * C * 4);
  L.trip_sum = take(tr * S * C * 8);
  // general couplings: device and staging couplings, int64 energies
  const size_t gk = p->coupling_kind == SG_COUPLINGS_FIXED ? 1 : 0;
  L.jfix = take(gk * S * (size_t)g.d * N * 4);
  L.E64 = take(gk * S * C * T * 8);
  L.meas_E64 = take(gk * S * C * T * 8);
  L.jstage = take(gk * S * N * (size_t)g.d * 4);
  L.total = off;
  return L;
}

uint32_t metropolis_threshold(double beta, int dE) {
  const double v = std::floor(std::ldexp(std::exp(-(beta * (double)dE)), 32));
  return v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
}

int max_dyn_smem() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  return v;
}

// Once per device: allow the kernels the opt-in shared memory (outside any capture).
std::mutex prep_mutex;
bool prepared[64] = {false};
cudaError_t prepare_device() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(prep_mutex);
  if (dev < 64 && prepared[dev]) return cudaSuccess;
  const int ms = max_dyn_smem();
  e = prepare_resident_kernels(ms);
  if (e == cudaSuccess) e = prepare_houdayer_kernels(ms);
  if (e == cudaSuccess) e = prepare_state_kernels(ms);
  if (e == cudaSuccess) e = prepare_gauss_kernels(ms);
  if (e == cudaSuccess && dev < 64) prepared[dev] = true;
  return e;
}

// Whether the packed resident kernel can run with this shape: the per-thread colour-1
// sites must keep the 8-plane vertical counter below 256, the words per CTA must divide
// the sample's words, and the lattice must fit in shared memory.
bool packed_shape_ok(const sg_handle *h, int nt, int wpc, int smem_limit, size_t *smem) {
  const Geo &g = h->job.g;
  if (nt != 64 && nt != 128 && nt != 256 && nt != 512 && nt != 1024) return false;
  if (wpc != 1 && wpc != 2) return false;
  if (h->job.W % wpc) return false;
  const int per_thread = (g.Nh + nt - 1) / nt;
  if (per_thread * 2 * g.d > 255) return false;
  const PackedSmem L = packed_smem(g.N, g.NW, g.d, nt, wpc);
  if (L.total > smem_limit) return false;
  *smem = (size_t)L.total;
  return true;
}

// Choose the resident kernel's default shape: two words per CTA (one sample's two
// chains) when two such CTAs fit on an SM, else one; the smallest CTA of 256/512/1024
// threads whose counters do not overflow.
bool choose_resident(sg_handle *h, int smem_limit) {
  const Geo &g = h->job.g;
  if (h->int8fmt) {
    const Int8Smem L = int8_smem(g.N, g.NW, g.d, h->job.T, h->job.Tp);
    h->nt = 256;
    h->wpc = 1;
    h->smem = (size_t)L.total;
    return L.total <= smem_limit;
  }
  // two words per CTA (one sample's two chains) when they fit: the site geometry, the
  // couplings and the site-level Philox work are then shared by 64 replicas
  for (int wpc : {2, 1}) {
    for (int nt : {256, 512, 1024}) {
      size_t sm = 0;
      if (!packed_shape_ok(h, nt, wpc, wpc == 2 ? smem_limit / 2 : smem_limit, &sm)) continue;
      h->nt = nt;
      h->wpc = wpc;
      h->smem = sm;
      return true;
    }
  }
  return false;
}

sg_status check(sg_handle *h, cudaError_t e) {
  if (e != cudaSuccess) {
    h->sticky = SG_ECUDA;
    return SG_ECUDA;
  }
  return SG_OK;
}

template <bool FUSE, bool EONLY>
sg_status launch_resident(sg_handle *h, cudaStream_t st, int n_mcs, int n_metro) {
  if (h->gauss) return check(h, sgmc::launch_gauss(h->job, h->dev, FUSE, EONLY, st, n_mcs, n_metro));
  return check(h, sgmc::launch_resident(h->job, h->dev, h->int8fmt != 0, h->nt, h->wpc, FUSE, EONLY, h->smem, st,
                                        n_mcs, n_metro, nullptr, nullptr, false, nullptr, 0,
                                        FUSE && !EONLY && h->pair_on));
}

cudaStream_t as_stream(uintptr_t s) { return reinterpret_cast<cudaStream_t>(s); }

uint2 *gtab_of(sg_handle *h) { return reinterpret_cast<uint2 *>(h->buf + h->lay.gtab); }
uint32_t *esum_of(sg_handle *h) { return reinterpret_cast<uint32_t *>(h->buf + h->lay.esum); }

sg_status sweeps(sg_handle *h, int n, cudaStream_t st) {
  if (n <= 0) return SG_OK;
  if (h->global) {
    for (int a = 0; a < n; ++a) {
      sg_status r = check(h, launch_global_sweep(h->job, h->dev, gtab_of(h), esum_of(h), st));
      if (r != SG_OK) return r;
      h->t_metro += 1;
    }
    return SG_OK;
  }
  sg_status r = launch_resident<false, false>(h, st, n, 1);
  if (r == SG_OK) h->t_metro += (uint64_t)n;
  return r;
}

sg_status exchange(sg_handle *h, cudaStream_t st) {
  // general couplings: the energy launch with its exchange fused (int64 energies)
  sg_status r = h->gauss ? launch_resident<true, true>(h, st, 1, 1) : check(h, launch_exchange(h->job, h->dev, st));
  if (r == SG_OK) h->t_pt += 1;
  return r;
}

sg_status recompute_energy(sg_handle *h, cudaStream_t st) {
  if (h->global) return check(h, launch_global_energy(h->job, h->dev, gtab_of(h), esum_of(h), st));
  return launch_resident<false, true>(h, st, 1, 1);
}

// The cluster move itself (spins only; energies are stale until recomputed).
sg_status houdayer_move(sg_handle *h, cudaStream_t st, bool multi, bool fused = false) {
  uint32_t *scratch = h->lay.houd_bytes ? reinterpret_cast<uint32_t *>(h->buf + h->lay.houd) : nullptr;
  sg_status r = check(h, launch_houdayer(h->job, h->dev, scratch, HOUD_SMEM_BUDGET, multi, st, fused));
  if (r == SG_OK) h->t_houd += 1;
  return r;
}

// Read the device error word; poison the handle if a bounded wait expired.
sg_status poll_device_error(sg_handle *h, cudaStream_t st) {
  unsigned long long err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, h->dev.ctr + CTR_ERROR, sizeof(err), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return check(h, e);
  if (err) {
    h->sticky = SG_ETIMEOUT;
    return SG_ETIMEOUT;
  }
  return SG_OK;
}

} // namespace

namespace {
// The copy stream and events of asynchronous measurements, created once per handle.
cudaError_t ensure_copy_stream(sg_handle *h) {
  if (h->cst) return cudaSuccess;
  cudaError_t e = cudaStreamCreateWithFlags(&h->cst, cudaStreamNonBlocking);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&h->ev_ready[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_done[i], cudaEventDisableTiming);
  }
  return e;
}

// Staging for a measurement into host buffers.  `side`: the copies run on the handle's
// copy stream from alternating staging slots, so that `st` goes on with its next work
// (not while `st` is being captured into a graph); otherwise on `st` from slot 0.  A
// slot is rewritten only after its previous copies have finished.
struct MeasStage {
  bool side;
  int slot;
  int32_t *dE, *dQ;
};

cudaError_t measure_stage(sg_handle *h, cudaStream_t st, bool side, MeasStage *ms) {
  if (side) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) side = false;
  }
  if (side && ensure_copy_stream(h) != cudaSuccess) side = false;
  const size_t nE = (size_t)h->job.S * h->job.C * h->job.T, nQ = (size_t)h->job.S * h->job.T;
  ms->side = side;
  ms->slot = side ? h->mslot : 0;
  if (side) h->mslot ^= 1;
  ms->dE = reinterpret_cast<int32_t *>(h->buf + h->lay.meas_E) + ms->slot * nE;
  ms->dQ = reinterpret_cast<int32_t *>(h->buf + h->lay.meas_Q) + ms->slot * nQ;
  if (side && h->slot_used[ms->slot]) return cudaStreamWaitEvent(st, h->ev_done[ms->slot], 0);
  return cudaSuccess;
}

cudaError_t measure_copy(sg_handle *h, cudaStream_t st, const MeasStage &ms, int32_t *E_out, int32_t *Q_out) {
  const size_t nE = (size_t)h->job.S * h->job.C * h->job.T, nQ = (size_t)h->job.S * h->job.T;
  cudaError_t e = cudaSuccess;
  cudaStream_t cp = st;
  if (ms.side) {
    e = cudaEventRecord(h->ev_ready[ms.slot], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->cst, h->ev_ready[ms.slot], 0);
    cp = h->cst;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(E_out, ms.dE, nE * 4, cudaMemcpyDeviceToHost, cp);
  if (e == cudaSuccess && Q_out) e = cudaMemcpyAsync(Q_out, ms.dQ, nQ * 4, cudaMemcpyDeviceToHost, cp);
  if (ms.side && e == cudaSuccess) {
    e = cudaEventRecord(h->ev_done[ms.slot], h->cst);
    h->slot_used[ms.slot] = true;
  }
  return e;
}

// E by slot and N q into host buffers (see measure_stage for `side`).
sg_status measure_to_host(sg_handle *h, int32_t *E_out, int32_t *Q_out, cudaStream_t st, bool side) {
  if (!h || !E_out) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (h->gauss) return SG_EUNSUPPORTED;
  if (h->job.C < 2) Q_out = nullptr;
  MeasStage ms;
  cudaError_t e = measure_stage(h, st, side, &ms);
  if (e == cudaSuccess) e = launch_measure(h->job, h->dev, h->int8fmt != 0, ms.dE, Q_out ? ms.dQ : nullptr, st);
  if (e == cudaSuccess) e = measure_copy(h, st, ms, E_out, Q_out);
  return check(h, e);
}
} // namespace

extern "C" {

sg_status sg_query_bytes(const sg_params *p, size_t *device_bytes) {
  if (!device_bytes) return SG_EINVAL;
  const sg_status v = validate(p);
  if (v != SG_OK) return v;
  Job jb;
  build_job(p, &jb);
  *device_bytes = layout_of(p, jb).total;
  return SG_OK;
}

sg_status sg_create(const sg_params *p, void *device_buf, size_t bytes, uintptr_t stream, sg_handle **out) {
  if (!out) return SG_EINVAL;
  *out = nullptr;
  const sg_status v = validate(p);
  if (v != SG_OK) return v;
  if (!device_buf || (reinterpret_cast<uintptr_t>(device_buf) & 255u)) return SG_EINVAL;
  sg_handle *h = new (std::nothrow) sg_handle();
  if (!h) return SG_ENOMEM;
  h->p = *p;
  h->temps.assign(p->temps, p->temps + p->n_temps);
  h->p.temps = nullptr;
  build_job(p, &h->job);
  h->lay = layout_of(p, h->job);
  if (bytes < h->lay.total) {
    delete h;
    return SG_ENOMEM;
  }
  h->buf = static_cast<char *>(device_buf);
  h->bytes = bytes;
  h->t_metro = h->t_pt = h->t_houd = 0;
  h->sticky = SG_OK;
  h->int8fmt = p->spin_format == SG_INT8;
  const int T = p->n_temps, d = p->ndim;
  h->global = false;
  h->pair_on = true;
  if (!choose_resident(h, max_dyn_smem())) {
    if (h->int8fmt) { // the int8 layout has no streaming path
      delete h;
      return SG_EUNSUPPORTED;
    }
    h->global = true; // the lattice does not fit a CTA: stream it from global memory
    h->nt = 256;
    h->wpc = 1;
    h->smem = 0;
  }
  if (p->coupling_kind == SG_COUPLINGS_FIXED) {
    h->smem = gauss_smem_bytes(h->job);
    if ((int)h->smem > max_dyn_smem()) {
      delete h;
      return SG_EUNSUPPORTED;
    }
  }
  h->fuse_pt = !h->global && (h->int8fmt ? true : (h->wpc % h->job.Wc == 0));
  h->n_ctr = CTR_PT + T;

  h->beta.resize(T);
  h->thr.assign((size_t)T * 4, 0u);
  for (int k = 0; k < T; ++k) {
    h->beta[k] = 1.0 / h->temps[k];
    for (int m = 1; m <= d; ++m) h->thr[(size_t)k * 4 + m] = metropolis_threshold(h->beta[k], 4 * m);
  }
  Dev &dv = h->dev;
  dv.spins = reinterpret_cast<uint32_t *>(h->buf + h->lay.spins);
  dv.jbits = reinterpret_cast<uint32_t *>(h->buf + h->lay.jbits);
  dv.E = reinterpret_cast<int32_t *>(h->buf + h->lay.E);
  dv.perm = reinterpret_cast<int32_t *>(h->buf + h->lay.perm);
  dv.slot = reinterpret_cast<int32_t *>(h->buf + h->lay.slot);
  dv.thr = reinterpret_cast<const uint32_t *>(h->buf + h->lay.thr);
  dv.beta = reinterpret_cast<const double *>(h->buf + h->lay.beta);
  dv.ctr = reinterpret_cast<unsigned long long *>(h->buf + h->lay.ctr);
  const bool tr = p->track_trips != 0;
  dv.trip_dir = tr ? reinterpret_cast<int32_t *>(h->buf + h->lay.trip_dir) : nullptr;
  dv.trip_t0 = tr ? reinterpret_cast<uint32_t *>(h->buf + h->lay.trip_t0) : nullptr;
  dv.trip_n = tr ? reinterpret_cast<uint32_t *>(h->buf + h->lay.trip_n) : nullptr;
  dv.trip_sum = tr ? reinterpret_cast<unsigned long long *>(h->buf + h->lay.trip_sum) : nullptr;
  h->gauss = p->coupling_kind == SG_COUPLINGS_FIXED;
  dv.jfix = h->gauss ? reinterpret_cast<int32_t *>(h->buf + h->lay.jfix) : nullptr;
  dv.E64 = h->gauss ? reinterpret_cast<long long *>(h->buf + h->lay.E64) : nullptr;

  cudaStream_t st = as_stream(stream);
  cudaError_t e = prepare_device();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->buf + h->lay.thr, h->thr.data(), h->thr.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->buf + h->lay.beta, h->beta.data(), h->beta.size() * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dv.ctr, 0, (size_t)h->n_ctr * 8, st);
  if (e == cudaSuccess && tr) e = cudaMemsetAsync(h->buf + h->lay.trip_dir, 0, h->lay.jfix - h->lay.trip_dir, st);
  if (e == cudaSuccess && h->gauss) e = cudaMemsetAsync(dv.jfix, 0, h->lay.E64 - h->lay.jfix, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->buf + h->lay.esum, 0, (size_t)h->job.S * h->job.W * 32 * 4, st);
  if (e == cudaSuccess) e = launch_init(h->job, dv, h->int8fmt != 0, st);
  if (e != cudaSuccess) {
    delete h;
    return SG_ECUDA;
  }
  if (recompute_energy(h, st) != SG_OK) {
    delete h;
    return SG_ECUDA;
  }
  // the pageable host tables above must not be freed before the copies have read them
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    delete h;
    return SG_ECUDA;
  }
  *out = h;
  return SG_OK;
}

sg_status sg_sweep(sg_handle *h, int32_t n_sweeps, uintptr_t stream) {
  if (!h || n_sweeps < 0) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  return sweeps(h, n_sweeps, as_stream(stream));
}

sg_status sg_exchange(sg_handle *h, uintptr_t stream) {
  if (!h) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  return exchange(h, as_stream(stream));
}

sg_status sg_houdayer(sg_handle *h, uintptr_t stream) {
  if (h && h->gauss) return SG_EUNSUPPORTED; // +-J (or packed-spin) only
  if (!h) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (h->job.C != 2) return SG_EINVAL;
  if (!houdayer_possible(&h->p, h->job)) return SG_EUNSUPPORTED;
  cudaStream_t st = as_stream(stream);
  sg_status r = houdayer_move(h, st, false);
  return r == SG_OK ? recompute_energy(h, st) : r;
}

// The multi-cluster variant needs the bitmap scratch (a handle made with houdayer != 0,
// or a lattice too large for the single-CTA kernel) and labels that fit shared memory.
bool multi_possible(const sg_handle *h) {
  return houdayer_possible(&h->p, h->job) && h->lay.houd_bytes > 0 && houdayer_labels(h->job);
}

// The words per CTA when this handle's fused MCS pairs its chains' last words (0: it
// does not).  Pairing holds whole chains, so it applies whatever the handle's own shape.
int pair_ok(const sg_handle *h) {
  if (!h->pair_on || h->int8fmt || h->global || h->gauss || h->p.houdayer) return 0;
  int nt = h->nt;
  size_t sm = 0;
  return pair_words(h->job, &nt, max_dyn_smem(), &sm);
}

// Whether an MCS with the move can give its first and last phases to the resident
// launches around it: packed spins in shared memory, one CTA per sample holding both
// one-word chains, the bitmap scratch present, the exchange fused.
bool houd_fused(const sg_handle *h) {
  return h->p.houdayer && h->fuse_pt && !h->global && !h->int8fmt && !h->gauss && h->lay.houd_bytes > 0 &&
         h->wpc == 2 && h->job.C == 2 && h->job.Wc == 1 && houdayer_possible(&h->p, h->job);
}

sg_status sg_houdayer_multi(sg_handle *h, uintptr_t stream) {
  if (h && h->gauss) return SG_EUNSUPPORTED; // +-J (or packed-spin) only
  if (!h) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (h->job.C != 2) return SG_EINVAL;
  if (!multi_possible(h)) return SG_EUNSUPPORTED;
  cudaStream_t st = as_stream(stream);
  sg_status r = houdayer_move(h, st, true);
  return r == SG_OK ? recompute_energy(h, st) : r;
}

namespace {
// Enqueue n_mcs Monte Carlo steps of one handle on `st` (Sec. 2.4 order) and advance
// the host copies of its step counters.
sg_status mcs_ops(sg_handle *h, int n_mcs, cudaStream_t st) {
  if (n_mcs == 0) return SG_OK;
  const int nm = h->p.n_metro;
  if (!h->p.houdayer && !h->global && (h->fuse_pt || pair_ok(h))) {
    sg_status r = launch_resident<true, false>(h, st, n_mcs, nm);
    if (r == SG_OK) {
      h->t_metro += (uint64_t)n_mcs * (uint64_t)nm;
      h->t_pt += (uint64_t)n_mcs;
    }
    return r;
  }
  if (h->p.houdayer && !houdayer_possible(&h->p, h->job)) return SG_EUNSUPPORTED;
  if (h->p.houdayer == 2 && !multi_possible(h)) return SG_EUNSUPPORTED;
  if (houd_fused(h)) {
    // the move's q bitmaps come out of the sweep launch and its flips go into the next
    // launch: the next MCS's sweep launch, which first takes the energies after the move
    // and that MCS's exchange (HOUD 3), or after the last MCS one energy launch with the
    // exchange (HOUD 2).  Two launches per MCS around the cluster phase, and one more
    // per call.
    const sgmc::HoudMaps hm = sgmc::houd_maps_of(h->job, reinterpret_cast<uint32_t *>(h->buf + h->lay.houd));
    for (int m = 0; m < n_mcs; ++m) {
      sg_status r =
          m == 0 ? check(h, sgmc::launch_resident(h->job, h->dev, false, h->nt, h->wpc, false, false, h->smem, st, nm,
                                                  1, nullptr, nullptr, false, &hm, 1))
                 : check(h, sgmc::launch_resident(h->job, h->dev, false, h->nt, h->wpc, true, false, h->smem, st, 1,
                                                  nm, nullptr, nullptr, false, &hm, 3));
      if (r != SG_OK) return r;
      if (m > 0) h->t_pt += 1;
      h->t_metro += (uint64_t)nm;
      r = houdayer_move(h, st, h->p.houdayer == 2, true);
      if (r != SG_OK) return r;
    }
    const sg_status r = check(h, sgmc::launch_resident(h->job, h->dev, false, h->nt, h->wpc, true, true, h->smem, st,
                                                       1, 1, nullptr, nullptr, true, &hm, 2));
    if (r == SG_OK) h->t_pt += 1;
    return r;
  }
  for (int m = 0; m < n_mcs; ++m) {
    sg_status r = sweeps(h, nm, st);
    if (r == SG_OK && h->p.houdayer) {
      r = houdayer_move(h, st, h->p.houdayer == 2);
      if (r == SG_OK && h->fuse_pt && !h->global) {
        // energies after the move, then the exchange, in one resident launch (chain 1's
        // energies from the conserved pair sums when a CTA holds both chains)
        r = check(h, sgmc::launch_resident(h->job, h->dev, false, h->nt, h->wpc, true, true, h->smem, st, 1, 1, nullptr,
                                           nullptr, true));
        if (r == SG_OK) h->t_pt += 1;
        if (r != SG_OK) return r;
        continue;
      }
      if (r == SG_OK) r = recompute_energy(h, st);
    }
    if (r == SG_OK) r = exchange(h, st);
    if (r != SG_OK) return r;
  }
  return SG_OK;
}
} // namespace

sg_status sg_run_mcs(sg_handle *h, int32_t n_mcs, uintptr_t stream) {
  if (!h || n_mcs < 0) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  return mcs_ops(h, n_mcs, as_stream(stream));
}

// ---------------------------------------------------------------------------------
// Batches: the MCS cycles of several jobs captured once into one CUDA graph, each job a
// branch of its own (its kernels run concurrently with the other jobs'), replayed as
// often as needed.  The kernels read their step counters on the device, so the same
// graph serves every replay.
// ---------------------------------------------------------------------------------
struct sg_batch {
  std::vector<sg_handle *> jobs;
  cudaStream_t origin;               // capture stream (the legacy default stream cannot be captured)
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events; // fork + one join per job
  int mcs_per_launch;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  std::vector<uint64_t> d_metro, d_pt, d_houd; // counter advance per replay, per job
};

void destroy_batch(sg_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  for (cudaStream_t q : b->streams) cudaStreamDestroy(q);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

sg_status sg_batch_create(sg_handle *const *handles, int32_t n_handles, int32_t mcs_per_launch, uintptr_t stream,
                          sg_batch **out) {
  if (!out || !handles || n_handles < 1 || mcs_per_launch < 1) return SG_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n_handles; ++i) {
    if (!handles[i]) return SG_EINVAL;
    if (handles[i]->sticky != SG_OK) return handles[i]->sticky;
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return SG_EINVAL;
  }
  sg_batch *b = new (std::nothrow) sg_batch();
  if (!b) return SG_ENOMEM;
  b->mcs_per_launch = mcs_per_launch;
  b->graph = nullptr;
  b->exec = nullptr;
  b->origin = nullptr;
  (void)stream; // nothing is enqueued here; sg_batch_run launches on its own stream
  cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  cudaStream_t origin = b->origin;
  b->events.resize((size_t)n_handles + 1, nullptr);
  for (auto &ev : b->events)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  // Each job's branch is captured on a stream of its own whose priority ranks the job by
  // the work of one of its CTAs (sites x words per CTA, x 2 for a chain split over CTAs
  // whose exchange runs as a second launch): the graph runs with these node priorities,
  // so the longest items are placed first and the short ones fill in around them instead
  // of leaving the long ones to run on alone at the end of every launch.
  int prio_least = 0, prio_greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) prio_least = prio_greatest = 0;
  const int smem_limit = max_dyn_smem();
  // words per CTA of the jobs whose fused sweeps pair their chains' last words (0: not
  // paired), with that launch's threads and shared memory
  std::vector<int> pair_w((size_t)n_handles, 0), pair_nt((size_t)n_handles, 0);
  std::vector<size_t> pair_sm((size_t)n_handles, 0);
  for (int i = 0; i < n_handles; ++i) {
    const sg_handle *h = handles[i];
    pair_nt[i] = h->nt;
    if (h->pair_on && !h->int8fmt && !h->global && !h->gauss && !h->p.houdayer)
      pair_w[i] = pair_words(h->job, &pair_nt[i], smem_limit, &pair_sm[i]);
  }
  std::vector<double> item_work((size_t)n_handles, 0.0);
  for (int i = 0; i < n_handles; ++i) {
    const sg_handle *h = handles[i];
    const int wpc = pair_w[i] ? pair_w[i] : (h->global ? 1 : h->wpc);
    item_work[i] = (double)h->job.g.N * wpc * (h->fuse_pt || pair_w[i] ? 1.0 : 2.0);
  }
  std::vector<double> ranked = item_work;
  std::sort(ranked.begin(), ranked.end());
  ranked.erase(std::unique(ranked.begin(), ranked.end()), ranked.end());
  const int levels = prio_least - prio_greatest + 1; // priorities prio_greatest..prio_least
  b->streams.resize((size_t)n_handles, nullptr);
  for (int i = 0; i < n_handles && e == cudaSuccess; ++i) {
    // rank 0 = the most work per item -> the greatest priority (the smallest number)
    const int rank = (int)(ranked.end() - std::upper_bound(ranked.begin(), ranked.end(), item_work[i]));
    const int prio = prio_greatest + (rank < levels ? rank : levels - 1);
    e = cudaStreamCreateWithPriority(&b->streams[i], cudaStreamNonBlocking, prio);
  }
  if (e != cudaSuccess) {
    destroy_batch(b);
    return SG_ECUDA;
  }
  // the kernels' shared-memory attributes were set when the handles were created, so the
  // capture holds kernel launches and event edges only
  e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    destroy_batch(b);
    return SG_ECUDA;
  }
  sg_status r = SG_OK;
  e = cudaEventRecord(b->events[0], origin);
  // jobs that the multi-job resident kernel can sweep together: packed spins, resident,
  // no Houdayer move; grouped by lattice shape and words per chain (one launch per group
  // and MCS chunk)
  std::vector<int> group_of((size_t)n_handles, -1);
  std::vector<std::vector<int>> groups;
  for (int i = 0; i < n_handles; ++i) {
    const sg_handle *h = handles[i];
    if (h->int8fmt || h->global || h->p.houdayer) continue;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      const sg_handle *o = handles[groups[gi][0]];
      if (o->job.g.d == h->job.g.d && o->job.g.L0 == h->job.g.L0 && o->job.g.L1 == h->job.g.L1 &&
          o->job.g.L2 == h->job.g.L2 && o->job.Wc == h->job.Wc && pair_w[groups[gi][0]] == pair_w[i] &&
          pair_nt[groups[gi][0]] == pair_nt[i]) {
        group_of[i] = (int)gi;
        groups[gi].push_back(i);
        break;
      }
    }
    if (group_of[i] < 0) {
      group_of[i] = (int)groups.size();
      groups.push_back({i});
    }
  }
  for (int i = 0; i < n_handles; ++i) b->jobs.push_back(handles[i]);
  std::vector<uint64_t> m0, p0, h0;
  for (sg_handle *h : b->jobs) {
    m0.push_back(h->t_metro);
    p0.push_back(h->t_pt);
    h0.push_back(h->t_houd);
  }
  for (size_t gi = 0; gi < groups.size() && r == SG_OK && e == cudaSuccess; ++gi) {
    cudaStream_t q = b->streams[groups[gi][0]];
    e = cudaStreamWaitEvent(q, b->events[0], 0);
    // one shape for the group: the first job's (tuned) shape, falling back to one word
    // per CTA when a job has an odd number of words or two do not fit; a group of paired
    // jobs holds a whole sample per CTA
    sg_handle *lead = handles[groups[gi][0]];
    const int pw = pair_w[groups[gi][0]];
    int wpc = pw ? pw : lead->wpc;
    int nt = pw ? pair_nt[groups[gi][0]] : lead->nt;
    size_t sm = pw ? pair_sm[groups[gi][0]] : 0;
    if (!pw) {
      for (int i : groups[gi])
        if (handles[i]->job.W % wpc) wpc = 1;
      if (wpc == 2 && !packed_shape_ok(lead, lead->nt, 2, smem_limit, &sm)) wpc = 1;
      if (!packed_shape_ok(lead, lead->nt, wpc, smem_limit, &sm)) {
        r = SG_EUNSUPPORTED;
        break;
      }
    }
    std::vector<JobDesc> descs;
    std::vector<sg_handle *> unfused;
    for (int i : groups[gi]) {
      sg_handle *h = handles[i];
      JobDesc jd;
      jd.jb = h->job;
      jd.dv = h->dev;
      jd.first_item = 0;
      jd.n_items = pw ? h->job.S : h->job.S * (h->job.W / wpc);
      jd.fuse = (pw || wpc % h->job.Wc == 0) ? 1 : 0;
      jd.n_metro = h->p.n_metro;
      descs.push_back(jd);
      if (!jd.fuse) unfused.push_back(h);
    }
    // a group is fused or not as a whole (same lattice and words per chain): fused groups
    // run the whole chunk in one launch, the others alternate sweeps and one exchange
    // launch for all their jobs
    const int chunk = unfused.empty() ? mcs_per_launch : 1;
    for (int m = 0; m < mcs_per_launch && e == cudaSuccess; m += chunk) {
      e = launch_resident_batch(descs.data(), (int)descs.size(), nt, wpc, sm, q, chunk, pw != 0);
      if (e == cudaSuccess && !unfused.empty()) e = launch_exchange_batch(descs.data(), (int)descs.size(), q);
    }
    for (int i : groups[gi]) {
      sg_handle *h = handles[i];
      h->t_metro += (uint64_t)mcs_per_launch * (uint64_t)h->p.n_metro;
      h->t_pt += (uint64_t)mcs_per_launch;
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->events[groups[gi][0] + 1], q);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, b->events[groups[gi][0] + 1], 0);
  }
  for (int i = 0; i < n_handles && r == SG_OK && e == cudaSuccess; ++i) {
    if (group_of[i] >= 0) continue;
    sg_handle *h = handles[i];
    e = cudaStreamWaitEvent(b->streams[i], b->events[0], 0);
    if (e == cudaSuccess) r = mcs_ops(h, mcs_per_launch, b->streams[i]);
    if (e == cudaSuccess && r == SG_OK) e = cudaEventRecord(b->events[i + 1], b->streams[i]);
    if (e == cudaSuccess && r == SG_OK) e = cudaStreamWaitEvent(origin, b->events[i + 1], 0);
  }
  // capture only records the work: the counters advance when the graph is launched
  for (size_t i = 0; i < b->jobs.size(); ++i) {
    sg_handle *h = b->jobs[i];
    b->d_metro.push_back(h->t_metro - m0[i]);
    b->d_pt.push_back(h->t_pt - p0[i]);
    b->d_houd.push_back(h->t_houd - h0[i]);
    h->t_metro = m0[i];
    h->t_pt = p0[i];
    h->t_houd = h0[i];
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(origin, &g);
  b->graph = g;
  if (r != SG_OK || e != cudaSuccess || e2 != cudaSuccess || !g) {
    for (sg_handle *h : b->jobs)
      if (h->sticky == SG_ECUDA) h->sticky = SG_OK; // a failed capture leaves the jobs untouched
    destroy_batch(b);
    return r != SG_OK ? r : SG_ECUDA;
  }
  if (cudaGraphInstantiate(&b->exec, g, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
    destroy_batch(b);
    return SG_ECUDA;
  }
  *out = b;
  return SG_OK;
}

sg_status sg_batch_run(sg_batch *b, int32_t n_launches, uintptr_t stream) {
  if (!b || n_launches < 0) return SG_EINVAL;
  for (sg_handle *h : b->jobs)
    if (h->sticky != SG_OK) return h->sticky;
  cudaStream_t st = as_stream(stream);
  for (int a = 0; a < n_launches; ++a) {
    const cudaError_t e = cudaGraphLaunch(b->exec, st);
    if (e != cudaSuccess) {
      for (sg_handle *h : b->jobs) h->sticky = SG_ECUDA;
      return SG_ECUDA;
    }
    for (size_t i = 0; i < b->jobs.size(); ++i) {
      b->jobs[i]->t_metro += b->d_metro[i];
      b->jobs[i]->t_pt += b->d_pt[i];
      b->jobs[i]->t_houd += b->d_houd[i];
    }
  }
  return SG_OK;
}

void sg_batch_destroy(sg_batch *b) { destroy_batch(b); }

sg_status sg_measure_device(sg_handle *h, int32_t *E_out, int32_t *Q_out, uintptr_t stream) {
  if (!h || !E_out) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (h->gauss) return SG_EUNSUPPORTED;
  cudaStream_t st = as_stream(stream);
  return check(h, launch_measure(h->job, h->dev, h->int8fmt != 0, E_out, Q_out, st));
}

sg_status sg_measure_async(sg_handle *h, int32_t *E_out, int32_t *Q_out, uintptr_t stream) {
  return measure_to_host(h, E_out, Q_out, as_stream(stream), true);
}

sg_status sg_measure_wait(sg_handle *h) {
  if (!h) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (!h->cst) return SG_OK;
  return check(h, cudaStreamSynchronize(h->cst));
}

sg_status sg_run_mcs_measure_async(sg_handle *h, int32_t n_mcs, int32_t *E_out, int32_t *Q_out, uintptr_t stream) {
  if (!h || n_mcs < 1 || !E_out) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (h->gauss) return SG_EUNSUPPORTED;
  cudaStream_t st = as_stream(stream);
  const bool fused = !h->int8fmt && !h->global && !h->p.houdayer && h->fuse_pt && h->job.C == 2 && h->job.Wc == 1 &&
                     h->wpc == 2;
  if (!fused) {
    const sg_status r = mcs_ops(h, n_mcs, st);
    if (r != SG_OK) return r;
    return measure_to_host(h, E_out, Q_out, st, true);
  }
  // the measurement runs inside the last MCS's launch, from the lattice in shared memory
  MeasStage ms;
  cudaError_t e = measure_stage(h, st, true, &ms);
  if (e == cudaSuccess)
    e = sgmc::launch_resident(h->job, h->dev, false, h->nt, h->wpc, true, false, h->smem, st, n_mcs, h->p.n_metro,
                              ms.dE, Q_out ? ms.dQ : nullptr);
  if (e == cudaSuccess) {
    h->t_metro += (uint64_t)n_mcs * (uint64_t)h->p.n_metro;
    h->t_pt += (uint64_t)n_mcs;
    e = measure_copy(h, st, ms, E_out, Q_out);
  }
  return check(h, e);
}

sg_status sg_measure(sg_handle *h, int32_t *E_out, int32_t *Q_out, uintptr_t stream) {
  const sg_status r = measure_to_host(h, E_out, Q_out, as_stream(stream), false);
  if (r != SG_OK) return r;
  return poll_device_error(h, as_stream(stream));
}

sg_status sg_trips(sg_handle *h, uint32_t *n_out, uint64_t *sum_out, uintptr_t stream) {
  if (!h || !n_out || !sum_out) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (!h->dev.trip_n) return SG_EINVAL;
  cudaStream_t st = as_stream(stream);
  const size_t n = (size_t)h->job.S * h->job.C;
  cudaError_t e = cudaMemcpyAsync(n_out, h->dev.trip_n, n * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sum_out, h->dev.trip_sum, n * 8, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return check(h, e);
  return poll_device_error(h, st);
}

sg_status sg_measure_qmodes_device(sg_handle *h, int32_t *P_out, uintptr_t stream) {
  if (!h || !P_out) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (h->job.C < 2) return SG_EINVAL;
  return check(h, launch_qmodes(h->job, h->dev, h->int8fmt != 0, P_out, as_stream(stream)));
}

sg_status sg_measure_qmodes(sg_handle *h, int32_t *P_out, uintptr_t stream) {
  if (!h || !P_out) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (h->job.C < 2) return SG_EINVAL;
  cudaStream_t st = as_stream(stream);
  int32_t *dP = reinterpret_cast<int32_t *>(h->buf + h->lay.meas_P);
  sg_status r = sg_measure_qmodes_device(h, dP, stream);
  if (r != SG_OK) return r;
  const size_t n = (size_t)h->job.S * h->job.T * h->job.g.d * (size_t)qmodes_lmax(h->job);
  const cudaError_t e = cudaMemcpyAsync(P_out, dP, n * 4, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return check(h, e);
  return poll_device_error(h, st);
}

sg_status sg_import_couplings_fixed(sg_handle *h, const int32_t *J_in, uintptr_t stream) {
  if (!h || !J_in) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (!h->gauss) return SG_EINVAL;
  const size_t n = (size_t)h->job.S * h->job.g.N * h->job.g.d;
  for (size_t i = 0; i < n; ++i)
    if (J_in[i] > (1 << 23) || J_in[i] < -(1 << 23)) return SG_EINVAL;
  cudaStream_t st = as_stream(stream);
  int32_t *stage = reinterpret_cast<int32_t *>(h->buf + h->lay.jstage);
  cudaError_t e = cudaMemcpyAsync(stage, J_in, n * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_gauss_import(h->job, h->dev, stage, st);
  if (e != cudaSuccess) return check(h, e);
  return recompute_energy(h, st);
}

sg_status sg_measure64(sg_handle *h, int64_t *E_out, int32_t *Q_out, uintptr_t stream) {
  if (!h || !E_out) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (!h->gauss) return SG_EINVAL;
  cudaStream_t st = as_stream(stream);
  long long *dE = reinterpret_cast<long long *>(h->buf + h->lay.meas_E64);
  int32_t *dQ = reinterpret_cast<int32_t *>(h->buf + h->lay.meas_Q);
  const bool want_q = Q_out && h->job.C >= 2;
  cudaError_t e = launch_gather_energy64(h->job, h->dev, dE, st);
  if (e == cudaSuccess && want_q) e = launch_measure(h->job, h->dev, true, reinterpret_cast<int32_t *>(
                                                         h->buf + h->lay.meas_E), dQ, st);
  const size_t nE = (size_t)h->job.S * h->job.C * h->job.T, nQ = (size_t)h->job.S * h->job.T;
  if (e == cudaSuccess) e = cudaMemcpyAsync(E_out, dE, nE * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && want_q) e = cudaMemcpyAsync(Q_out, dQ, nQ * 4, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return check(h, e);
  return poll_device_error(h, st);
}

sg_status sg_get_state64(sg_handle *h, int64_t *E_out, int32_t *perm_out, uint64_t *steps_out, uintptr_t stream) {
  if (!h) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (!h->gauss) return SG_EINVAL;
  cudaStream_t st = as_stream(stream);
  const size_t n = (size_t)h->job.S * h->job.C * h->job.T;
  cudaError_t e = cudaSuccess;
  if (E_out) e = cudaMemcpyAsync(E_out, h->dev.E64, n * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && perm_out) e = cudaMemcpyAsync(perm_out, h->dev.perm, n * 4, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return check(h, e);
  if (steps_out) {
    steps_out[0] = h->t_metro;
    steps_out[1] = h->t_pt;
    steps_out[2] = h->t_houd;
  }
  return poll_device_error(h, st);
}

sg_status sg_export_spins(sg_handle *h, uint8_t *spins_out, uintptr_t stream) {
  if (!h || !spins_out) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  return check(h, launch_export_spins(h->job, h->dev, h->int8fmt != 0, spins_out, as_stream(stream)));
}

sg_status sg_import_spins(sg_handle *h, const uint8_t *spins_in, uintptr_t stream) {
  if (!h || !spins_in) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  cudaStream_t st = as_stream(stream);
  sg_status r = check(h, launch_import_spins(h->job, h->dev, h->int8fmt != 0, spins_in, st));
  return r == SG_OK ? recompute_energy(h, st) : r;
}

sg_status sg_export_couplings(sg_handle *h, int8_t *J_out, uintptr_t stream) {
  if (h && h->gauss) return SG_EUNSUPPORTED; // +-J (or packed-spin) only
  if (!h || !J_out) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  return check(h, launch_export_couplings(h->job, h->dev, J_out, as_stream(stream)));
}

sg_status sg_import_couplings(sg_handle *h, const int8_t *J_in, uintptr_t stream) {
  if (h && h->gauss) return SG_EUNSUPPORTED; // +-J (or packed-spin) only
  if (!h || !J_in) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  cudaStream_t st = as_stream(stream);
  sg_status r = check(h, launch_import_couplings(h->job, h->dev, J_in, st));
  return r == SG_OK ? recompute_energy(h, st) : r;
}

sg_status sg_get_state(sg_handle *h, int32_t *E_out, int32_t *perm_out, uint64_t *steps_out, uintptr_t stream) {
  if (!h) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (h->gauss && E_out) return SG_EUNSUPPORTED;
  cudaStream_t st = as_stream(stream);
  const size_t n = (size_t)h->job.S * h->job.C * h->job.T;
  cudaError_t e = cudaSuccess;
  if (E_out) e = cudaMemcpyAsync(E_out, h->dev.E, n * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && perm_out) e = cudaMemcpyAsync(perm_out, h->dev.perm, n * 4, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return check(h, e);
  if (steps_out) {
    steps_out[0] = h->t_metro;
    steps_out[1] = h->t_pt;
    steps_out[2] = h->t_houd;
  }
  return poll_device_error(h, st);
}

sg_status sg_counters(sg_handle *h, uint64_t *near_threshold, uint64_t *pt_accepts, uint64_t *houdayer_sites,
                      uintptr_t stream) {
  if (!h) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  cudaStream_t st = as_stream(stream);
  std::vector<unsigned long long> c((size_t)h->n_ctr);
  cudaError_t e = cudaMemcpyAsync(c.data(), h->dev.ctr, c.size() * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return check(h, e);
  if (c[CTR_ERROR]) {
    h->sticky = SG_ETIMEOUT;
    return SG_ETIMEOUT;
  }
  if (near_threshold) *near_threshold = c[CTR_NEAR];
  if (houdayer_sites) *houdayer_sites = c[CTR_HSITES];
  if (pt_accepts)
    for (int k = 0; k + 1 < h->job.T; ++k) pt_accepts[k] = c[CTR_PT + k];
  return SG_OK;
}

sg_status sg_exact_path_counters(sg_handle *h, uint64_t *exchange_exact, uint64_t *metropolis_band,
                                 uintptr_t stream) {
  if (!h) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  cudaStream_t st = as_stream(stream);
  unsigned long long c[CTR_PT] = {0};
  cudaError_t e = cudaMemcpyAsync(c, h->dev.ctr, sizeof(c), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return check(h, e);
  if (c[CTR_ERROR]) {
    h->sticky = SG_ETIMEOUT;
    return SG_ETIMEOUT;
  }
  if (exchange_exact) *exchange_exact = c[CTR_XEXACT];
  if (metropolis_band) *metropolis_band = c[CTR_GBAND];
  return SG_OK;
}

sg_status sg_thresholds(sg_handle *h, uint32_t *thr_out) {
  if (h && h->gauss) return SG_EUNSUPPORTED; // +-J (or packed-spin) only
  if (!h || !thr_out) return SG_EINVAL;
  const int d = h->job.g.d;
  for (int k = 0; k < h->job.T; ++k)
    for (int m = 1; m <= d; ++m) thr_out[k * d + (m - 1)] = h->thr[(size_t)k * 4 + m];
  return SG_OK;
}

sg_status sg_set_launch(sg_handle *h, int32_t threads, int32_t words) {
  if (h && h->gauss) return SG_EUNSUPPORTED; // +-J (or packed-spin) only
  if (!h) return SG_EINVAL;
  if (h->int8fmt) return (threads == 0 || threads == 256) && (words == 0 || words == 1) ? SG_OK : SG_EUNSUPPORTED;
  if (words == -1) { // stream the lattice from global memory
    h->global = true;
    h->fuse_pt = false;
    return SG_OK;
  }
  const int nt = threads ? threads : h->nt;
  const int wpc = words ? words : (h->global ? 1 : h->wpc);
  size_t sm = 0;
  if (!packed_shape_ok(h, nt, wpc, max_dyn_smem(), &sm)) return SG_EUNSUPPORTED;
  h->nt = nt;
  h->wpc = wpc;
  h->smem = sm;
  h->global = false;
  h->fuse_pt = wpc % h->job.Wc == 0;
  return SG_OK;
}

sg_status sg_set_pairing(sg_handle *h, int32_t on) {
  if (!h || (on != 0 && on != 1)) return SG_EINVAL;
  h->pair_on = on != 0;
  return SG_OK;
}

sg_status sg_get_launch(sg_handle *h, int32_t *threads, int32_t *words, int32_t *smem_bytes) {
  if (!h) return SG_EINVAL;
  if (threads) *threads = h->nt;
  if (words) *words = h->global ? -1 : h->wpc;
  if (smem_bytes) *smem_bytes = (int32_t)h->smem;
  return SG_OK;
}

sg_status sg_sweep_streaming_static(sg_handle *h, int32_t n_sweeps, uintptr_t stream) {
  if (h && h->gauss) return SG_EUNSUPPORTED; // +-J (or packed-spin) only
  if (!h || n_sweeps < 0) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (h->int8fmt) return SG_EUNSUPPORTED;
  if ((long long)h->job.S * h->job.W > STATIC_SWEEP_ITEMS) return SG_ELIMIT;
  if (n_sweeps == 0) return SG_OK;
  void *base = nullptr;
  sg_status r = check(h, static_sweep_scratch(&base)); // first call on a device: symbol lookup
  if (r != SG_OK) return r;
  uint2 *tables = reinterpret_cast<uint2 *>(base);
  uint32_t *esum = reinterpret_cast<uint32_t *>(static_cast<char *>(base) + STATIC_SWEEP_TABLES);
  cudaStream_t st = as_stream(stream);
  // the array keeps the previous call's contents: the bond sums must start at zero
  r = check(h, cudaMemsetAsync(esum, 0, (size_t)h->job.S * h->job.W * 32 * 4, st));
  for (int a = 0; a < n_sweeps && r == SG_OK; ++a) {
    r = check(h, launch_global_sweep(h->job, h->dev, tables, esum, st));
    if (r == SG_OK) h->t_metro += 1;
  }
  return r;
}

// Checkpoints: a fixed header (the parameters that fix the buffer's layout and the
// dynamics, and the host step counters), the temperatures, then the handle's whole
// device buffer.  The engine's state lives entirely in that buffer and those counters.
namespace {
struct CkptHeader {
  uint64_t magic;
  uint32_t version, reserved;
  int32_t ndim, dims[3], n_samples, sample_offset, n_chains, n_temps, spin_format, houdayer, n_metro, track_trips,
      coupling_kind, houdayer_slots;
  uint64_t sim_seed, coupling_seed;
  double p_plus;
  uint64_t t_metro, t_pt, t_houd, device_bytes;
};
constexpr uint64_t CKPT_MAGIC = 0x31544B5043474D53ull; // "SMGCPKT1"

CkptHeader header_of(const sg_handle *h) {
  CkptHeader c;
  memset(&c, 0, sizeof(c));
  c.magic = CKPT_MAGIC;
  c.version = 1;
  c.ndim = h->p.ndim;
  for (int a = 0; a < 3; ++a) c.dims[a] = a < h->p.ndim ? h->p.dims[a] : 1;
  c.n_samples = h->p.n_samples;
  c.sample_offset = h->p.sample_offset;
  c.n_chains = h->p.n_chains;
  c.n_temps = h->p.n_temps;
  c.spin_format = h->p.spin_format;
  c.houdayer = h->p.houdayer;
  c.n_metro = h->p.n_metro;
  c.track_trips = h->p.track_trips;
  c.coupling_kind = h->p.coupling_kind;
  c.houdayer_slots = h->p.houdayer_slots;
  c.sim_seed = h->p.sim_seed;
  c.coupling_seed = h->p.coupling_seed;
  c.p_plus = h->p.p_plus;
  c.t_metro = h->t_metro;
  c.t_pt = h->t_pt;
  c.t_houd = h->t_houd;
  c.device_bytes = h->lay.total;
  return c;
}

size_t ckpt_bytes(const sg_handle *h) {
  return sizeof(CkptHeader) + sizeof(double) * (size_t)h->p.n_temps + h->lay.total;
}
} // namespace

sg_status sg_checkpoint_bytes(sg_handle *h, size_t *bytes) {
  if (!h || !bytes) return SG_EINVAL;
  *bytes = ckpt_bytes(h);
  return SG_OK;
}

sg_status sg_checkpoint(sg_handle *h, void *host_out, size_t bytes, uintptr_t stream) {
  if (!h || !host_out) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (bytes < ckpt_bytes(h)) return SG_EINVAL;
  cudaStream_t st = as_stream(stream);
  const CkptHeader c = header_of(h);
  char *out = static_cast<char *>(host_out);
  memcpy(out, &c, sizeof(c));
  memcpy(out + sizeof(c), h->temps.data(), sizeof(double) * (size_t)h->p.n_temps);
  const cudaError_t e = cudaMemcpyAsync(out + sizeof(c) + sizeof(double) * (size_t)h->p.n_temps, h->buf,
                                        h->lay.total, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return check(h, e);
  return poll_device_error(h, st);
}

sg_status sg_restore(sg_handle *h, const void *host_in, size_t bytes, uintptr_t stream) {
  if (!h || !host_in) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  if (bytes < ckpt_bytes(h)) return SG_EINVAL;
  const char *in = static_cast<const char *>(host_in);
  if (h->cst) { // asynchronous measurements still copying from the staging slots
    const cudaError_t w = cudaStreamSynchronize(h->cst);
    if (w != cudaSuccess) return check(h, w);
  }
  CkptHeader c, mine = header_of(h);
  memcpy(&c, in, sizeof(c));
  // everything but the step counters must match this handle
  mine.t_metro = c.t_metro;
  mine.t_pt = c.t_pt;
  mine.t_houd = c.t_houd;
  if (memcmp(&c, &mine, sizeof(c)) != 0) return SG_EINVAL;
  if (memcmp(in + sizeof(c), h->temps.data(), sizeof(double) * (size_t)h->p.n_temps) != 0) return SG_EINVAL;
  cudaStream_t st = as_stream(stream);
  cudaError_t e = cudaMemcpyAsync(h->buf, in + sizeof(c) + sizeof(double) * (size_t)h->p.n_temps, h->lay.total,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return check(h, e);
  h->t_metro = c.t_metro;
  h->t_pt = c.t_pt;
  h->t_houd = c.t_houd;
  return SG_OK;
}

sg_status sg_selftest_wait(sg_handle *h, int32_t max_tries, uintptr_t stream) {
  if (!h || max_tries < 1 || max_tries > (1 << 20)) return SG_EINVAL;
  if (h->sticky != SG_OK) return h->sticky;
  cudaStream_t st = as_stream(stream);
  const sg_status r = check(h, launch_wait_selftest(h->dev, (uint32_t)max_tries, st));
  return r == SG_OK ? poll_device_error(h, st) : r;
}

void sg_destroy(sg_handle *h) { delete h; }

const char *sg_strerror(sg_status s) {
  switch (s) {
  case SG_OK: return "ok";
  case SG_EINVAL: return "invalid argument";
  case SG_ENOMEM: return "device buffer too small";
  case SG_ECUDA: return "CUDA error";
  case SG_ETIMEOUT: return "bounded device wait expired";
  case SG_EUNSUPPORTED: return "unsupported parameters";
  case SG_ELIMIT: return "exceeds a fixed capacity of the call";
  }
  return "unknown status";
}

} // extern "C"
