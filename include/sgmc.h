/*
 * sgmc.h -- C-ABI of the GB300 (sm_103a) engine for parallel-tempering Monte Carlo of
 * +-J Edwards-Anderson Ising spin glasses, after Kumar, Gross, Janke & Weigel,
 * "Massively parallel simulations for disordered systems" (arXiv:2003.04621).
 *
 * The engine simulates n_samples disorder samples x n_chains independent copies x
 * n_temps temperatures at once (Sec. 3).  Every call below is a plain C function over
 * host or device pointers and sizes; no C++ or framework types cross the boundary.
 *
 * Conventions
 *   - Every call returns an sg_status.  No call aborts or prints.
 *   - The handle owns NO device memory: the caller allocates one device buffer of
 *     sg_query_bytes() bytes and passes it to sg_create(); it must outlive the handle.
 *   - `stream` is a cudaStream_t cast to uintptr_t (0 = legacy default stream).  All
 *     device work of a call is enqueued on that stream; calls that return host data say
 *     so and synchronise that stream.
 *   - After SG_ECUDA or SG_ETIMEOUT the handle is poisoned: every later call except
 *     sg_destroy/sg_strerror returns the same status.
 *   - A handle is not thread-safe; use one stream per handle at a time.
 *   - Results depend only on the parameters and on the sequence of calls made: never
 *     on the device, the launch shape, or other handles running alongside.
 *
 * Model and readings (Sec. 2.1, Eqs. 1-2, H = 0)
 *   Lattice: ndim = 2 or 3, extents dims[0..ndim-1] (x fastest), periodic.  Site index
 *   i = x + L0 (y + L1 z).  Bond (i, mu) joins i and i + e_mu (forward bonds only; on an
 *   L = 2 axis both bonds between a pair are kept).  Couplings J = +-1 with
 *   P(J = +1) = p_plus (Eq. 2).  Spin bit 1 <-> s = -1.
 *   Sweep order: checkerboard, colour (x+y+z) mod 2, colour 0 first; so every extent must
 *   be even (SG_EUNSUPPORTED otherwise).
 *   Random numbers: Philox4x32-10 (counter-based, Sec. 3; Salmon et al. 2011), with
 *     couplings  key = coupling_seed, ctr = (i, mu, s, 4), word 0, J = +1 iff w < floor(p 2^32)
 *     hot start  key = sim_seed, ctr = (i, 0, s, c<<20 | (j>>2)<<8 | 3), word j&3, top bit
 *     Metropolis key = sim_seed, ctr = (i, t_metro, s, c<<20 | (j>>2)<<8 | 0), word j&3
 *     exchange   key = sim_seed, ctr = (k, t_pt, s, c<<20 | 1), word 0
 *     Houdayer   key = sim_seed, ctr = (k, t_houd, s, 2), word 0
 *   where s = sample_offset + local sample, c = chain, j = replica within its chain,
 *   k = temperature slot and t_* = the number of such steps made before.
 *
 * Device memory is laid out by the engine inside the caller's buffer; callers reach the
 * state only through the calls below (the import/export calls use plain layouts).
 */
#ifndef SGMC_H
#define SGMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_handle sg_handle; /* opaque host object */

typedef enum {
  SG_OK = 0,
  SG_EINVAL = 1,        /* invalid argument (null pointer, bad size, bad parameter)      */
  SG_ENOMEM = 2,        /* the caller's device buffer is smaller than sg_query_bytes()   */
  SG_ECUDA = 3,         /* a CUDA call failed; the handle is poisoned                    */
  SG_ETIMEOUT = 4,      /* a bounded device-side wait expired; the handle is poisoned    */
  SG_EUNSUPPORTED = 5,  /* valid but outside what this engine implements (odd extents,
                           a lattice too large for the resident kernels, ...)          */
  SG_ELIMIT = 6         /* the job exceeds a fixed capacity of the call (see the call)   */
} sg_status;

enum { SG_PACKED32 = 0, SG_INT8 = 1 };
/* Couplings: +-J drawn from coupling_seed (Eq. 2), or general couplings (e.g. Gaussian,
 * Sec. 2.1) supplied by the caller as fixed point in units of 2^-20 (sg_import_couplings_fixed). */
enum { SG_COUPLINGS_PM = 0, SG_COUPLINGS_FIXED = 1 };

/* Parameters of one simulation job (Sec. 2; the problem statement of Sec. 2.1-2.4). */
typedef struct {
  int32_t ndim;          /* 2 or 3                                                        */
  int32_t dims[3];       /* L0, L1, L2 (entries >= ndim ignored); each even and >= 2      */
  int32_t n_samples;     /* disorder samples on this handle, >= 1                         */
  int32_t sample_offset; /* job-wide index of the first sample; random keys use it, so a
                            job split over handles (or GPUs) reproduces the whole job     */
  int32_t n_chains;      /* copies per temperature: 1, or 2 (needed for q and Houdayer;
                            the paper's N_C = 2, Sec. 2.4)                                */
  int32_t n_temps;       /* temperatures per chain, >= 1                                  */
  const double *temps;   /* host, n_temps strictly ascending positive temperatures; the
                            engine copies them; beta_k = 1.0 / temps[k] in fp64         */
  uint64_t coupling_seed;
  double p_plus;         /* P(J = +1) of Eq. 2, in [0, 1]                                 */
  uint64_t sim_seed;
  int32_t spin_format;   /* SG_PACKED32: 32 replicas of one site per 32-bit word;
                            SG_INT8: one int8 +-1 per spin (the paper's layout)           */
  int32_t houdayer;      /* 1: sg_run_mcs performs one Houdayer move per (sample, slot);
                            2: the multi-cluster variant (sg_houdayer_multi) instead;
                            nonzero also reserves the bitmap scratch of the split move  */
  int32_t n_metro;       /* Metropolis sweeps per MCS (Sec. 2.4 step 1; usually 1), >= 1  */
  int32_t track_trips;   /* 1: count round trips in temperature after every exchange
                            pass (the tunnelling time of Sec. 2.3; see sg_trips); 0: off */
  int32_t coupling_kind; /* SG_COUPLINGS_PM or SG_COUPLINGS_FIXED (needs SG_INT8 spins and
                            houdayer == 0; SG_EUNSUPPORTED otherwise)                     */
  int32_t houdayer_slots; /* 0: the Houdayer move (either variant) acts at every slot;
                             K in 1..n_temps: only on the pairs at the K lowest
                             temperature slots k < K, the others are left alone (the
                             three-dimensional restriction that Secs. 1 and 2.4 point
                             to: cluster moves kept below the temperature where q = -1
                             clusters percolate); SG_EINVAL outside 0..n_temps         */
} sg_params;

/* Bytes of device memory a handle with these parameters needs. */
sg_status sg_query_bytes(const sg_params *p, size_t *device_bytes);

/* Create a simulation in the caller's device buffer (>= sg_query_bytes bytes, 256-byte
 * aligned).  Draws the couplings (Eq. 2) and a hot start, computes every energy (Eq. 1)
 * and sets each chain's temperature map to the identity.  Enqueued on `stream`; the
 * handle is usable as soon as this returns.  *out receives the handle. */
sg_status sg_create(const sg_params *p, void *device_buf, size_t bytes, uintptr_t stream,
                    sg_handle **out);

/* n_sweeps Metropolis sweeps of every replica (Sec. 2.2 and Sec. 2.4 step 1):
 * single-spin flips, accepted iff dE <= 0 or r < floor(exp(-beta dE) 2^32), r the
 * replica's Philox word for that site and sweep. */
sg_status sg_sweep(sg_handle *h, int32_t n_sweeps, uintptr_t stream);

/* One replica-exchange pass (Eq. 5; Sec. 2.4 step 3): in every (sample, chain), for
 * k = 0..n_temps-2 in order, swap the temperatures of the replicas at slots k and k+1
 * with probability min[1, exp((1/T_k - 1/T_k+1)(E_k - E_k+1))] (fp64 on the device).
 * Temperatures, not configurations, are exchanged (two maps, Sec. 3). */
sg_status sg_exchange(sg_handle *h, uintptr_t stream);

/* One Houdayer cluster move (Sec. 2.4, Eq. 10) for every (sample, temperature slot):
 * the chain-0 and chain-1 replicas at that slot exchange their spins on the connected
 * q = -1 cluster grown from the floor(u M / 2^32)-th q = -1 site (M = number of such
 * sites; no move if M = 0).  Needs n_chains == 2. */
sg_status sg_houdayer(sg_handle *h, uintptr_t stream);

/* Multi-cluster variant of the move (the remedy for idle threads named in Sec. 3): for
 * every (sample, slot) pair, every q = -1 cluster is exchanged between the two replicas
 * with probability 1/2, by the top bit of its own Philox word, counter (i_min, t_houd,
 * sample, slot << 8 | 5) with i_min the cluster's smallest site index (canonical order
 * x + L0 (y + L1 z)).  Needs n_chains == 2, a handle made with houdayer != 0 (or a
 * lattice whose bitmaps exceed the single-CTA kernel), and cluster labels that fit one
 * CTA's shared memory (about 95,000 sites); otherwise SG_EUNSUPPORTED. */
sg_status sg_houdayer_multi(sg_handle *h, uintptr_t stream);

/* n_mcs Monte Carlo steps (Sec. 2.4): n_metro sweeps, then (if houdayer) one Houdayer
 * move per pair (the multi-cluster variant when houdayer == 2), then one exchange pass.
 * Identical to the same sequence of the calls above. */
sg_status sg_run_mcs(sg_handle *h, int32_t n_mcs, uintptr_t stream);

/* Observables (Eqs. 3-4) into HOST buffers; synchronises `stream`.
 *   E_out [n_samples][n_chains][n_temps]  energy of the replica at each slot
 *   Q_out [n_samples][n_temps]            N q = sum_i s_i^(a) s_i^(b), a/b the chain-0 and
 *                                         chain-1 replicas at the slot (may be NULL;
 *                                         ignored if n_chains == 1) */
sg_status sg_measure(sg_handle *h, int32_t *E_out, int32_t *Q_out, uintptr_t stream);

/* As sg_measure, into DEVICE buffers of the same shapes, without synchronising. */
sg_status sg_measure_device(sg_handle *h, int32_t *E_out, int32_t *Q_out, uintptr_t stream);

/* As sg_measure into HOST buffers, but only enqueued: the measurement kernel runs on
 * `stream` when it gets there, and the two device-to-host copies then run on a copy
 * stream owned by the handle, so `stream` goes on with its next work (the next MCS)
 * while they run.  Two staging slots alternate; a slot is rewritten only after its
 * previous copies have finished.  The values are in the host buffers once
 * sg_measure_wait(h) has returned (or the device has been synchronised); the caller
 * keeps the buffers alive and unread until then.  Page-locked (pinned) buffers let the
 * copies run without blocking the host.  While `stream` is being captured into a CUDA
 * graph the copies stay on `stream` (no second stream enters the capture).  A
 * device-side error (a bulk-copy wait that ran out) is reported by the next call that
 * synchronises. */
sg_status sg_measure_async(sg_handle *h, int32_t *E_out, int32_t *Q_out, uintptr_t stream);

/* n_mcs MCS as sg_run_mcs, then the observables of the resulting state into HOST
 * buffers as sg_measure_async (same buffers, staging and waiting rules).  When the
 * sweep kernel holds both one-word chains of a sample in each CTA (n_chains == 2,
 * n_temps <= 32, the fused exchange, a launch shape of two words per CTA) the
 * measurement runs inside the last MCS's launch, from the lattice in shared memory;
 * otherwise the two calls run one after the other.  SG_EINVAL if n_mcs < 1. */
sg_status sg_run_mcs_measure_async(sg_handle *h, int32_t n_mcs, int32_t *E_out, int32_t *Q_out, uintptr_t stream);

/* Wait for every copy that sg_measure_async has enqueued on the handle's copy stream.
 * sg_restore and sg_destroy wait for them too before they touch or release anything. */
sg_status sg_measure_wait(sg_handle *h);

/* Round trips in temperature (Sec. 2.3: lowest -> highest -> lowest), counted after
 * every exchange pass t = 1, 2, ...: a replica at the lowest slot whose last extreme was
 * the highest completes a trip that began at its previous arrival at the lowest slot.
 * n_out[s][c] = trips completed in chain c of sample s, sum_out[s][c] = their total
 * duration in passes (host buffers; synchronises).  SG_EINVAL unless the handle was
 * made with track_trips = 1. */
sg_status sg_trips(sg_handle *h, uint32_t *n_out, uint64_t *sum_out, uintptr_t stream);

/* General couplings (SG_COUPLINGS_FIXED).  The couplings start at 0; this call sets them
 * from a host array J[s][i][mu] (int32, canonical site order i = x + L0 (y + L1 z), bond
 * (i, mu) joining i and i + e_mu), J = J_fixed 2^-20 with |J_fixed| <= 2^23 (else
 * SG_EINVAL), and recomputes every energy.  The Metropolis rule of these jobs: accept
 * iff dE <= 0 or r < floor(e 2^32), e an fp32 evaluation of exp(-beta dE) by Cody &
 * Waite's reduction and a Taylor series to r^6 in single IEEE operations (k_gauss.cu).
 * Energies of these jobs are int64 in units of 2^-20: sg_measure64 / sg_get_state64
 * (the int32 calls return SG_EUNSUPPORTED for them). */
sg_status sg_import_couplings_fixed(sg_handle *h, const int32_t *J_in, uintptr_t stream);
/* E by temperature slot [S][C][T] (int64, units 2^-20) and N q [S][T]; host buffers, syncs. */
sg_status sg_measure64(sg_handle *h, int64_t *E_out, int32_t *Q_out, uintptr_t stream);
/* Energies by replica [S][C][T] (int64, units 2^-20), maps and step counters; syncs. */
sg_status sg_get_state64(sg_handle *h, int64_t *E_out, int32_t *perm_out, uint64_t *steps_out, uintptr_t stream);

/* Overlap plane sums, the integer part of the Fourier modes of the overlap field behind
 * the spin-glass susceptibility and the correlation length (two-replica measurements,
 * Sec. 3): P_out[s][k][mu][x] = sum of s_i^(a) s_i^(b) (the summand of Eq. 4) over the
 * sites i with coordinate x along axis mu, a / b the chain-0 / chain-1 replicas at
 * temperature slot k; x < Lmax = the largest extent, entries x >= L_mu are 0.  Then
 * q(k e_mu) = (1/N) sum_x exp(i k x) P[mu][x].  Needs n_chains == 2 (else SG_EINVAL).
 * sg_measure_qmodes writes a host buffer and synchronises the stream;
 * sg_measure_qmodes_device writes device memory and does not. */
sg_status sg_measure_qmodes(sg_handle *h, int32_t *P_out, uintptr_t stream);
sg_status sg_measure_qmodes_device(sg_handle *h, int32_t *P_out, uintptr_t stream);

/* Spins in a plain layout, DEVICE buffers: uint8 [n_samples][n_chains][n_temps][N],
 * indexed by replica j (not slot) and site i, 1 iff s = -1.  Import recomputes the
 * energies. */
sg_status sg_export_spins(sg_handle *h, uint8_t *spins_out, uintptr_t stream);
sg_status sg_import_spins(sg_handle *h, const uint8_t *spins_in, uintptr_t stream);

/* Couplings, DEVICE buffers: int8 [n_samples][N][ndim], +-1, entry (i, mu) is the bond
 * from i to i + e_mu.  Import recomputes the energies. */
sg_status sg_export_couplings(sg_handle *h, int8_t *J_out, uintptr_t stream);
sg_status sg_import_couplings(sg_handle *h, const int8_t *J_in, uintptr_t stream);

/* Replica state into HOST buffers; synchronises `stream`.  Any pointer may be NULL.
 *   E_out     [n_samples][n_chains][n_temps]  energy of replica j (Eq. 1)
 *   perm_out  [n_samples][n_chains][n_temps]  replica at temperature slot k
 *   steps_out [3]                             t_metro, t_pt, t_houd */
sg_status sg_get_state(sg_handle *h, int32_t *E_out, int32_t *perm_out, uint64_t *steps_out,
                       uintptr_t stream);

/* Counters into HOST buffers; synchronises `stream`.  Any pointer may be NULL.
 *   near_threshold  exchange decisions with |u 2^-32 - exp(delta)| < 1e-12 (expected 0)
 *   pt_accepts      [n_temps-1] accepted exchanges per pair (k, k+1), summed over chains
 *   houdayer_sites  total sites flipped by Houdayer moves (each pair counts once) */
sg_status sg_counters(sg_handle *h, uint64_t *near_threshold, uint64_t *pt_accepts,
                      uint64_t *houdayer_sites, uintptr_t stream);

/* How often the fast screens of the fused kernels deferred to the exact rule (HOST
 * buffers; synchronises `stream`; either pointer may be NULL).  These decisions are the
 * plain fp64 / fixed-function ones in every case; the counts show that those paths ran.
 *   exchange_exact   exchange decisions (Eq. 5) of the one-warp exchanges inside the
 *                    sweep kernels whose draw u fell within the fp32 screening margin of
 *                    the threshold (or u = 0), so that exp(delta) was evaluated in fp64
 *   metropolis_band  general-coupling Metropolis draws (Sec. 2.1) that fell inside the
 *                    2^-14 band around the hardware-exp estimate of the threshold, so
 *                    that the fixed fp32 threshold floor(e 2^32) was evaluated */
sg_status sg_exact_path_counters(sg_handle *h, uint64_t *exchange_exact, uint64_t *metropolis_band,
                                 uintptr_t stream);

/* Metropolis thresholds thr[k][m-1] = min(floor(exp(-4 m beta_k) 2^32), 2^32 - 1),
 * m = 1..ndim, computed on the host in fp64 (HOST buffer [n_temps][ndim]). */
sg_status sg_thresholds(sg_handle *h, uint32_t *thr_out);

/* Launch shape of the resident sweep kernel (not part of the paper: a tuning knob).
 *   threads  CTA size: 64, 128, 256, 512 or 1024 (0 keeps the current choice)
 *   words    32-replica words of one sample held by one CTA: 1 or 2 (0 keeps);
 *            -1 streams the lattice from global memory instead of keeping it in a CTA
 *            (the path taken automatically when a word lattice does not fit)
 * Every accepted choice gives bit-identical results; a shape that does not fit the
 * lattice (shared memory, per-thread counter range, word count) is refused with
 * SG_EUNSUPPORTED and the previous shape is kept.  Host-only; no device work. */
sg_status sg_set_launch(sg_handle *h, int32_t threads, int32_t words);

/* Paired last words (a tuning knob, on by default).  For two chains whose last
 * 32-replica word holds at most 16 replicas (n_temps <= 16, or 33..48), the fused MCS
 * (sg_run_mcs without the cluster move, and batches) may hold a whole sample per CTA
 * and sweep the two chains' last words as ONE word: lanes 0..15 chain 0's, 16..31 chain
 * 1's.  Every replica draws the same Philox words and takes the same decisions, so the
 * results are bit-identical either way; the per-site work of one word is saved.  The
 * words are re-split in global memory after every launch; the unused lanes of those
 * last words (replicas >= n_temps) are then 0.
 *   on  1 allows pairing where it applies (shape, shared memory), 0 never pairs
 * SG_EINVAL for another value.  Host-only; no device work. */
sg_status sg_set_pairing(sg_handle *h, int32_t on);

/* Current launch shape: threads, words per CTA (-1: streaming path), shared memory bytes. */
sg_status sg_get_launch(sg_handle *h, int32_t *threads, int32_t *words, int32_t *smem_bytes);

/* Batches (not a step of the paper's method: a way to run many jobs at once).  The MCS
 * cycles of n_handles jobs (any mix of lattices, temperatures and sample counts) are
 * captured once into one CUDA graph, mcs_per_launch MCS per job per launch, each job a
 * branch of the graph so that the jobs' kernels run concurrently.  Each job advances
 * exactly as it would under sg_run_mcs (bit-identical results).  The handles must
 * outlive the batch and must not be used by other calls while its launches run;
 * sg_batch_create enqueues nothing, sg_batch_run enqueues n_launches graph launches
 * on `stream`. */
typedef struct sg_batch sg_batch;
sg_status sg_batch_create(sg_handle *const *handles, int32_t n_handles, int32_t mcs_per_launch,
                          uintptr_t stream, sg_batch **out);
sg_status sg_batch_run(sg_batch *b, int32_t n_launches, uintptr_t stream);
void sg_batch_destroy(sg_batch *b);

/* n_sweeps Metropolis sweeps by the streaming (global-memory) path, allocating nothing
 * and using no scratch from the handle's buffer.  The paper has no counterpart: this is
 * for callers that cannot allocate device memory -- a host framework that owns all
 * device memory and hands a job only its state, or code that runs while a CUDA graph is
 * being captured, where cudaMalloc is not allowed -- and still want a sweep whose
 * working memory is not theirs to provide.
 * Results are bit-identical to sg_sweep on the same handle.
 * Working memory: one file-scope device array in the library (about 8.9 MB, holding up
 * to 4096 (sample, word) pairs: lane-pair tables and bond sums), which every GPU that
 * loads the library keeps until the process exits.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress) with the device current; make that
 * first call before any stream capture.  The address is kept for the life of the process,
 * so the library must not outlive a reset of the device (cudaDeviceReset, or a new
 * primary context on it): after one, this call would use a stale address.  Every call
 * uses the same array and clears what must start at zero, so calls whose work overlaps
 * on the GPU (other streams, other threads, other handles) race and must be serialised
 * by the caller.
 * Errors: SG_ELIMIT if n_samples x words per site exceeds 4096 (words per site =
 * n_chains x ceil(n_temps / 32)); SG_EUNSUPPORTED for int8 spins. */
sg_status sg_sweep_streaming_static(sg_handle *h, int32_t n_sweeps, uintptr_t stream);

/* Checkpoint and resume (long runs): a checkpoint is a host blob of
 * sg_checkpoint_bytes bytes holding the parameters that fix the layout and the
 * dynamics, the temperatures, the step counters and the handle's whole device buffer.
 * sg_checkpoint writes it (synchronises the stream); sg_restore loads it into a handle
 * made with the same parameters (else SG_EINVAL), after which the job continues exactly
 * as the checkpointed one would have. */
sg_status sg_checkpoint_bytes(sg_handle *h, size_t *bytes);
sg_status sg_checkpoint(sg_handle *h, void *host_out, size_t bytes, uintptr_t stream);
sg_status sg_restore(sg_handle *h, const void *host_in, size_t bytes, uintptr_t stream);

/* Failure-detection self-test: a kernel waits (at most max_tries polls, 1..2^20) on an
 * mbarrier that nothing completes, as the kernels' waits on their bulk copies are
 * bounded.  The wait runs out, the kernel records the error and returns, and the call
 * reports SG_ETIMEOUT; the handle is then poisoned (every later call returns
 * SG_ETIMEOUT), exactly as after a copy that never landed.  No fault, trap or hang. */
sg_status sg_selftest_wait(sg_handle *h, int32_t max_tries, uintptr_t stream);

/* Measurement probe (not a step of the paper's method): the Philox work of n_sweeps
 * packed sweeps over n_sites sites of two 32-replica words each -- the draws of one
 * Philox4x32-10 word per attempt (Sec. 3), with the rounds that a sweep and a site share
 * computed once, as the sweep kernel does -- and nothing else.  Its rate, 64 n_sites
 * n_sweeps words over the time it takes, is an upper bound on the sweep's attempts per
 * ns.  Launches n_blocks CTAs of 256 threads on `stream` (enqueued only; the caller
 * times it).  `out`: DEVICE buffer of n_blocks x 256 uint32 that the kernel may write
 * (its outputs are folded into a value that is stored only if it matches a sentinel, so
 * no work is optimised away).  SG_EINVAL for sizes below 1 or a NULL buffer. */
sg_status sg_probe_philox(int32_t n_sites, int32_t n_sweeps, int32_t n_blocks, uint64_t sim_seed, uint32_t *out,
                          uintptr_t stream);

/* Free the host-side handle.  The caller frees the device buffer afterwards. */
void sg_destroy(sg_handle *h);

/* Static description of a status code. */
const char *sg_strerror(sg_status s);

#ifdef __cplusplus
}
#endif
#endif /* SGMC_H */
