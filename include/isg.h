/*
 * isg.h -- C-ABI of the GB300 (sm_103a) checkerboard Metropolis engine for the
 * 3D Edwards-Anderson +-J spin glass (Lulli, Bernaschi, Parisi, arXiv:1411.0127).
 *
 * Model and update rule
 *   H = -sum_<ik> J_ik s_i s_k on an L x L x L periodic cubic lattice (Sec. 1,
 *   Eq. 1), J_ik = +-1 with probability 1/2 (Eq. 2).  A sweep updates the "red"
 *   sites (x+y+z even) and then the "blue" ones (Sec. 1); an attempt with u
 *   unsatisfied bonds has dE = 12 - 4u and flips when u >= 3 or when its own
 *   32-bit draw d satisfies d < floor(2^32 exp(-beta dE)) (Sec. 4).  Spins and
 *   couplings are stored one bit each (Sec. 4 bit map: s = +1 -> 1,
 *   J = -1 -> 1), colour by colour, in row-major bit planes.
 *
 * Conventions of every call
 *   - Every function returns ISG_OK (0) or a negative ISG_ERR_* code and never
 *     throws.  isg_last_error() returns a message for the calling thread.
 *   - `cuda_stream` is a cudaStream_t owned by the caller (NULL = the legacy
 *     default stream).  Calls marked "async" only enqueue work on it; calls
 *     marked "sync" enqueue, then wait for that stream.
 *   - Device memory comes from the allocator installed with isg_set_allocator
 *     (cudaMalloc/cudaFree by default) and stays owned by the handle until
 *     isg_destroy / isg_batch_destroy.
 *   - Host pointers are plain pageable or pinned host memory owned by the
 *     caller; they are only accessed during the call.
 *   - Site order of host arrays: i = x + L*y + L*L*z.  Coupling arrays hold
 *     3*N values, direction-major: [d][i], d = 0 (x), 1 (y), 2 (z), where
 *     J[d][i] joins site i and its +d neighbour.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef ISG_H
#define ISG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ISG_OK = 0,
    ISG_ERR_ARG = -1,      /* invalid argument (nothing was changed) */
    ISG_ERR_NOMEM = -2,    /* the allocator returned NULL */
    ISG_ERR_CUDA = -3,     /* a CUDA runtime call failed (message has the name) */
    ISG_ERR_TIMEOUT = -4,  /* a bounded device wait gave up (device error word) */
    ISG_ERR_MISMATCH = -5, /* two handles do not describe the same sample */
    ISG_ERR_STATE = -6     /* call not valid in the handle's current state */
};

enum { ISG_RNG_MINSTD = 0, ISG_RNG_MT19937 = 1, ISG_RNG_PARISI_RAPUANO = 2 };

typedef struct isg_sim isg_sim;
typedef struct isg_batch isg_batch;

/* ---------------------------------------------------------------- setup --- */

/* Create one lattice (sync on the legacy default stream).
 *   L          even, 4 <= L <= 2048 (else ISG_ERR_ARG)
 *   seed_J     coupling sample: J_d(i) from the SplitMix64 counter hash
 *   seed_spin  initial spins and the RNG streams of this replica
 *   beta       inverse temperature, > 0, may be +INFINITY; 0, negative or NaN
 *              give ISG_ERR_ARG (beta = 0 would need a threshold of 2^32)
 *   rng_kind   ISG_RNG_MINSTD (Sec. 3 Lehmer generator), ISG_RNG_MT19937 or
 *              ISG_RNG_PARISI_RAPUANO (Sec. 3: ira[i] = ira[i-24] + ira[i-55],
 *              draw ira[i] ^ ira[i-61]; seeded with ira[j] = SplitMix64(v, j)
 *              >> 32 for j < 61 and ira[60] made odd, v the stream's seed word)
 * Cites: Eq. 1-2 (model), Sec. 4 (threshold table), Sec. 3 (generators). */
int isg_create(int L, uint64_t seed_J, uint64_t seed_spin, double beta, int rng_kind,
               isg_sim **out);

/* As isg_create, but the RNG streams are seeded from seed_rng instead of
 * seed_spin.  Sec. 4's asynchronous multispin coding shares one draw per site
 * among the samples of a word; each of those samples follows exactly the
 * trajectory of an isg_create2 handle with the common seed_rng. */
int isg_create2(int L, uint64_t seed_J, uint64_t seed_spin, uint64_t seed_rng, double beta, int rng_kind,
                isg_sim **out);

/* Free every device buffer of the handle (NULL is ignored). */
void isg_destroy(isg_sim *h);

/* Install the device allocator used by every later allocation: alloc(size, ctx)
 * returns device memory or NULL, free(ptr, ctx) releases it.  Passing NULL for
 * both restores cudaMalloc/cudaFree.  Handles keep the allocator they were
 * created with. */
int isg_set_allocator(void *(*alloc)(size_t size, void *ctx),
                      void (*free_fn)(void *ptr, void *ctx), void *ctx);

/* Message of the last failed call made by this thread ("" if none). */
const char *isg_last_error(void);

/* Geometry of a handle: L, word width in bits (32 or 64), words per row and
 * colour, number of RNG streams and rows per stream.  Any pointer may be NULL. */
int isg_info(const isg_sim *h, int *L, int *word_bits, int *words_per_row,
             int64_t *streams, int64_t *rows_per_stream);

/* ---------------------------------------------------------------- sweep --- */

/* Enqueue n full sweeps (red pass, then blue pass) on cuda_stream (async).
 * n >= 0.  The fused energy change of every accepted flip is accumulated on the
 * device (read with isg_tracked_energy).  Sec. 1 (colour order), Sec. 4 (rule).
 * Calls of at least 8 sweeps on MINSTD and MT19937 lattices with more RNG
 * streams than such a launch has warps (see isg_sweep_info) run their passes
 * in persistent launches of up to 64 sweeps: a stream starts a colour pass
 * once the streams that hold its neighbouring rows have finished the previous
 * pass.  Those waits are bounded.  If one gives up, the remaining passes of the
 * launch are skipped, so are those of later multi-pass launches of the handle
 * until the error has been read, and the next isg_energy / isg_tracked_energy
 * returns ISG_ERR_TIMEOUT (once: reading it clears it); the configuration is
 * then off its trajectory.  Every form gives the same trajectory. */
int isg_sweep(isg_sim *h, int64_t n, void *cuda_stream);

/* How isg_sweep launches this handle's passes on the current device (host
 * only): *passes_per_launch = 128 when calls of 8 or more sweeps run in
 * persistent launches of up to 64 sweeps (a MINSTD or MT19937 lattice with at
 * least as many RNG streams as the launch has warps, plus a margin: L >= ~640
 * on a GB300), else 1 (one launch per colour pass, as for every call of fewer
 * sweeps and every Parisi-Rapuano lattice). */
int isg_sweep_info(const isg_sim *h, int *passes_per_launch);

/* Same as isg_sweep but with the plain per-colour kernel: one stream per warp,
 * draws and bit logic in separate phases, no persistence.  Results are
 * bit-identical to isg_sweep; it is kept as the comparison kernel. */
int isg_sweep_plain(isg_sim *h, int64_t n, void *cuda_stream);

/* Number of sweeps done since creation (or since the loaded checkpoint). */
int isg_sweeps_done(const isg_sim *h, int64_t *n);

/* ------------------------------------------------------------- measures --- */

/* E = -sum_<ik> J_ik s_i s_k from scratch (sync).  Eq. 1. */
int isg_energy(isg_sim *h, int64_t *E, void *cuda_stream);

/* Initial energy plus the sum of accepted dE of every sweep so far (sync on
 * the stream of the last sweep).  Equals isg_energy when the kernels are right. */
int isg_tracked_energy(isg_sim *h, int64_t *E);

/* Q = sum_i s^a_i s^b_i (sync).  a and b must have the same L and seed_J, else
 * ISG_ERR_MISMATCH.  q = Q/N is the replica overlap. */
int isg_overlap(const isg_sim *a, const isg_sim *b, int64_t *Q, void *cuda_stream);

/* Zobrist hash H = XOR over sites with s_i = +1 of SplitMix64(0xA54FF53A5F1D36F1, i)
 * (sync).  Equal configurations give equal hashes. */
int isg_hash(const isg_sim *h, uint64_t *H, void *cuda_stream);

/* Copy the spins to host_out as int8 +-1 in site order (sync).  n must be
 * at least L^3 (else ISG_ERR_ARG). */
int isg_read_spins(const isg_sim *h, int8_t *host_out, size_t n, void *cuda_stream);

/* Overwrite the spins from a host int8 array of +-1 in site order (sync); the
 * tracked energy restarts from the new configuration.  Any value other than
 * +1 or -1 gives ISG_ERR_ARG and changes nothing. */
int isg_write_spins(isg_sim *h, const int8_t *host_in, size_t n, void *cuda_stream);

/* Spins as packed bits in site order (sync): bit (i & 7) of byte i >> 3 of
 * host_out is site i, 1 meaning s = +1 (Sec. 4 bit map).  nbytes must be at
 * least ceil(L^3 / 8) (else ISG_ERR_ARG).  The compact form of isg_read_spins:
 * one eighth of the bytes to move. */
int isg_read_spins_packed(const isg_sim *h, uint8_t *host_out, size_t nbytes, void *cuda_stream);

/* Streaming exchange, asynchronous: enqueue on cuda_stream, in this order,
 *   1. if in != NULL: overwrite the spins from packed bits (the format of
 *      isg_read_spins_packed, Sec. 4 bit map; every bit pattern is a valid
 *      configuration) and restart the energy bookkeeping (Eq. 1) from the new
 *      configuration, on the device: with sweeps > 0 the first colour pass
 *      counts the configuration's unsatisfied bonds before its flips (every
 *      bond has one site of each colour), otherwise a separate popcount pass;
 *   2. `sweeps` sweeps (as isg_sweep);
 *   3. if out != NULL: the packed spins into out;
 *   4. if E_out != NULL: the tracked energy (int64, as isg_tracked_energy) into
 *      the host word *E_out.
 * Nothing is synchronised.  in must stay valid and unchanged, and out / E_out
 * must not be read, until the stream has passed this call (an event or
 * cudaStreamSynchronize).  With pinned host memory the copies run on the copy
 * engines and overlap work on other streams: a loop over a few handles on a few
 * streams keeps the SMs sweeping while configurations move in and out (the
 * end-to-end benchmark does this).  nbytes is the size of in and of out (at
 * least ceil(L^3 / 8) when either is given).  The first call with in or out
 * allocates a staging buffer of ceil(L^3 / 32) words that the handle keeps.
 * ISG_ERR_ARG for a NULL handle, sweeps < 0 or short buffers. */
int isg_exchange_async(isg_sim *h, const uint8_t *in, uint8_t *out, size_t nbytes, int64_t sweeps,
                       long long *E_out, void *cuda_stream);

/* Overwrite the spins from packed bits in the format of isg_read_spins_packed
 * (sync; every bit pattern is a valid configuration); the tracked energy
 * restarts.  nbytes >= ceil(L^3 / 8) (else ISG_ERR_ARG and nothing changes). */
int isg_write_spins_packed(isg_sim *h, const uint8_t *host_in, size_t nbytes, void *cuda_stream);

/* Copy the couplings to host_out as int8 +-1, [d][i] (sync); n >= 3 L^3. */
int isg_read_couplings(const isg_sim *h, int8_t *host_out, size_t n, void *cuda_stream);

/* Overwrite the couplings from a host int8 +-1 array [d][i] (sync); the
 * tracked energy restarts.  Other values give ISG_ERR_ARG. */
int isg_write_couplings(isg_sim *h, const int8_t *host_in, size_t n, void *cuda_stream);

/* ----------------------------------------------------------- checkpoint --- */

/* Serialise the whole state (spins, couplings, RNG streams with their
 * positions, sweep count, energy bookkeeping, parameters) into host_buf (sync).
 * With host_buf == NULL only *n is set to the size needed.  If *n is smaller
 * than needed, ISG_ERR_ARG and *n = size needed. */
int isg_save(const isg_sim *h, void *host_buf, size_t *n, void *cuda_stream);

/* Create a new handle from a buffer written by isg_save (sync).  A corrupt or
 * truncated buffer gives ISG_ERR_ARG.  Continuing the loaded handle gives the
 * same trajectory, bit for bit, as continuing the saved one. */
int isg_load(const void *host_buf, size_t n, isg_sim **out);

/* --------------------------------------------------------------- batch --- */

/* Many disorder samples swept together, as the paper fills the GPU with many
 * coded samples (Sec. 2, samples k; Sec. 4 results against k).  Sample s has
 * size L[s] (even, 4..2048), couplings from seed_J[s], inverse temperature
 * beta[s] > 0, and two replicas whose spins and streams come from seed_spin[2s]
 * and seed_spin[2s+1]; all samples use rng_kind.  Every replica follows exactly
 * the trajectory of a lone isg_create handle with the same arguments.
 * Sync; ISG_ERR_ARG on a bad size, beta or kind (nothing allocated). */
int isg_batch_create(int n, const int *L, const uint64_t *seed_J, const uint64_t *seed_spin,
                     const double *beta, int rng_kind, isg_batch **out);

/* Free the batch and all its replicas (NULL is ignored). */
void isg_batch_destroy(isg_batch *b);

/* Number of samples, of work bundles (streams of small lattices packed 32 per
 * bundle; with the pass engines, shapes 4 and 5: the (lattice, stream) items) and of
 * spin-flip attempts per sweep of the whole batch. */
int isg_batch_info(const isg_batch *b, int *samples, int *bundles, int64_t *attempts_per_sweep);

/* Execution configuration of the batch's launches, the space the autotuner
 * (paper_1411_0127_gb300/autotune.py) searches.  No configuration changes a
 * result: every replica follows its own trajectory whatever the bundles, so
 * all of them give bit-identical states.  Replicas keep their spins and
 * couplings in 64-bit words whatever L.
 *   shape     CTA shape: 0 = one CTA of 32 warps per SM, 1 = one of 24,
 *             2 = one of 16, 3 = two of 16 (the "tile": warps sweeping a bundle),
 *             all persistent over a whole sweep group; 4 and 5 = the pass
 *             engines, no bundles: 4-warp CTAs take (lattice, stream) items of
 *             a colour pass by ticket, longest streams first; with 4 each
 *             colour pass of all replicas is one launch, with 5 one persistent
 *             launch per sweep group takes the items pass by pass and an item
 *             waits (bounded) only until its own lattice has finished the
 *             previous pass (capacity and resident do not apply to 4 and 5:
 *             every stream's state is loaded and stored around each pass)
 *   capacity  streams per packed bundle of small lattices, 1 .. warps of the
 *             shape; 0 = the shape's warps
 *   resident  1: the generator state of a bundle that fits in the CTA stays in
 *             shared memory / registers for a whole launch; 0: it is loaded and
 *             stored around every colour pass
 *   words_per_lane  words of a row group each lane updates, 1 or 2
 *             (a row group is 32 * words_per_lane words: its draws are made in
 *             one run, and 2 halves the groups per pass)
 * Synchronises the device, re-plans the bundles and drops the captured graph;
 * ISG_ERR_ARG for an unknown shape, a capacity above the shape's warps, a
 * resident flag other than 0/1 or words_per_lane other than 1/2.  The default
 * is (0, 32, 1, 1). */
int isg_batch_set_config(isg_batch *b, int shape, int capacity, int resident, int words_per_lane);

/* The current configuration (any pointer may be NULL). */
int isg_batch_get_config(const isg_batch *b, int *shape, int *capacity, int *resident, int *words_per_lane);

/* Handle of replica i (0 <= i < 2n; replicas 2s, 2s+1 belong to sample s).  The
 * handle stays owned by the batch: use it with the measuring, reading and
 * checkpoint calls, never with isg_destroy. */
int isg_batch_member(isg_batch *b, int i, isg_sim **out);

/* Enqueue `sweeps` sweeps of every replica (async).  The work runs as persistent
 * launches of group_sweeps sweeps (<= 0 picks 64): the CTAs of the execution
 * configuration (isg_batch_set_config) take task after task; the group
 * launch is captured once into a CUDA graph and replayed; a remainder of
 * sweeps % group_sweeps is launched directly.  A task is a bundle of RNG
 * streams for all of the launch's sweeps or, for a bundle longer than a sixth
 * of the average work per CTA, one of up to 8 consecutive parts of them; a
 * part waits (bounded, about 4 s) for the previous part, run by another CTA.
 * If such a wait ever gives up, the next isg_batch_measure / isg_batch_tracked
 * returns ISG_ERR_TIMEOUT once (the bundle's lattices then missed sweeps). */
int isg_batch_run(isg_batch *b, int64_t sweeps, int group_sweeps, void *cuda_stream);

/* Energies from scratch of the 2n replicas (E[2s], E[2s+1]) and overlaps
 * Q[s] = sum_i s^a_i s^b_i of the two replicas of each sample (sync).  Either
 * pointer may be NULL. */
int isg_batch_measure(isg_batch *b, int64_t *E, int64_t *Q, void *cuda_stream);

/* Tracked energies (2n) and Zobrist hashes (2n) of the replicas (sync).  Either
 * pointer may be NULL. */
int isg_batch_tracked(isg_batch *b, int64_t *E, uint64_t *H, void *cuda_stream);

/* -------------------------------------------------------------- server --- */

/* A request server for quench jobs (one lattice, isg_create arguments, and a
 * number of sweeps) that serves them by continuous batching: jobs are admitted
 * as they arrive, in arrival order, while their device memory fits
 * hbm_budget_bytes and fewer than max_active jobs (<= 0: 4096) are on the
 * device; every quantum of quantum_sweeps sweeps (<= 0: 64) sweeps all active
 * jobs at once (the streams of all active jobs of one generator kind as items
 * of one launch per colour pass, longest first; lattices are held in 64-bit
 * words); finished jobs release their memory at once.  The paper has no serving layer; each job
 * follows exactly the trajectory of a lone isg_create handle. */
typedef struct isg_server isg_server;
int isg_server_create(size_t hbm_budget_bytes, int quantum_sweeps, int max_active, isg_server **out);
void isg_server_destroy(isg_server *s);

/* Queue a job arriving arrival_s seconds after isg_server_run starts; *job_id
 * numbers jobs 0, 1, ... in submission order.  Thread-safe.  ISG_ERR_ARG for
 * invalid lattice arguments, sweeps < 0, or a job larger than the budget. */
int isg_server_submit(isg_server *s, int L, uint64_t seed_J, uint64_t seed_spin, double beta, int rng_kind,
                      int64_t sweeps, double arrival_s, int64_t *job_id);

/* Serve every queued job, in real time, until all have finished (sync).
 * time_limit_s > 0 stops with ISG_ERR_TIMEOUT once that many seconds have
 * passed with jobs unfinished. */
int isg_server_run(isg_server *s, double time_limit_s);

/* Outcome of one job: status 2 = finished (1 active, 0 waiting, < 0 the
 * ISG_ERR_* that failed it), energy from scratch, Zobrist hash, and arrival,
 * admission and completion times in seconds from the start of the run.
 * Latency = done - arrival.  Any output pointer may be NULL. */
int isg_server_job(const isg_server *s, int64_t id, int *status, int64_t *E, uint64_t *H, double *arrival_s,
                   double *admit_s, double *done_s);

/* Statistics of the last run: quanta, spin-flip attempts, wall time, time with
 * work on the device, peak active jobs and peak device bytes admitted. */
int isg_server_stats(const isg_server *s, int64_t *iterations, int64_t *attempts, double *wall_s, double *busy_s,
                     int *peak_active, size_t *peak_bytes);

/* ---------------------------------------------- asynchronous multispin --- */

/* Asynchronous multispin coding (Sec. 4): 32 systems of the same size L share
 * every word, bit b of the word at a site belonging to system b, and ONE draw
 * per site serves all 32 (the paper's cond masks are all ones or all zeros).
 * System b has couplings from seed_J[b] and spins from seed_spin[b] (arrays of
 * 32); the draws come from streams seeded by seed_rng, with the stream
 * partition and site -> (stream, draw) map of a single lattice.  Hence system b
 * follows, bit for bit, the trajectory of
 * isg_create2(L, seed_J[b], seed_spin[b], seed_rng, beta, rng_kind): the 32
 * systems are correlated through their shared draws, as the paper notes.
 * L even, 4 <= L <= 1024; beta > 0.  Device memory: 8 planes of L^3/2 words
 * (4 L^3 bytes) plus the streams, from cudaMalloc.  Sync; ISG_ERR_ARG on a bad
 * argument (nothing allocated), ISG_ERR_CUDA on a device error. */
typedef struct isg_amsc isg_amsc;
int isg_amsc_create(int L, const uint64_t *seed_J, const uint64_t *seed_spin, uint64_t seed_rng, double beta,
                    int rng_kind, isg_amsc **out);

/* Free the ensemble (NULL is ignored; synchronises the device first). */
void isg_amsc_destroy(isg_amsc *m);

/* Enqueue n sweeps of all 32 systems on cuda_stream (async): per colour one
 * persistent launch in which a warp takes stream after stream and each lane
 * updates one site word with its own draw.  ISG_ERR_ARG for n < 0. */
int isg_amsc_sweep(isg_amsc *m, int64_t n, void *cuda_stream);

/* Facts of an ensemble (any output pointer may be NULL): its size L, its
 * number of RNG streams and rows per stream (the single-lattice partition),
 * and the form of the sweep kernel on the current device: 0 = the chunked form
 * (rows of a multiple of 128 sites per colour, i.e. L a multiple of 256: each
 * lane updates four consecutive sites of a 128-site chunk with 16-byte loads,
 * the next chunk's words in flight while the current one is computed), else
 * the site-strided form with `form` blocks of 32 sites in flight per lane: 8
 * when the ensemble has fewer than 16 streams per SM (latency bound), 4
 * otherwise.  Host only. */
int isg_amsc_info(const isg_amsc *m, int *L, int64_t *streams, int64_t *rows_per_stream, int *form);

/* Energies E[b] = -sum J s s' of the 32 systems (Eq. 1), counted bit-parallel
 * on the device (sync on cuda_stream).  E must hold 32 entries. */
int isg_amsc_energies(isg_amsc *m, int64_t *E, void *cuda_stream);

/* Spins of system `sample` (0..31) as +-1 in site order i = x + L y + L^2 z
 * into host_out (n >= L^3; sync).  Uses an L^3-byte temporary device buffer. */
int isg_amsc_read_spins(const isg_amsc *m, int sample, int8_t *host_out, size_t n, void *cuda_stream);

/* ----------------------------------------------------------- benchmark --- */

/* Device-API generator benchmark of Sec. 3 (Table MYTEST: produce numbers on
 * the device and count the odd ones).  `streams` streams of rng_kind, seeded as
 * the streams of a lattice with seed_spin = seed, each produce n consecutive
 * raw outputs (MT19937: the tempered word; MINSTD: the state x) with the warp
 * engines of the flip kernels.  Sync; *odd = number of odd outputs, *gen_ms
 * (may be NULL) = device time of the generation kernel alone.  Allocates its
 * own temporary buffers. */
int isg_rng_count_odd(int rng_kind, uint64_t seed, int64_t streams, int64_t n, uint64_t *odd, double *gen_ms);

/* Integer issue-rate microbenchmark (a measurement tool, not part of the
 * method): the 32-bit integer operations per second the GPU sustains on
 * independent chains of mode 0 = LOP3 and IMAD alternating, 1 = LOP3 only,
 * 2 = IMAD only, over all SMs (sync; about a millisecond).  These are the
 * measured counterparts of the derived integer peak of the flip kernel's
 * roofline. */
int isg_int_rate(int mode, double *ops_per_s);

/* ------------------------------------------------------- no allocation --- */

/* The same energy that isg_energy returns, for callers that must not allocate
 * device memory when they ask for it: real-time loops that cannot take the
 * device-wide synchronisation an allocation may cause, and processes (or
 * embedding runtimes with their own memory pool) that work inside a
 * device-memory budget fixed up front, where any cudaMalloc outside that
 * budget is an error.  The paper has no counterpart to this call; it exists
 * only for those callers.
 *
 * Async: enqueues two kernels on cuda_stream and writes E (int64) to the
 * caller's device pointer dev_E; it calls no cudaMalloc, cudaFree or other
 * allocating routine.  Its partial sums live in a fixed array of 8192 int64
 * (64 KiB) compiled into the library, held by every device that loads it until
 * the process exits.  Lattices needing more partial sums (L > 1448) give
 * ISG_ERR_ARG.  All calls share that array: calls whose kernels overlap on the
 * GPU (e.g. on two streams) race and give wrong results.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current) and keeps it for the life of the process; make
 * that first call before any stream capture begins.  The kept address assumes
 * the device's context lives as long as the process: after cudaDeviceReset
 * (or a released and re-created primary context) the call must not be used. */
int isg_energy_static_scratch(const isg_sim *h, long long *dev_E, void *cuda_stream);

/* ------------------------------------------------------------- testing --- */

/* Run the device flip rule on n stencils (sync).  code[j] bits: 0 = spin bit,
 * 1..6 = neighbour spin bits, 7..12 = coupling bits (Sec. 4 bit map; bond k
 * joins the site and neighbour k).  draw[j] is the attempt's 32-bit draw.
 * Writes flip[j] = 1 when the kernel's bit logic flips the spin, and u[j] = its
 * count of unsatisfied bonds.  thr = {thr1, thr2, thr3}.  Host arrays. */
int isg_stencil_decisions(const uint16_t *code, const uint32_t *draw, int64_t n,
                          const uint32_t thr[3], uint8_t *flip, uint8_t *u);

/* First n draws of stream t of the handle's generator, from its current
 * position, without advancing it (sync); host_out gets the 32-bit draws. */
int isg_peek_draws(const isg_sim *h, int64_t t, int64_t n, uint32_t *host_out);

/* Make the next multi-pass sweep launch of the handle (see isg_sweep) wait for
 * a pass that never comes in its second pass, so that its bounded waits run out
 * (about a second) and the error path can be tested: the launch skips its
 * remaining passes and the next energy read returns ISG_ERR_TIMEOUT.
 * ISG_ERR_STATE if the handle's sweeps do not run as multi-pass launches. */
int isg_sweep_test_stall(isg_sim *h);

/* Make one wait of the batch's launches wait for something that never comes,
 * so that its bounded wait runs out (about 4 s per launch) and the error path
 * can be tested: with the bundle shapes, the last task waits for its own done
 * flag; with the group pass engine (shape 5), the pass-1 items of the lattice
 * with the fewest streams wait for one completed item too many.  The next
 * isg_batch_set_config restores the plan.  ISG_ERR_STATE with shape 4 (its
 * launches have no waits) or if a bundle plan has fewer than two tasks. */
int isg_batch_test_stall(isg_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* ISG_H */
