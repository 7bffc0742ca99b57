/*
 * surfmcmc — C ABI of a GB300 (sm_103a) implementation of the single-temperature
 * Markov chain Monte Carlo decoder for the planar surface code of Hutter,
 * Wootton and Loss, "An efficient Markov chain Monte Carlo algorithm for the
 * surface code" (arXiv:1302.2669).
 *
 * What is computed (Sec. IV and IV.A of the paper): given the anyon
 * configuration (syndrome) of a size-L planar code under depolarizing noise
 * of rate p, sample <n>_{beta*,E}, the mean number of single-qubit errors of
 * the error chains of each equivalence class E, with Metropolis chains over
 * stabilizer moves at beta* = beta_bar = -log((p/3)/(1-p)) (Eq. 2), and
 * return the class with the smallest mean.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Geometry (Sec. II; Fig. 1 is not available, so this is the unrotated planar
 * layout): a (2L-1) x (2L-1) grid, data qubits at r+c even with index
 * q = (r(2L-1)+c)/2, n_q = 2L^2-2L+1; sigma_x generators (s-anyons) at odd r,
 * even c; sigma_z generators (p-anyons) at even r, odd c; n_stab = 2L(L-1).
 *
 * Syndrome layout: uint8 0/1 per generator, n_stab bytes per syndrome: first
 * the sigma_x generators row-major over (i=(r-1)/2, j=c/2), then the sigma_z
 * generators row-major over (i=r/2, j=(c-1)/2).
 *
 * Frame layout: a Pauli frame is two bit planes (x then z) of W = ceil(n_q/32)
 * uint32 words each; qubit q is bit q%32 of word q/32; bits past n_q are zero.
 *
 * Class code: a + 2b, a = parity of x on the column-0 qubits, b = parity of z
 * on the row-0 qubits (Sec. II identifies classes by error parities along a
 * line joining opposite boundaries).  Class k chains start at the pure error
 * times the logical that gives them class code k.
 *
 * Pointers: every buffer is owned by the caller and may be host or device
 * memory (detected per pointer).  With device pointers and a non-NULL stream
 * the call is stream-ordered and returns once the work is queued; with host
 * buffers, or stream == NULL, the call returns after the results are in the
 * caller's buffers.  The library keeps no pointer after a call returns.
 *
 * Errors: 0 on success, a negative SURFMCMC_E* code otherwise; no exception
 * crosses the ABI.  surfmcmc_last_error() gives a message for the last
 * failing call on a context.  Contexts are not thread-safe; use one per host
 * thread.
 */
#ifndef SURFMCMC_H
#define SURFMCMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SURFMCMC_OK 0
#define SURFMCMC_EINVAL (-1)    /* bad argument: L, p, sizes, NULL pointer, options */
#define SURFMCMC_ENOMEM (-2)    /* device allocation failed */
#define SURFMCMC_ECUDA (-3)     /* a CUDA call failed; see surfmcmc_last_error */
#define SURFMCMC_ENODEV (-4)    /* no such device, or not an sm_103 device */

#define SURFMCMC_MAX_L 31       /* largest code size accepted */

typedef struct surfmcmc_ctx surfmcmc_ctx;
typedef struct surfmcmc_plan surfmcmc_plan;
typedef struct surfmcmc_server surfmcmc_server;

/* Decoder options.
 *   n_classes        number of equivalence classes: 4 (planar code, Sec. II
 *                    "there are four such equivalence classes"), or 16: the
 *                    toric code on an L x L torus (L even, 2..30; decode,
 *                    decode_ex and decode_ti only).  Torus layout: the
 *                    periodic 2L x 2L grid, 2L^2 qubits at r+c odd with
 *                    index r L + (c div 2); syndrome = 2L^2 bytes, the stars
 *                    (sigma_x generators at (2i, 2j)) row-major, then the
 *                    plaquettes (sigma_z at (2i+1, 2j+1)); class code
 *                    a1 + 2 a2 + 4 b1 + 8 b2 with a1 (a2) the x parity on
 *                    column 0, odd rows (row 0, odd columns) and b1 (b2)
 *                    the z parity on row 1, even columns (column 1, even
 *                    rows); colours 0/1 stars, 2/3 plaquettes by (i+j)
 *                    parity.  Pure error: defects of each type paired in
 *                    syndrome order, joined towards increasing c to the
 *                    partner's column, then towards increasing r.
 *   chains_per_class R >= 1 independent replica chains per class;
 *                    n_classes * R <= 1024.
 *   n_sweeps         sweeps per chain; one sweep proposes every generator
 *                    once, colour by colour (the four non-overlapping groups
 *                    of Sec. V), so n_sample = n_sweeps * n_stab per chain.
 *   burn_in          sweeps before sampling starts (the paper uses none).
 *   beta_scale       beta* = beta_scale * beta_bar (Sec. IV.A sets beta* =
 *                    beta_bar, i.e. 1.0); 0 <= beta_scale <= +infinity.
 *   lanes_per_bundle GPU tuning knob: threads sharing one 32-chain bundle, a
 *                    power of two in 2..32, or 0 for automatic.  Results do
 *                    not depend on it.
 *   anneal_stages    S >= 0.  With S > 0 the burn-in prepares the start
 *                    (Sec. IV wants each chain to start near the low-energy
 *                    configurations of its class, since heating up from them
 *                    is fast and cooling down is slow): burn-in sweeps
 *                    floor(jB/S) .. floor((j+1)B/S)-1 (B = burn_in) run at
 *                    beta* (a0 + (1 - a0) j / S), j = 0..S-1; needs
 *                    S <= burn_in and S <= 64.
 *   anneal_beta0     a0 in (0, 1], the first stage's fraction of beta*.
 *   scan             0: sweeps as above.  1: Sec. IV as written, one
 *                    generator picked at random per step, g = floor(w0
 *                    n_stab / 2^32), applied when Delta n <= 0 or w1 <
 *                    T[Delta n], with Philox4x32-10 words (w0, w1) of
 *                    counter (syndrome id, chain k R + r, sweep t, step)
 *                    and key (seed_lo, seed_hi); a sweep is n_stab steps and
 *                    n is summed after every step, so the sample count is
 *                    n_stab R (n_sweeps - burn_in) per class.  Needs
 *                    lanes_per_bundle 0 or 32.
 *   noise            0: depolarizing (Sec. IV), p in (0, 3/4]: n = number of
 *                    qubits with an error, e^{-beta_bar} = (p/3)/(1-p).
 *                    1: independent bit and phase flips (Sec. IV.B), p in
 *                    (0, 1/2] the probability of each: n = bit flips + phase
 *                    flips, e^{-beta_bar} = p/(1-p) (the paper finds beta* =
 *                    0.85 beta_bar best, beta_scale = 0.85).
 *                    2: general Pauli channel (Eq. 1) with integer energies
 *                    pauli_energy = (eX, eY, eZ) in 1..8: p_X : p_Y : p_Z :
 *                    p_I = r^eX : r^eY : r^eZ : 1, p in (0, 3/4] the total
 *                    error probability, r = e^{-beta_bar} the root of
 *                    (1 - p)(r^eX + r^eY + r^eZ) = p after 100 halvings of
 *                    [0, 1]; n = the summed energies of the qubits' Paulis.
 *                    Needs scan = 1 (the sweep kernels are specialised to
 *                    the two models above).
 *   pauli_energy     (eX, eY, eZ) of noise 2; ignored otherwise. */
typedef struct {
    int32_t n_classes;
    int32_t chains_per_class;
    uint32_t n_sweeps;
    uint32_t burn_in;
    double beta_scale;
    int32_t lanes_per_bundle;
    int32_t anneal_stages;
    double anneal_beta0;
    int32_t scan;
    int32_t noise;
    int32_t pauli_energy[3];
} surfmcmc_opts;

/* Fills opts with K = 4, R = 4, 2000 sweeps, no burn-in, beta* = beta_bar,
 * no annealing (a0 = 1), automatic tuning. */
void surfmcmc_default_opts(surfmcmc_opts* opts);

/* Creates a context bound to CUDA device `device`; *ctx receives it.
 * Returns ENODEV if the device does not exist or is not compute capability
 * 10.3, EINVAL if ctx is NULL. */
int surfmcmc_create(surfmcmc_ctx** ctx, int device);

/* Releases the context and the device scratch it owns.  NULL is ignored. */
void surfmcmc_destroy(surfmcmc_ctx* ctx);

/* Static description of an error code. */
const char* surfmcmc_strerror(int code);

/* Message of the last failing call on ctx ("" if none). */
const char* surfmcmc_last_error(const surfmcmc_ctx* ctx);

/* Synthetic input: n syndromes of i.i.d. depolarizing noise (Eq. 1 with
 * p_x = p_y = p_z = p/3, Sec. II) with ids id0 .. id0+n-1.
 *   syndromes  [n][n_stab] uint8 out.
 *   true_class [n] int32 out (may be NULL): class code of the sampled error,
 *              the answer of a perfect decoder.
 * Qubit q of syndrome id takes word q%4 of the Philox4x32-10 block with
 * counter (id, q/4, 0, 0) and key (seed_lo, seed_hi ^ 0x53594E44); with
 * tau = floor((p/3) 2^32): u < tau X, u < 2tau Y, u < 3tau Z, else I.
 * EINVAL: L outside 2..SURFMCMC_MAX_L, p outside [0, 0.75], n < 0,
 * id0 + n > 2^32, NULL syndromes with n > 0. */
int surfmcmc_gen_syndromes(surfmcmc_ctx* ctx, uint64_t seed, uint32_t id0, int64_t n, int32_t L,
                           double p, uint8_t* syndromes, int32_t* true_class, void* stream);
/* As surfmcmc_gen_syndromes for the error model noise (0: depolarizing, p in
 * [0, 3/4]; 1: independent bit and phase flips with probability p in [0, 1]
 * each: sigma_x on qubit q iff word 2 (q mod 2) < floor(p 2^32), sigma_z iff
 * word 2 (q mod 2) + 1 < floor(p 2^32), of the Philox block with counter
 * (id, q div 2, 1, 0) and the same key). */
int surfmcmc_gen_syndromes_noise(surfmcmc_ctx* ctx, uint64_t seed, uint32_t id0, int64_t n, int32_t L, double p,
                                 int32_t noise, uint8_t* syndromes, int32_t* true_class, void* stream);

/* Errors of a general Pauli channel with probabilities pX, pY, pZ (>= 0,
 * sum <= 3/4): u = word q mod 4 of the Philox block with counter (id, q div
 * 4, 2, 0) (same key); X if u < floor(pX 2^32), Y if u < floor((pX + pY)
 * 2^32), Z if u < floor((pX + pY + pZ) 2^32), else I.  Outputs as for
 * surfmcmc_gen_syndromes. */
int surfmcmc_gen_syndromes_pauli(surfmcmc_ctx* ctx, uint64_t seed, uint32_t id0, int64_t n, int32_t L, double px,
                                 double py, double pz, uint8_t* syndromes, int32_t* true_class, void* stream);

/* Depolarizing errors on the toric code (n_classes = 16 layout above, even L
 * in 2..30): the same per-qubit draws as surfmcmc_gen_syndromes with the
 * torus's 2L^2 qubits; syndromes [n][2L^2], true_class = 4-bit class code. */
int surfmcmc_gen_syndromes_toric(surfmcmc_ctx* ctx, uint64_t seed, uint32_t id0, int64_t n, int32_t L, double p,
                                 uint8_t* syndromes, int32_t* true_class, void* stream);

/* Start state (Sec. IV: one syndrome-compatible error per class, Sec. III's
 * boundary rule): the pure error joins every anyon to its nearer absorbing
 * boundary by a straight string (s-anyons up/down, p-anyons left/right,
 * ties up/left).
 *   syndromes [n][n_stab] uint8 in.
 *   frames    [n][2][W] uint32 out: the pure error e0.
 *   e0_class  [n] int32 out (may be NULL): class code of e0.
 * EINVAL as above. */
int surfmcmc_start_frames(surfmcmc_ctx* ctx, const uint8_t* syndromes, int64_t n, int32_t L,
                          uint32_t* frames, int32_t* e0_class, void* stream);

/* The single-temperature decoder (Sec. IV.A, algorithm C) on n syndromes.
 *   syndromes     [n][n_stab] uint8 in.
 *   p             depolarizing rate, 0 < p <= 0.75.
 *   opts          see surfmcmc_opts (NULL: defaults).
 *   seed, id0     randomness key and id of syndrome 0; syndrome i uses id
 *                 id0 + i, so a result does not depend on the batch it is in.
 *   out_class     [n] int32 out: class code with the smallest sum of sampled
 *                 n (lowest code on ties).
 *   out_class_sum [n][4] uint64 out (may be NULL): S_k, the sum over the R
 *                 chains of class k of n sampled after every colour phase of
 *                 every sweep t >= burn_in (4 R (n_sweeps - burn_in) samples);
 *                 sweeps t count from 0 through the burn-in.
 *   out_log_ratio [n][4] double out (may be NULL): -beta_bar (<n>_k -
 *                 min_k <n>_k), a single-temperature proxy of log Z_k/Z_best.
 * Randomness: Philox4x32-10 with key (seed_lo, seed_hi); acceptance of a
 * proposal with Delta n = d > 0 iff u < floor(r*^d 2^32), r* = e^{-beta*},
 * u assembled from bit planes as described for surfmcmc_decode_ex.
 * EINVAL: bad L, p, n, options or NULL required pointers. */
int surfmcmc_decode(surfmcmc_ctx* ctx, const uint8_t* syndromes, int64_t n, int32_t L, double p,
                    const surfmcmc_opts* opts, uint64_t seed, uint32_t id0, int32_t* out_class,
                    uint64_t* out_class_sum, double* out_log_ratio, void* stream);

/* surfmcmc_decode with per-chain state in and out, for resuming a run and for
 * checking single chains (Sec. IV: the chain of each class, its sampled n
 * and its accepted moves).  Runs sweeps sweep_begin .. opts->n_sweeps-1.
 *   init_frames     [n][C][2][W] uint32 in (may be NULL): chain states at
 *                   sweep_begin; NULL starts from the start frames (then
 *                   sweep_begin must be 0).  C = 4 * chains_per_class; chain
 *                   c has class c / chains_per_class.
 *   init_chain_sum  [n][C] uint64 in (may be NULL = zeros): sums so far.
 *   out_chain_sum   [n][C] uint64 out (may be NULL).
 *   out_chain_n     [n][C] int32 out (may be NULL): final n of every chain.
 *   out_chain_frames[n][C][2][W] uint32 out (may be NULL): final states.
 *   out_chain_accepts [n][C] uint64 out (may be NULL): accepted proposals
 *                   of every chain in the sweeps run by this call (annealing
 *                   sweeps included); counting them costs 4.6 KB of shared
 *                   memory per block and a few operations per proposal.
 * The per-chain uniform: G = min(32, smallest power of two >= C) is the plane
 * width, chain c has group w = c/G and lane b = c%G.  For the proposal of
 * the m-th generator of colour col (row-major order within the colour) in
 * sweep t of syndrome id s, Philox blocks j = 0, 1, .. with counter
 * (s, t, (col<<24)|m, (w<<8)|j) form a bit stream (block j = bits 128j..,
 * word i of a block = the next 32 bits, least significant first); plane k is
 * stream bits kG .. kG+G-1 and u_c = sum_k bit(kG+b) 2^(31-k). */
int surfmcmc_decode_ex(surfmcmc_ctx* ctx, const uint8_t* syndromes, int64_t n, int32_t L, double p,
                       const surfmcmc_opts* opts, uint64_t seed, uint32_t id0, uint32_t sweep_begin,
                       const uint32_t* init_frames, const uint64_t* init_chain_sum, int32_t* out_class,
                       uint64_t* out_class_sum, double* out_log_ratio, uint64_t* out_chain_sum,
                       int32_t* out_chain_n, uint32_t* out_chain_frames, uint64_t* out_chain_accepts,
                       void* stream);

/* Ragged batches: syndromes of different code sizes (and sweep counts) in one
 * call, with the algorithm of surfmcmc_decode applied to every item; item i
 * gives exactly what surfmcmc_decode gives for it alone (same L_i, sweeps,
 * id), since the randomness is keyed by the syndrome id.
 *   syndromes     concatenated rows in item order, item i has n_stab(L_i)
 *                 bytes (layout as for surfmcmc_decode).
 *   Ls            [n] int32 code sizes (host or device).
 *   n_sweeps      [n] uint32 sweeps per item (host or device), or NULL for
 *                 opts->n_sweeps; item i's burn-in is
 *                 floor(n_sweeps_i * opts->burn_in / opts->n_sweeps) and its
 *                 annealing stages are those of opts.
 *   ids           [n] uint32 syndrome ids, or NULL for id0 + i.
 *   out_*         as for surfmcmc_decode, in item order.
 * Items are grouped by (L, n_sweeps); one call takes at most 8 distinct
 * groups.  All groups run in the same persistent kernel launches (one per
 * annealing stage plus one), largest work first.  EINVAL: bad sizes, more than
 * 8 groups, a burn-in shorter than the annealing stages, or as for
 * surfmcmc_decode. */
int surfmcmc_decode_ragged(surfmcmc_ctx* ctx, const uint8_t* syndromes, const int32_t* Ls, const uint32_t* n_sweeps,
                           int64_t n, double p, const surfmcmc_opts* opts, uint64_t seed, const uint32_t* ids,
                           uint32_t id0, int32_t* out_class, uint64_t* out_class_sum, double* out_log_ratio,
                           void* stream);

/* A captured ragged batch: the device work of surfmcmc_decode_ragged for a
 * fixed shape (Ls, n_sweeps, options, seed) and fixed DEVICE buffers is
 * recorded once as a CUDA graph; every surfmcmc_plan_launch replays it on
 * the current contents of those buffers (refill syndromes and ids between
 * launches).  The plan owns its scratch (allocated at creation) and must not
 * outlive ctx.  Launches of one plan must not overlap on the GPU. */
int surfmcmc_ragged_plan_create(surfmcmc_ctx* ctx, const int32_t* Ls, const uint32_t* n_sweeps, int64_t n, double p,
                                const surfmcmc_opts* opts, uint64_t seed, const uint8_t* syndromes,
                                const uint32_t* ids, uint32_t id0, int32_t* out_class, uint64_t* out_class_sum,
                                double* out_log_ratio, surfmcmc_plan** plan);
int surfmcmc_plan_launch(surfmcmc_plan* plan, void* stream);
void surfmcmc_plan_destroy(surfmcmc_plan* plan);

/* Autotuning of the launch shape (the paper has no counterpart): times the
 * sweep kernel on n_probe synthetic size-L syndromes for `sweeps` sweeps at
 * rate p for every supported lanes_per_bundle (2, 4, 8, 16, 32: threads per
 * 32-chain bundle, hence 32/lanes bundles and 32 x 32/lanes chains per warp,
 * and ceil(generators per colour / lanes) proposals per lane and colour)
 * combined with every cap of 6, 5, 4, 3 resident blocks per multiprocessor
 * (the persistent grid; a cap above what fits counts as no cap), and records
 * the fastest pair in ctx for later calls with lanes_per_bundle = 0 and the
 * same (L, chains_per_class); ragged calls use the entry of their heaviest
 * size.  Results never depend on the choice.  *best_lanes and
 * *best_blocks_per_sm receive it, ms[SURFMCMC_TUNE_LANES][SURFMCMC_TUNE_BLOCKS]
 * the timings in milliseconds (NaN where the shape does not fit); any of the
 * three may be NULL.  EINVAL for bad arguments. */
#define SURFMCMC_TUNE_LANES 5
#define SURFMCMC_TUNE_BLOCKS 4
int surfmcmc_autotune(surfmcmc_ctx* ctx, int32_t L, int32_t chains_per_class, double p, int64_t n_probe,
                      uint32_t sweeps, int32_t* best_lanes, int32_t* best_blocks_per_sm, double* ms);

/* Thermodynamic integration (Eq. 6: log Z_E(beta) = -int_0^beta <n>_{b,E} db
 * + n_stab log 2; Sec. IV: the integral by Simpson's rule; Sec. IV.A: 21
 * equidistant temperatures).  For grid point j = 1..n_beta-1 the chains run
 * at beta_j = beta* j/(n_beta-1) with the options of surfmcmc_decode (burn-in
 * annealing scaled to beta_j) and randomness key seed + j; <n> at beta = 0 is
 * 3/4 n_q (Sec. IV.A).  I_k = h/3 sum_j w_j <n>_{beta_j,k} (w = 1,4,2,..,4,1,
 * h = beta* / (n_beta-1)) in double precision, summed in order j = 0..n_beta-1.
 *   n_beta        odd, 3..129 (21 in the paper).
 *   out_class     [n] int32 out: argmin_k I_k (= argmax Z_k), lowest on ties.
 *   out_log_z     [n][4] double out (may be NULL): log Z_k - max_k log Z_k
 *                 = -(I_k - min_k I_k).
 *   out_mean      [n][4][n_beta] double out (may be NULL): <n>_{beta_j,k}.
 * EINVAL as for surfmcmc_decode, or for an even/out-of-range n_beta, an
 * infinite beta*, or no sampled sweeps. */
int surfmcmc_decode_ti(surfmcmc_ctx* ctx, const uint8_t* syndromes, int64_t n, int32_t L, double p,
                       const surfmcmc_opts* opts, int32_t n_beta, uint64_t seed, uint32_t id0, int32_t* out_class,
                       double* out_log_z, double* out_mean, void* stream);

/* Request serving (the paper has no counterpart): continuous batching of
 * single syndromes of mixed sizes.  Callers submit requests from any thread;
 * a scheduler thread takes pending requests in arrival order into batches
 * (at most max_batch; a partial batch waits at most max_wait_us for company),
 * admits a batch when one of `slots` slots is free and its device scratch
 * fits memory_budget next to the batches in flight (0 = no budget), and
 * decodes it with surfmcmc_decode_ragged on the slot's own context and
 * stream; slots run concurrently, so requests that arrive while others are on
 * the GPU join the next free slot.  Each slot's scratch is sized at creation
 * for max_batch syndromes of size max_L, so serving allocates nothing.  A
 * request's randomness is keyed by its id (the syndrome id of
 * surfmcmc_decode), so its result is the same alone or in any batch. */
typedef struct {
    int32_t max_batch;      /* >= 1 */
    int32_t slots;          /* 1..64 batches in flight */
    int32_t max_L;          /* largest code size accepted, 2..SURFMCMC_MAX_L */
    int64_t memory_budget;  /* bytes of device scratch for the batches in flight; 0 = unlimited */
    double max_wait_us;     /* longest wait of a partial batch */
} surfmcmc_server_opts;

/* Defaults: 256 per batch, 4 slots, max_L = SURFMCMC_MAX_L, no budget, 200 us. */
void surfmcmc_server_default_opts(surfmcmc_server_opts* opts);

/* Creates a server on `device` for rate p with the decoder options `opts`
 * (opts->n_sweeps and opts->burn_in set each request's burn-in fraction as in
 * surfmcmc_decode_ragged) and randomness key `seed`.  EINVAL, ENOMEM, ENODEV. */
int surfmcmc_server_create(int device, double p, const surfmcmc_opts* opts, uint64_t seed,
                           const surfmcmc_server_opts* server_opts, surfmcmc_server** server);

/* Queues one request: n_stab(L) syndrome bytes (host memory, copied), L <=
 * max_L, n_sweeps >= 1.  EINVAL for bad arguments or after shutdown began. */
int surfmcmc_server_submit(surfmcmc_server* server, uint32_t request_id, int32_t L, uint32_t n_sweeps,
                           const uint8_t* syndrome);

/* Takes up to max_results finished requests (waiting up to wait_us for the
 * first): ids[k], classes[k] (a negative SURFMCMC_E* code if the batch
 * failed), class_sums[4k..4k+3] and latency_us[k] (submission to completion)
 * (the last two may be NULL); *n_out receives the count.  Host buffers. */
int surfmcmc_server_poll(surfmcmc_server* server, int64_t max_results, uint32_t* ids, int32_t* classes,
                         uint64_t* class_sums, double* latency_us, int64_t* n_out, int32_t wait_us);

/* Counters since creation: requests admitted to batches, batches launched,
 * times admission had to wait for memory (a free slot and waiting requests,
 * but not even one request's scratch fits the budget next to the batches in
 * flight; counted once per wait), requests waiting now. */
int surfmcmc_server_stats(surfmcmc_server* server, int64_t* admitted, int64_t* batches, int64_t* memory_stalls,
                          int64_t* pending);

/* Finishes every submitted request, then releases the server. */
void surfmcmc_server_destroy(surfmcmc_server* server);

/* Instrumentation (the paper has no counterpart): with enable != 0 every
 * later decode call records a pair of CUDA events on its stream around its
 * sweep kernel.  surfmcmc_sweep_time waits for the recorded events, returns
 * in *ms the summed sweep-kernel time in milliseconds and in *launches the
 * number of sweep launches since the previous query (either pointer may be
 * NULL), and clears the record.  EINVAL for a NULL ctx. */
int surfmcmc_set_timing(surfmcmc_ctx* ctx, int enable);
int surfmcmc_sweep_time(surfmcmc_ctx* ctx, double* ms, int64_t* launches);

/* Allocation-free decoding.  The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory, for example a
 * host program whose device memory is already entirely reserved by another
 * allocator, or one that runs under a fixed device-memory budget.  It does the
 * same work as surfmcmc_decode with the same results, but calls no cudaMalloc,
 * cudaFree or allocating library routine and needs no context: its scratch
 * (pure errors, their class codes and the per-chain sums) is one fixed
 * SURFMCMC_NOALLOC_SCRATCH_BYTES array in the library's device memory, which
 * every GPU that loads the library holds until the process exits.
 *   Buffers: syndromes, out_class and (if not NULL) out_class_sum and
 *   out_log_ratio must be device memory of the current device; the layouts
 *   and results are those of surfmcmc_decode.  opts->lanes_per_bundle,
 *   opts->anneal_stages, opts->scan and opts->noise must be 0.  With stream == NULL the call returns after the results are
 *   written; otherwise it is stream-ordered.
 *   Scratch: the call needs surfmcmc_noalloc_scratch_needed(n, L, R) bytes;
 *   a batch needing more than SURFMCMC_NOALLOC_SCRATCH_BYTES is rejected with
 *   EINVAL before any work is queued (split it into smaller batches).
 *   Sharing: every call on a device uses the same array and leaves its
 *   contents behind; the call initialises all of it that it reads.  Calls
 *   whose work overlaps on the GPU (other host threads, or other streams not
 *   ordered with this one) race on the array and give wrong results.
 *   Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   Errors: EINVAL for bad arguments, host pointers, buffers of another
 *   device or an oversized batch,
 *   ECUDA if a CUDA call fails. */
#define SURFMCMC_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
size_t surfmcmc_noalloc_scratch_needed(int64_t n, int32_t L, int32_t chains_per_class);
int surfmcmc_decode_noalloc(const uint8_t* syndromes, int64_t n, int32_t L, double p, const surfmcmc_opts* opts,
                            uint64_t seed, uint32_t id0, int32_t* out_class, uint64_t* out_class_sum,
                            double* out_log_ratio, void* stream);

/* ------------------------------------------------------------------------
 * Early-stop network.  The paper has no counterpart: a small convolutional
 * network that reads a syndrome and predicts the posterior of its 4 classes,
 * used to stop the chains of syndromes whose class is already clear.
 *   Input: the syndrome of a size-L code as two L x L maps, channel 0 the
 *   sigma_x generators ((L-1) x L, row i column j = syndrome entry i L + j,
 *   last row zero), channel 1 the sigma_z generators (L x (L-1), row i column
 *   j = entry (L-1) L + i (L-1) + j, last column zero).
 *   Network: five 3x3 convolutions with zero padding, 2 -> 64 -> 64 -> 64 ->
 *   64 -> 2 channels, bias, ReLU after the first four.  Weights and
 *   activations are bfloat16 (round to nearest even), sums float32 (tensor
 *   cores; the last layer only at the 2L outputs the readout reads, on the
 *   CUDA cores).
 *   Readout: class k = a + 2b, a (b) the parity of an error's sigma_x
 *   (sigma_z) part on qubit column (row) 0.  With e0 the decoder's pure error
 *   (surfmcmc_start_frames) of class code a0 + 2 b0 and m = (L-1) div 2, the
 *   last layer's channel 0 at map position (i, m) and channel 1 at (m, j) are
 *   the logits s of flips of E + e0 on qubits (2i, 2m) and (2m, 2j) (E + e0
 *   has the same parities on the middle column/row as on column/row 0);
 *   M_x = prod_i -tanh(s_i / 2) (likewise M_z), clipped to +-(1 - 1e-6);
 *   log p_k = log((1 + (-1)^(a xor a0) M_x) / 2) + log((1 + (-1)^(b xor b0)
 *   M_z) / 2).
 *   Parameters: surfmcmc_cnn_n_params() (= 113154) float32 values, layer
 *   after layer, each layer W[co][kh][kw][ci] then b[co].
 *   Training: mean over the batch of the cross entropy -sum_k q_k log p_k
 *   against soft targets q, Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * A network object belongs to one context's device; it is not thread-safe.
 * Every entry point returns EINVAL for bad arguments, ENOMEM/ECUDA for CUDA
 * failures, and ECUDA if a tensor-core pipeline wait timed out (the device
 * stays usable).  Pointers may be host or device memory unless stated. */
typedef struct surfmcmc_cnn surfmcmc_cnn;

int64_t surfmcmc_cnn_n_params(void);

/* Allocates the parameters (all zero until set), the optimizer state and the
 * activations of up to max_batch (1..2^20) syndromes of size L (3..31). */
int surfmcmc_cnn_create(surfmcmc_ctx* ctx, int32_t L, int64_t max_batch, surfmcmc_cnn** out);
void surfmcmc_cnn_destroy(surfmcmc_cnn* net);

/* Copies n_params floats in / out; set_params also clears the Adam state. */
int surfmcmc_cnn_set_params(surfmcmc_cnn* net, const float* params);
int surfmcmc_cnn_get_params(surfmcmc_cnn* net, float* params);

/* Log-probabilities [n][4] of n syndromes [n][2L(L-1)] (any n >= 0; batches
 * of max_batch internally).  Returns after the results are written. */
int surfmcmc_cnn_forward(surfmcmc_cnn* net, const uint8_t* syndromes, int64_t n, float* out_logprob,
                         void* stream);

/* Loss (1 float) and its gradient with respect to the parameters (n_params
 * floats; either output may be NULL) for 1 <= n <= max_batch syndromes and
 * soft targets [n][4].  Returns after the results are written. */
int surfmcmc_cnn_gradient(surfmcmc_cnn* net, const uint8_t* syndromes, const float* targets, int64_t n,
                          float* out_loss, float* out_grad, void* stream);

/* One Adam step with learning rate lr on the gradient of the batch.  With
 * device inputs and out_loss NULL or device memory the call is stream-ordered
 * and does not wait; surfmcmc_cnn_status then reports a timed-out wait. */
int surfmcmc_cnn_train_step(surfmcmc_cnn* net, const uint8_t* syndromes, const float* targets, int64_t n,
                            float lr, float* out_loss, void* stream);
int surfmcmc_cnn_status(surfmcmc_cnn* net, void* stream);

/* Bound on every pipeline wait of the network kernels, in polls of the
 * mbarrier (0 restores the default, 2^22).  A wait that reaches the bound
 * gives up: the block stops its other roles, waits out the copies and
 * tensor-core operations it has in flight, frees its tensor memory and
 * exits; the device error flag then makes the call (or the next
 * surfmcmc_cnn_status) return ECUDA with "a pipeline wait timed out" in
 * surfmcmc_last_error, and clears the flag.  Outputs of such a call are
 * undefined.  Small bounds exist to exercise that path; the default is far
 * above the duration of any wait of a working pipeline.  EINVAL for a NULL
 * net. */
int surfmcmc_cnn_set_wait_limit(surfmcmc_cnn* net, uint32_t polls);

/* Decoding with early stop (the paper has no counterpart).  The same chains
 * as surfmcmc_decode with opts (same seed, ids id0 + i, same sweeps), run in
 * chunks: checkpoints at burn_in + k chunk_sweeps (k = 1, 2, ...) below
 * n_sweeps, and n_sweeps.  At a checkpoint the decision so far is argmin_k of
 * the class sums; syndrome i stops there when the network (net, built for
 * this L) is confident, log p_a - max_{k != a} log p_k > tau for its argmax
 * a, and a equals that decision.  The others continue; at n_sweeps every
 * syndrome stops.  A syndrome that never stops early gets exactly the
 * results of surfmcmc_decode; tau = +infinity reproduces surfmcmc_decode.
 *   reorder 1 (budget reordering): at the first checkpoint every syndrome
 *   that goes on has the chains of the network's two least likely classes
 *   continue as further replicas of its two most likely ones (classes
 *   ranked by log p, ties to the lower class: a, b, c, d; slot c R + r takes
 *   the state of slot a R + r, slot d R + r that of b R + r, and keeps its
 *   own random stream); the sums of c and d are frozen there.  From then on
 *   the decision is the class with the smallest mean: a and b over their own
 *   chains since the burn-in plus their replicas since that checkpoint, c
 *   and d over the frozen sums (exact comparison, lowest class on ties), and
 *   out_class_sum holds those sums.  reorder 0: no reordering.
 *   out_class [n] int32: the decision at the syndrome's stop.
 *   out_class_sum [n][4] uint64 (may be NULL): the class sums at the stop.
 *   out_sweeps [n] uint32 (may be NULL): the sweeps run (the stop).
 * Buffers may be host or device memory.  The call waits for the device at
 * every checkpoint (to size the next chunk).  EINVAL: bad arguments, a net
 * for another L, chunk_sweeps 0, tau NaN. */
int surfmcmc_decode_early(surfmcmc_ctx* ctx, surfmcmc_cnn* net, const uint8_t* syndromes, int64_t n, int32_t L,
                          double p, const surfmcmc_opts* opts, uint32_t chunk_sweeps, float tau, int32_t reorder,
                          uint64_t seed,
                          uint32_t id0, int32_t* out_class, uint64_t* out_class_sum, uint32_t* out_sweeps,
                          void* stream);

/* Soft targets for training: targets[i][k] = softmax_k(log_ratio[i][k])
 * (float32) from the [n][4] double log-ratios of a decode.  Both buffers are
 * device memory of the current device; stream-ordered.  EINVAL for n < 0,
 * NULL or host pointers. */
int surfmcmc_cnn_soft_targets(const double* log_ratio, int64_t n, float* targets, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SURFMCMC_H */
