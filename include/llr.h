/*
 * llr.h -- C ABI of the GB300 (sm_103a) library for the LLR density-of-states
 * method applied to 4-D compact U(1) lattice gauge theory.
 *
 * Paper: K. Langfeld, B. Lucini, R. Pellegrini, A. Rago, "An efficient
 * algorithm for numerical computations of continuous densities of states",
 * arXiv:1509.08391.  Equations are cited by their printed numbers
 * (eq. (2.30) = the under-relaxed Robbins-Monro update of Sec. 2.2).
 *
 * Conventions shared by every entry point
 *   - Return value: 0 on success, a negative LLR_ERR_* code on failure;
 *     llr_last_error() then gives a message (per calling thread).
 *   - "host" pointers are read or written only during the call; the caller
 *     owns them.  "device" pointers are CUDA device memory on the handle's
 *     device, owned by the caller, accessed in stream order on the handle's
 *     stream (the call returns before the work finishes).
 *   - A handle owns all the lattice state it allocates (link angles, per
 *     lattice energies, windows and counters) until llr_destroy.  Calls on
 *     one handle are not thread safe; they are ordered on the stream given to
 *     llr_init_lattice (NULL = the legacy default stream).
 *   - The slope convention follows eq. (2.4): a = d ln rho / dE, and the
 *     restricted ensemble has weight exp(-a E) on the closed window
 *     E_lo <= E <= E_lo + dE (eqs. (2.13)-(2.14)).  In the physical range a < 0
 *     and the canonical coupling is beta = -a.
 *   - Link angles are float32 in [-pi, pi); E = sum over plaquettes of
 *     cos(theta_P) (Sec. 3.1, beta factored out).  The canonical host layout
 *     of a lattice's links is index mu * V + s, with V = L^4 and site
 *     s = ((x3 L + x2) L + x1) L + x0.
 */
#ifndef LLR_H
#define LLR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LLR_OK 0
#define LLR_ERR_ARG (-1)      /* invalid argument or configuration           */
#define LLR_ERR_CUDA (-2)     /* a CUDA runtime call failed                  */
#define LLR_ERR_WINDOW (-3)   /* the approach phase did not reach the window */
#define LLR_ERR_TIMEOUT (-4)  /* a bounded device wait ran out               */
#define LLR_ERR_NUMERIC (-5)  /* NaN or infinity in a, E or an accumulator   */

typedef struct llr_ctx *llr_handle;

/* Configuration of a batch of independent (interval, replica) chains.
 * All arrays are host arrays of length n_lattices. */
typedef struct {
    int n_lattices;
    const int *L;             /* lattice side, even, 2 <= L <= 64              */
    const double *E_lo;       /* window lower edge E_k (absolute action)       */
    const double *dE;         /* window width dE > 0                            */
    const int *interval_id;   /* Philox key word 0 is seed_lo ^ interval_id     */
    const int *replica_id;    /* Philox key word 1 is seed_hi ^ replica_id      */
    uint64_t seed;
    int n_or;                 /* overrelaxation passes per heat-bath pass (>=0) */
    int accept_block;         /* B: links per window-accept block, 1..32, 2^k   */
    double beta_up;           /* approach heat-bath beta while E < E_lo         */
    double beta_dn;           /* approach heat-bath beta while E > E_lo + dE    */
    int max_approach;         /* approach sweeps at init; 0 = no approach       */
} llr_config;

/* Create a handle: allocate the lattices in device memory, hot start every
 * link uniformly on [-pi, pi) (Haar measure, Sec. 3.1) from Philox, compute
 * the energies, then (if cfg->max_approach > 0) run llr_approach.
 * cuda_stream: a cudaStream_t or NULL.  Errors: LLR_ERR_ARG (bad config),
 * LLR_ERR_CUDA, LLR_ERR_WINDOW (approach failed; the handle is still
 * returned in *out and must be destroyed). */
int llr_init_lattice(llr_handle *out, const llr_config *cfg, void *cuda_stream);

/* Drive every lattice that is outside its window into it: composite sweeps
 * at a = -beta_up (E below the window) or a = -beta_dn (E above), accepting
 * only moves that do not increase the distance to the window, until E lies
 * in the window after a sweep (the paper does not describe this step).
 * sweeps_out: host int[n_lattices] or NULL.  Synchronous.
 * Errors: LLR_ERR_WINDOW if a lattice is still outside after max_sweeps. */
int llr_approach(llr_handle h, int max_sweeps, int *sweeps_out);

/* n_sweeps composite sweeps at fixed slopes a (host double[n_lattices]),
 * each one heat-bath pass plus n_or overrelaxation passes restricted to the
 * window (Sec. 2.4: the importance-sampling update of Algorithm 1 with the
 * window imposed after the proposal), followed by a fresh plaquette sum.
 * Window rule, applied block by block in link order to the running energy
 * E (int64 fixed point, 2^-32, fed by the float32 dE of every move): a
 * heat-bath block is taken iff dist(E + dE) <= dist(E), dist the distance
 * from the closed window; an overrelaxation block (a reflection, which keeps
 * E in exact arithmetic) is taken iff E + dE lies in the window or E does
 * not, and a reflection with |dE| > 2^-14 is refused.  Inside the window both
 * are the indicator of eq. (2.13).
 * If measure != 0, dE_sum_out (host double[n_lattices], nullable) receives
 * the sum over these sweeps of E - E_lo - dE/2 (eq. (2.16)).  Synchronous. */
int llr_sweep(llr_handle h, const double *a, int n_sweeps, int measure, double *dE_sum_out);

/* One pass of a composite sweep for every lattice, without the energy
 * resync and without advancing the sweep counter: kind 0 = heat-bath at the
 * slopes a (host double[n_lattices]), kind 1 = overrelaxation (a may be
 * NULL), kind 2 = the multicanonical heat-bath pass of llr_muca_sweep (a is
 * ignored; needs llr_set_muca_weight).  Each selected checkerboard class (bit c of class_mask selects
 * class c = 2 mu + parity; 0xFF = the whole pass, in class order) draws its
 * proposals and accepts them in link order with the window rule of
 * llr_sweep.  kind 3 = the end of a composite sweep: the running energy is
 * re-synchronised with the fresh plaquette sum and the sweep counter
 * advances (a and class_mask ignored), so heat-bath classes, overrelaxation
 * passes and kind 3 in the order of llr_sweep reproduce its sweeps bit for
 * bit.  Synchronous. */
int llr_pass(llr_handle h, int kind, const double *a, int class_mask);

/* One Robbins-Monro iteration for every lattice (Algorithm 1, eq. (2.30)):
 * n_therm + n_meas composite sweeps at a, <<dE>> = mean over the last n_meas
 * sweeps of E - E_lo - dE/2, then a <- a + 12 <<dE>> / (dE^2 (rm_index + 1)).
 * a_inout: host double[n_lattices]; dE_mean_out: host double[n_lattices] or
 * NULL.  The host buffers are copied to and from the device inside the call.
 * Synchronous.  Errors: LLR_ERR_NUMERIC if a lattice produced a NaN. */
int llr_rm_step(llr_handle h, int n_therm, int n_meas, int rm_index, double *a_inout,
                double *dE_mean_out);

/* The same iteration with device buffers and no synchronisation: a_in and
 * a_out (may alias) and dE_mean_out (nullable) are device double[n_lattices].
 * All lattices advance in one launch on the handle's stream, so the call can
 * be captured in a CUDA graph.  A bounded wait that runs out is reported by
 * the next llr_status (or any other synchronous call on the handle). */
int llr_rm_step_dev(llr_handle h, int n_therm, int n_meas, int rm_index, const double *a_in,
                    double *a_out, double *dE_mean_out);

/* n_steps Robbins-Monro iterations (Algorithm 1's loop over n) of every
 * lattice, as replays of one captured CUDA graph (reset of the work queue,
 * the persistent kernel, and an increment of a device step counter): step k
 * uses rm_index0 + k in eq. (2.30).  a_dev: device double[n_lattices], a^(n)
 * in, a^(n + n_steps) out; hist_dev: device double[n_steps][n_lattices] of
 * a after each step, or NULL.  Asynchronous on the handle's stream.  The
 * graph is captured on the first call and reused while the arguments stay
 * the same.  A bounded wait that runs out in any replay is reported by the
 * next llr_status (or any other synchronous call on the handle); once one has
 * run out, the remaining sweeps of every replay that would wait skip at once. */
int llr_rm_run(llr_handle h, int n_therm, int n_meas, int rm_index0, int n_steps, double *a_dev,
               double *hist_dev);

/* The plain per-interval form of the same iteration, kept as the reference
 * point of the batched form: lattices are processed one after another with
 * one kernel launch per pass, per energy resync and per update (no batching,
 * no graph).  Same arguments and results as llr_rm_step.  Synchronous. */
int llr_rm_step_plain(llr_handle h, int n_therm, int n_meas, int rm_index, double *a_inout,
                      double *dE_mean_out);

/* Weight of the multicanonical run (Sec. 2.6, eq. (2.50)): W(E) = 1/rho~(E),
 * with ln rho~ the piecewise-linear density of eq. (2.10) on n contiguous
 * intervals of width de starting at e0 (ln rho~ = 0 at e0, slope a[k] inside
 * interval k) and continued beyond the first / last interval with their
 * slopes (the tails of eq. (2.50) at the micro-canonical beta_1, beta_2).
 * a0 is the slope of the heat-bath proposals (any value; Metropolis-Hastings
 * corrects it, and a0 near the slopes keeps the acceptance high).  a: host
 * double[n].  Copied to the device; applies to every lattice of the handle.
 * Errors: LLR_ERR_ARG for n < 1, de <= 0 or a non-finite value. */
int llr_set_muca_weight(llr_handle h, int n, double e0, double de, const double *a, double a0);

/* n_sweeps multicanonical composite sweeps of every lattice (Sec. 2.6):
 * a heat-bath pass whose proposals (the conditional at slope a0, the same
 * draws as the restricted heat-bath) are taken in link order with
 * probability min(1, exp(a0 dE - (ln rho~(E + dE) - ln rho~(E)))) (uniform
 * from Philox counter (link, sweep, 12, 0)), n_or overrelaxation passes
 * (they keep E, so any weight of E accepts them), and the fresh-energy
 * resync.  No window is imposed.  E_out: host double[n_sweeps][n_lattices],
 * the energy after each sweep, or NULL.  Synchronous.
 * Errors: LLR_ERR_ARG if no weight was set. */
int llr_muca_sweep(llr_handle h, int n_sweeps, double *E_out);

/* One round of replica exchange between overlapping intervals (Sec. 2.5).
 * For each pair (I1, I2) = (pairs[2k], pairs[2k+1]) of lattice indices: if
 * the tracked energies of both current configurations lie in the common part
 * of the two closed windows, the configurations are exchanged with the
 * Metropolis probability min(1, exp((a[I1] - a[I2]) (E_C1 - E_C2))).  The
 * decision uses a 53-bit uniform from Philox keyed by I1's key, counter
 * (0, round, 13, 0); pass a different round to every call.  An exchange
 * moves the link angles and the tracked energy; the window, slope, Philox
 * key, sweep counter and statistics stay with the lattice index.
 *   pairs: host int[2 n_pairs]; every lattice appears at most once and both
 *     lattices of a pair have the same L.  a: host double[n_lattices], the
 *     current slopes a^(n).  accepted_out: host int[n_pairs] (1 = exchanged)
 *     or NULL.  Synchronous.
 * Errors: LLR_ERR_ARG for an index out of range, a repeated lattice, pairs
 * of different L, n_pairs < 0 or > n_lattices / 2, or a non-finite slope. */
int llr_replica_exchange(llr_handle h, int n_pairs, const int *pairs, const double *a,
                         uint32_t round, int *accepted_out);

/* Fresh energies E = sum_P cos(theta_P) of every lattice, accumulated in
 * FP64 from the float32 angles (Sec. 3.1).  E_out: host double[n_lattices]. */
int llr_energy(llr_handle h, double *E_out);

/* The tracked energies that the window test uses (after the last resync).
 * E_out: host double[n_lattices]. */
int llr_tracked_energy(llr_handle h, double *E_out);

/* Copy one lattice's links to / from a host float[4 L^4] in the canonical
 * layout (index mu * V + s).  llr_set_links also sets that lattice's tracked
 * energy to the FP64 plaquette sum of the new angles. */
int llr_get_links(llr_handle h, int lattice, float *out);
int llr_set_links(llr_handle h, int lattice, const float *in);

/* Composite-sweep counter of a lattice (Philox counter word 1). */
int llr_get_sweep_counter(llr_handle h, int lattice, uint32_t *out);
int llr_set_sweep_counter(llr_handle h, int lattice, uint32_t value);

/* Per-lattice statistics, host double[n_lattices][8]: heat-bath accepted,
 * heat-bath proposed, overrelaxation accepted, overrelaxation proposed,
 * sampler attempt caps, max |tracked - fresh| energy at a resync (since the
 * last reset), composite sweeps done, status (0 or an LLR_ERR_* code).
 * reset != 0 clears the counters afterwards. */
int llr_stats(llr_handle h, double *out, int reset);

/* Per-lattice status words (0 = fine); host int[n_lattices].  Returns
 * LLR_ERR_TIMEOUT if, in any batched launch since the last synchronous call,
 * a bounded device wait for a lattice's previous sweep ran out (that sweep
 * and the later ones of the launch that would have waited were skipped);
 * reading it clears it. */
int llr_status(llr_handle h, int *out);

/* Reconstruction of ln rho at the interval centres by the trapezium rule
 * (eqs. (2.6), (2.7)): ln_rho[0] = 0, ln_rho[k+1] = ln_rho[k] + (c[k+1] - c[k])
 * (a[k] + a[k+1]) / 2.  centres (ascending), a, ln_rho_out: host double[n].
 * Computed in FP64 on the device. */
int llr_reconstruct_lnrho(int n, const double *centres, const double *a, double *ln_rho_out);

/* Action observables from the reconstructed density (eqs. (2.46), (2.47)) at each
 * of n_beta couplings: ln Z, <E>, <E^2>, in FP64 log-space on the device.
 * Centres must be equally spaced (weight = spacing).  All host arrays. */
int llr_observables(int n, const double *centres, const double *a, int n_beta,
                    const double *beta, double *lnZ_out, double *E_out, double *E2_out);

/* Largest number of interval centres llr_observables_noalloc accepts. */
#define LLR_NOALLOC_MAX_CENTRES 65536

/* llr_observables for callers that cannot allocate device memory, such as a
 * host application that hands out all device memory from its own
 * preallocated pool, or code that must not call cudaMalloc/cudaFree while it
 * runs (they synchronise the device).  It computes the same ln Z, <E>, <E^2>
 * without any allocation: the intermediate ln rho lives in a fixed device
 * array of LLR_NOALLOC_MAX_CENTRES doubles (512 KiB) that every GPU loading
 * this library keeps until the process exits.  The paper has no counterpart
 * of this entry point.
 *   centres, a: device double[n] (centres equally spaced and ascending: they
 *     are not checked, they stay on the device); beta: device double[n_beta];
 *   lnZ_out, E_out, E2_out: device double[n_beta]; cuda_stream: a
 *     cudaStream_t or NULL.  The call only enqueues work on that stream.
 *   Errors: LLR_ERR_ARG if n is outside 1..LLR_NOALLOC_MAX_CENTRES or a
 *     pointer is NULL; LLR_ERR_CUDA if the set-up or a launch fails.
 * Every call looks up the device address of the array in the current
 * device's context (cudaGetSymbolAddress, with that device current).  The
 * first call on a device may be the one that loads this library's device
 * code there, which is when the 512 KiB array is allocated by the CUDA
 * runtime; make that first call before any stream capture.
 * Every call reuses the same array and leaves its last contents there; calls
 * whose work overlaps on the GPU (different streams, or different host
 * threads on one device) race on it and must be serialised by the caller. */
int llr_observables_noalloc(int n, const double *centres, const double *a, int n_beta,
                            const double *beta, double *lnZ_out, double *E_out, double *E2_out,
                            void *cuda_stream);

/* Location of the specific-heat peak C_V = <E^2> - <E>^2 (Sec. 3.4) in
 * [beta_lo, beta_hi]: a scan over n_grid couplings, then golden-section
 * refinement to |interval| < tol, all on the device in FP64.
 * out: host double[2] = {beta_c, C_V(beta_c)}. */
int llr_cv_peak(int n, const double *centres, const double *a, double beta_lo, double beta_hi,
                int n_grid, double tol, double *out);

/* Canonical averages from the samples of a multicanonical run (Sec. 2.6,
 * eq. (2.56)).  A run with weight W = 1/rho~ (llr_muca_sweep) visits E_i;
 * reweighted to the coupling beta, sample i carries
 * exp(beta E_i) / W(E_i) = exp(beta E_i + ln rho~(E_i)), with ln rho~ the
 * table of llr_set_muca_weight: 0 at e0, slope a[k] on [e0 + k de,
 * e0 + (k + 1) de), the first / last slope beyond the n intervals.  For each
 * of n_beta couplings, <E> and <E^2> over all samples, in FP64 log space on
 * the device (sums over E - e0).
 *   E: host double[n_samples] (any order: the chains' samples pooled);
 *   a: host double[n]; beta: host double[n_beta];
 *   E_out, E2_out: host double[n_beta].  Synchronous, default stream; the
 *   call allocates and frees its device buffers (~16 bytes per sample).
 *   Errors: LLR_ERR_ARG (n_samples < 1, n < 1, de <= 0, non-finite e0,
 *   sample, slope or beta, null array; checked on the host before any device
 *   work), LLR_ERR_CUDA. */
int llr_muca_reweight(long long n_samples, const double *E, int n, double e0, double de,
                      const double *a, int n_beta, const double *beta, double *E_out,
                      double *E2_out);

/* The specific-heat peak (Sec. 3.4) of the reweighted samples of
 * llr_muca_reweight: C_V(beta) = <E^2> - <E>^2 on n_grid equally spaced
 * couplings in [beta_lo, beta_hi], then golden-section search between the
 * best grid point's neighbours to |interval| < tol.  Every evaluation is a
 * reweighting of all samples on the device.  Arguments as llr_muca_reweight.
 * out: host double[2] = {beta_c, C_V(beta_c)}.
 * Errors: as llr_muca_reweight, and LLR_ERR_ARG for n_grid < 2,
 * beta_hi <= beta_lo or tol <= 0. */
int llr_muca_cv_peak(long long n_samples, const double *E, int n, double e0, double de,
                     const double *a, double beta_lo, double beta_hi, int n_grid, double tol,
                     double *out);

/* Tunnellings of multicanonical chains, the ergodicity check of Sec. 2.6:
 * E: host double[n_steps][n_chains], the energy of every chain after each
 * sweep (the layout llr_muca_sweep writes); a passage of a chain from
 * E < lo to E > hi, or from E > hi to E < lo, counts once (E = lo or hi
 * counts as neither end).  out: host int[n_chains].  Synchronous.
 * Errors: LLR_ERR_ARG (n_steps < 0, n_chains < 1, lo > hi, null array),
 * LLR_ERR_CUDA. */
int llr_muca_tunnellings(int n_steps, int n_chains, const double *E, double lo, double hi,
                         int *out);

/* Launch shape of the batched sweep kernel: threads per CTA (128, 160, 192,
 * 256 or 512; one warp scans the window decisions, the others propose; one
 * CTA owns one lattice) and fast_math (1: hardware sine/cosine
 * approximations for the staples, 0: correctly rounded-class sincosf).
 * Chosen per lattice size by the autotuner; default 256 threads, fast math. */
int llr_set_kernel_config(llr_handle h, int threads, int fast_math);

/* The full launch shape of the batched sweep kernel, as the autotuner sets
 * it; none of these changes the chains (every shape runs the same per-link
 * arithmetic in the same order), only the speed.
 *   threads, fast_math: as llr_set_kernel_config.
 *   ring: stages of the heat-bath producer/consumer ring in use, 1, 2 or 4
 *     (how many 32-link-group chunks the proposing warps may run ahead of
 *     the warp that takes the window decisions).
 *   carveout: preferred share of the SM's unified L1/shared storage given to
 *     shared memory, in percent: 50, 75 or 100, or -1 for the driver's default
 *     (a hint; it is a property of the kernel variant in this process, so the
 *     last value set for a variant applies to every handle launching it).
 * Errors: LLR_ERR_ARG for any other value. */
int llr_set_kernel_shape(llr_handle h, int threads, int fast_math, int ring, int carveout);

/* The shape of the last launch of the batched sweep kernel on this handle:
 * out (host int[5]) = {threads per CTA, fast math, ring stages, carve-out,
 * CTAs launched}; all zero before the first launch. */
int llr_get_last_launch(llr_handle h, int *out);

/* ---------------------------------------------------------------------------
 * Learned warm start of the Robbins-Monro iteration (no counterpart in the
 * paper's algorithm; the paper's justification is that a_k is an intrinsic,
 * volume independent quantity, Sec. 2.2 eq. (2.5) and the appendix eqs.
 * (A.11)-(A.13), and that the initial a only needs to be close, Sec. 2.4).
 * A multilayer perceptron 3 -> 64 -> 64 -> 64 -> 1 with GELU (erf form)
 * maps the standardised features (1/V, E/6V, dE/6V), V = L^4 (finite-volume
 * corrections of a_k are O(1/V), eq. (A.12)), to a; FP32 parameters
 * in one array: W1 (3x64, [in][out]), b1, W2 (64x64), b2, W3 (64x64), b3,
 * W4 (64x1), b4 (llr_mlp_num_params() floats).  Loss: mean squared error.
 * All input arrays are host double[n]; calls are synchronous on the stream
 * given at creation (NULL = legacy default stream).
 * ------------------------------------------------------------------------ */
typedef struct llr_mlp *llr_mlp_handle;

/* Create a network with weights ~ N(0, 1/fan_in) from Philox(seed), zero
 * biases, identity standardisation (mean 0, std 1). */
int llr_mlp_create(llr_mlp_handle *out, uint64_t seed, void *cuda_stream);
int llr_mlp_num_params(void);
/* Copy the parameter array to / from a host float[llr_mlp_num_params()];
 * setting parameters also resets the Adam moments and step count. */
int llr_mlp_get_params(llr_mlp_handle h, float *out);
int llr_mlp_set_params(llr_mlp_handle h, const float *in);
/* Feature standardisation x = (raw - mean) / std, host double[3] each. */
int llr_mlp_set_norm(llr_mlp_handle h, const double *mean, const double *std);
int llr_mlp_get_norm(llr_mlp_handle h, double *mean, double *std);
/* Predicted slopes a_out[n] for inputs (L, E/6V, dE/6V). */
int llr_mlp_predict(llr_mlp_handle h, int n, const double *L, const double *e6v,
                    const double *dE6v, double *a_out);
/* Gradient of the loss on (inputs, a_target) with respect to every
 * parameter (grad_out: host float[llr_mlp_num_params()]) and the loss. */
int llr_mlp_grad(llr_mlp_handle h, int n, const double *L, const double *e6v,
                 const double *dE6v, const double *a_target, float *grad_out, double *loss_out);
/* Full-batch Adam (beta1 0.9, beta2 0.999, eps 1e-8) for `epochs` steps at
 * learning rate lr; standardise != 0 first sets mean/std from these inputs.
 * loss_out (nullable) gets the loss of the final parameters.  The epoch is
 * captured once in a CUDA graph and replayed. */
int llr_mlp_fit(llr_mlp_handle h, int n, const double *L, const double *e6v, const double *dE6v,
                const double *a_target, int epochs, double lr, int standardise,
                double *loss_out);
int llr_mlp_destroy(llr_mlp_handle h);

/* Upper bound on how long a work item of the batched kernel waits for the
 * previous sweep of its lattice (default 20 s).  When it runs out the item
 * is skipped, the lattice keeps its state and llr_status / the synchronous
 * calls return LLR_ERR_TIMEOUT; the CUDA context stays usable. */
int llr_set_wait_limit(llr_handle h, unsigned long long ns);

/* Checkpoint / resume.  The whole chain state of every lattice (link angles,
 * tracked energies, sweep counters, slopes, statistics) fits in
 * llr_state_bytes(h) bytes; llr_save_state copies it to the host buffer
 * `out`, llr_load_state copies it back into a handle created with the same
 * configuration (checked: LLR_ERR_ARG otherwise; the arrangement of link
 * arrays that replica exchanges produced is part of the state).  Random numbers are keyed
 * by the sweep counter, so a resumed run continues bit-identically. */
size_t llr_state_bytes(llr_handle h);
int llr_save_state(llr_handle h, void *out);
int llr_load_state(llr_handle h, const void *in);

/* Release everything the handle owns. */
int llr_destroy(llr_handle h);

/* Message of the last failed call on this thread ("" if none). */
const char *llr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LLR_H */
