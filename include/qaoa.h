/*
 * qaoa.h -- C ABI of the B300 LR-QAOA state-vector library (libqaoa.so).
 *
 * The library simulates depth-p linear-ramp QAOA (LR-QAOA) on weighted MaxCut
 * as defined in arxiv 2604.26423, Sec. II-B:
 *   H_C = sum_{(i,j) in E} w_ij Z_i Z_j                       (Eq. H_C)
 *   U_C(gamma_k) = exp(-i gamma_k s H_C)                      (Eq. UC)
 *   U_B(beta_k)  = exp(+i beta_k sum_q X_q)                   (Eq. UB)
 *   |psi_p> = U_B(beta_{p-1}) U_C(gamma_{p-1}) ... U_B(beta_0) U_C(gamma_0) |+>^n
 *   beta_k = (1 - k/p) dbeta, gamma_k = (k+1)/p dgamma, k = 0..p-1
 *   C(x) = sum_{k<l} w_kl (x_k + x_l - 2 x_k x_l)             (Eq. for C(x))
 *   r = (<C> - C_min) / (C_max - C_min)                       (Eq. r, exact mean)
 * The integer weights w_ij enter the phases multiplied by s = weight_scale.
 * Bit q of every amplitude or sample index is qubit q.
 *
 * Conventions for every call:
 *   - Return value: QAOA_OK or one of the QAOA_E* codes below; the message of
 *     the last failure on a context is available from qaoa_last_error().
 *   - Host pointers are read or written before the call returns. Device
 *     pointers must stay valid while the context uses them.
 *   - All GPU work is ordered on the CUDA stream given to qaoa_init_graph.
 *     Calls that return host results synchronise that stream.
 *   - The library never frees memory it did not allocate.
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef QAOA_H
#define QAOA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define QAOA_OK 0
#define QAOA_EINVAL 1   /* invalid argument (sizes, graph, angles, shots) */
#define QAOA_ENOMEM 2   /* allocation failed or a caller buffer is too small */
#define QAOA_ECUDA 3    /* a CUDA runtime call failed; see qaoa_last_error */
#define QAOA_ETIMEOUT 4 /* a bounded device-side wait gave up (batched queue; a forward
                           pass's tensor tile load, reported by qaoa_expect) */
#define QAOA_ESTATE 5   /* call order violated (e.g. qaoa_expect before qaoa_run) */

/* state precision: complex64 (2 x fp32 per amplitude) or complex128 */
#define QAOA_C64 0
#define QAOA_C128 1

/* how the cost phase obtains C(x): choose automatically (the choice recorded
 * for (n, precision) with qaoa_set_cost_choice, else recompute), recompute it
 * from the weight matrix inside each tile, or stream a precomputed int32
 * diagonal */
#define QAOA_COST_AUTO 0
#define QAOA_COST_RECOMPUTE 1
#define QAOA_COST_STREAM 2

/* largest qubit counts accepted: 2^34 complex64 amplitudes (128 GiB) and
 * 2^33 complex128 amplitudes (128 GiB) */
#define QAOA_MAX_QUBITS_C64 34
#define QAOA_MAX_QUBITS_C128 33

typedef struct qaoa_ctx qaoa_ctx;

/* Bytes of one state vector: 2^n * 8 (C64) or 2^n * 16 (C128); 0 if invalid. */
size_t qaoa_state_bytes(int n, int precision);

/*
 * Largest sum of |w| that qaoa_init_graph accepts: 2^30 - 1 for complex64 with
 * n >= 13 (the passes take the cost phase from 64-bit fixed-point turn
 * products of the integer cut value), 2^20 otherwise (a phase table indexed
 * by C(x)).
 */
int64_t qaoa_max_weight_sum(int n, int precision);

/*
 * Real-valued weights (Sec. II-G: the paper's instances have weights in
 * U[0, 1]) as integers for qaoa_init_graph: *unit = sum |w| / (max_abs_sum - m)
 * and w_int[e] = round(w[e] / unit), so sum |w_int| <= max_abs_sum and every
 * weight is off by at most unit / 2. Initialise with weight_scale s * unit to
 * keep the phases exp(-i gamma s w); cut values and <C> from the library are
 * then in units of `unit`. Host only. Errors: EINVAL (m < 1, a zero or
 * non-finite weight, a weight below unit / 2, max_abs_sum outside (2m, 2^31)).
 */
int qaoa_quantize_weights(int m, const double *w, int64_t max_abs_sum, int32_t *w_int, double *unit);

/*
 * Bytes of the optional auxiliary device buffer: the adjoint vector lambda
 * (one state's worth, needed by qaoa_grad) followed by the int32 cost diagonal
 * (2^n * 4 bytes, needed by QAOA_COST_STREAM). with_grad selects the first part,
 * cost_mode the second.
 */
size_t qaoa_aux_bytes(int n, int precision, int cost_mode, int with_grad);

/*
 * Records the cost mode (QAOA_COST_RECOMPUTE or QAOA_COST_STREAM) that
 * QAOA_COST_AUTO selects for contexts of n qubits in `precision` created after
 * this call, e.g. the faster one in an autotuner's timing; QAOA_COST_AUTO
 * forgets the record (AUTO then selects recompute). Process-wide and thread
 * safe; host only. qaoa_aux_bytes resolves AUTO the same way, so size the aux
 * buffer after recording. Errors: EINVAL (n or precision out of range, bad mode).
 */
int qaoa_set_cost_choice(int n, int precision, int cost_mode);

/*
 * Creates a context for one graph (Sec. II-B: weighted MaxCut instance).
 *   n            qubits = vertices, 1 <= n <= QAOA_MAX_QUBITS_*.
 *   n_edges      number of edges m >= 0; u[e] != v[e], both in [0, n), no
 *                repeated pair, w[e] != 0, sum |w| <= qaoa_max_weight_sum(n,
 *                precision). Host arrays of
 *                length m, copied; the caller keeps ownership.
 *   weight_scale s > 0 in the phases exp(-i gamma s h(x)); <C>, C_min and C_max
 *                are reported in integer weight units.
 *   precision    QAOA_C64 or QAOA_C128.
 *   cost_mode    QAOA_COST_*; AUTO takes the choice recorded for (n,
 *                precision) by qaoa_set_cost_choice, else recompute.
 *   state_dev    device buffer of exactly qaoa_state_bytes(n, precision)
 *                bytes, 256-byte aligned, or NULL (the library allocates).
 *   aux_dev      device buffer of aux_bytes >= qaoa_aux_bytes(...) or NULL
 *                (the library allocates lazily when first needed).
 *   cuda_stream  cudaStream_t to order all work on (NULL = legacy stream).
 * Stream mode writes the int32 diagonal and computes the exhaustive C_min /
 * C_max (with smallest argmin / argmax) on the GPU before returning; recompute
 * mode obtains them with the first run (its |+> pass visits every index once)
 * or, when qaoa_expect asks for them before any run, with the exhaustive
 * kernel. Errors: EINVAL (bad graph or sizes), ENOMEM (buffer too small or
 * allocation failure), ECUDA. On failure *ctx is NULL.
 */
int qaoa_init_graph(qaoa_ctx **ctx, int n, int n_edges, const int32_t *u, const int32_t *v,
                    const int32_t *w, double weight_scale, int precision, int cost_mode,
                    void *state_dev, size_t state_bytes, void *aux_dev, size_t aux_bytes,
                    void *cuda_stream);

/*
 * Kernel configuration of one context. The paper fixes none of these: they
 * select among equivalent ways to execute the same circuit (results agree to
 * the state precision's rounding). 0 in a field keeps the library default;
 * for a field left 0, the environment variable named beside it (read when the
 * context plans a run) replaces the default, so a process can set defaults
 * without code changes.
 */
#define QAOA_ON 1
#define QAOA_OFF 2
#define QAOA_ORDER_LOW_LAST 1   /* the last layer ends on the low index group */
#define QAOA_ORDER_LOW_MIDDLE 2 /* the low group away from the fused passes */
#define QAOA_SHAPE_5x3 1        /* 2^5 registers x 8 warps (T = 13) */
#define QAOA_SHAPE_4x4 2        /* 2^4 registers x 16 warps (T = 13), complex64 */
#define QAOA_SHAPE_5x2 3        /* 2^5 registers x 4 warps (T = 12), complex64 */
#define QAOA_SHAPE_4x3 4        /* 2^4 registers x 8 warps (T = 12) */
#define QAOA_SHAPE_5x4 5        /* 2^5 registers x 16 warps (T = 14), complex64 */
typedef struct qaoa_opts {
  int fwd_shape;       /* forward tile, QAOA_SHAPE_* (QAOA_FWD_SHAPE, QAOA_FWD_SHAPE_C128:
                          "5x3", "4x4", "5x2", "4x3", "5x4"); complex128 takes 5x3 or 4x3 */
  int super_tile;      /* largest forward super-tile in index bits, T..20 (QAOA_SMAX) */
  int group_order;     /* QAOA_ORDER_* of qaoa_run's plans (QAOA_GROUP_ORDER: "last", "middle") */
  int float_lanes;     /* QAOA_ON / QAOA_OFF: coalescing bits applied in a plain high-group
                          pass (QAOA_FLOAT_LANES: 1, 0) */
  int specialised;     /* QAOA_ON / QAOA_OFF: kernels compiled per round sequence (QAOA_SPEC) */
  int tile_tables;     /* QAOA_ON / QAOA_OFF: per-tile C(x) constants from tables (QAOA_TILE_TABLES) */
  int l2_prefetch;     /* QAOA_ON / QAOA_OFF: next tile prefetched into L2 (QAOA_L2PREFETCH) */
  int grad_order;      /* QAOA_ORDER_* of qaoa_grad's plans (QAOA_GRAD_ORDER) */
  int grad_checkpoint; /* QAOA_ON / QAOA_OFF: stored forward states in qaoa_grad
                          (QAOA_GRAD_CHECKPOINT) */
  int adj_l2_prefetch; /* QAOA_ON / QAOA_OFF: qaoa_grad's adjoint passes prefetch the next
                          tile of both vectors into L2 (QAOA_ADJ_L2_PREFETCH) */
  int tma_load;        /* QAOA_ON / QAOA_OFF: complex64 passes with a tensor prefetch load
                          each tile into shared memory by one tensor load issued during the
                          previous tile's last round (QAOA_TMA_LOAD) */
} qaoa_opts;

/* Sets the context's configuration (copied); later runs are planned with it.
 * Errors: EINVAL (NULL arguments or a value outside the encodings above). */
int qaoa_set_opts(qaoa_ctx *ctx, const qaoa_opts *opts);

/* The configuration in effect (options, else environment, else defaults) for
 * the context's precision, every field filled in. Errors: EINVAL. */
int qaoa_get_opts(const qaoa_ctx *ctx, qaoa_opts *opts);

/*
 * Prepares |psi_p> with the linear-ramp schedule (Sec. II-B) and computes <C>
 * and the norm on the GPU. p >= 0 (p = 0 leaves |+>^n). Asynchronous: results
 * are read by qaoa_expect. Errors: EINVAL, ECUDA.
 */
int qaoa_run(qaoa_ctx *ctx, int p, double dgamma, double dbeta);

/* As qaoa_run with explicit angles gamma[0..p-1], beta[0..p-1] (host arrays). */
int qaoa_run_angles(qaoa_ctx *ctx, int p, const double *gamma, const double *beta);

/*
 * Results of the last run (any output pointer may be NULL): <C> and the norm
 * (FP64 reductions), r = (<C> - C_min)/(C_max - C_min) (Eq. r with the exact
 * mean; 1 when C_max == C_min), and the exhaustive extremes with their smallest
 * indices (available before any run: then only the extremes may be requested).
 * Synchronises the stream. Errors: ESTATE (<C>, r or norm before a run), ECUDA,
 * ETIMEOUT (a bounded wait of the run's kernels gave up: the results are invalid;
 * the error is cleared, so the next run can proceed).
 */
int qaoa_expect(qaoa_ctx *ctx, double *exp_c, double *r, double *norm, int64_t *c_min,
                int64_t *c_max, uint64_t *argmin, uint64_t *argmax);

/*
 * Draws `shots` measurement samples from the last prepared state (Sec. II-B:
 * repeated preparation and measurement). Shot i is the smallest index x with
 * F(x) > u_i * total, where F is the cumulative |psi|^2 in index order and
 * total = F(2^n - 1), both accumulated in FP64. u_i = uniforms[i] if uniforms
 * is non-NULL (host array of `shots` values in [0, 1)), else u_i is draw i of
 * SplitMix64 stream `seed`: (mix(seed + (i+1) * 0x9E3779B97F4A7C15) >> 11) * 2^-53.
 * out: host array of `shots` indices. Errors: EINVAL, ESTATE, ECUDA.
 */
int qaoa_sample(qaoa_ctx *ctx, int shots, const double *uniforms, uint64_t seed, uint64_t *out);

/*
 * Adjoint gradient of <C> for the linear-ramp schedule: runs the forward
 * circuit, sets lambda = C psi_p and walks the layers backwards, uncomputing
 * psi and lambda with the inverse gates while accumulating
 *   g_beta[k]  = 2 Re <lambda| i H_B |psi>        (at layer k's mixer)
 *   g_gamma[k] = 2 Re <lambda| -i s H_C |psi>     (at layer k's cost phase)
 * and the chain rule d<C>/d dgamma = sum_k (k+1)/p g_gamma[k],
 * d<C>/d dbeta = sum_k (1 - k/p) g_beta[k]. Holds two state vectors (psi in
 * state_dev, lambda in the aux buffer). When the adjoint's passes retrace the
 * forward's and half of the free device memory holds (passes - 1) more states,
 * the forward instead keeps every pass's output in library-owned device memory
 * (held until qaoa_free; reused by later calls) and the adjoint reads psi from
 * it rather than writing the uncomputed psi back: one state write fewer per
 * adjoint pass. The grad_checkpoint option (qaoa_set_opts) turns this off.
 * Any output may be NULL; g_gamma and
 * g_beta hold p doubles; exp_c receives <C> = <psi_p|lambda> (taken in the
 * first adjoint pass). Leaves the context without a prepared state or result
 * (the walk back ends near |+>), so call qaoa_run again before qaoa_sample or
 * qaoa_expect (which then returns ESTATE).
 * Errors: EINVAL (p < 1), ENOMEM, ECUDA.
 */
int qaoa_grad(qaoa_ctx *ctx, int p, double dgamma, double dbeta, double *g_gamma,
              double *g_beta, double *d_dgamma, double *d_dbeta, double *exp_c);

/* As qaoa_grad with explicit angles; returns the per-layer gradients only. */
int qaoa_grad_angles(qaoa_ctx *ctx, int p, const double *gamma, const double *beta,
                     double *g_gamma, double *g_beta, double *exp_c);

/*
 * Writes C(x) for all x (int32, 2^n entries) into the device buffer out_dev,
 * using the same GPU evaluation as the cost phase. Errors: EINVAL, ECUDA.
 */
int qaoa_cost_diag(qaoa_ctx *ctx, int32_t *out_dev);

/*
 * Shots from a state vector without allocating any device memory. The paper
 * has no counterpart: this serves callers that must not call cudaMalloc while
 * they run (plugins whose host framework owns all device memory, serving
 * loops with a fixed memory budget that an allocation would break).
 *   state_dev     2^n amplitudes on the current device (complex64 or
 *                 complex128 per `precision`), read only.
 *   uniforms_dev  `shots` doubles in [0, 1) on the device, or NULL to draw u_i
 *                 from SplitMix64 stream `seed` exactly as qaoa_sample does.
 *   out_dev       `shots` uint64 indices on the device (written).
 * Same rule as qaoa_sample: shot i is the smallest x whose cumulative |psi|^2
 * exceeds u_i * total. Blocks of 2^12 amplitudes are used while the number of
 * blocks stays within QAOA_NOALLOC_MAX_BLOCKS, larger blocks beyond.
 * Scratch: one file-scope device array of 2 * QAOA_NOALLOC_MAX_BLOCKS + 1
 * doubles (about 1 MiB per GPU, held until exit), shared by every call. The
 * first call on a device looks up the array's address (kept until exit), so
 * make that first call before any stream capture; a device reset makes the
 * kept address stale, so do not call this again on a device after resetting
 * it. Calls whose GPU work overlaps (e.g. on two streams) race on the shared
 * scratch. Work is queued on cuda_stream and not waited for. Errors: EINVAL
 * (precision, n outside [1, QAOA_NOALLOC_MAX_QUBITS], shots < 0, NULL
 * buffers), ECUDA.
 */
#define QAOA_NOALLOC_MAX_BLOCKS 65536
#define QAOA_NOALLOC_MAX_QUBITS 34
int qaoa_sample_state_noalloc(const void *state_dev, int n, int precision, int shots,
                              const double *uniforms_dev, uint64_t seed, uint64_t *out_dev,
                              void *cuda_stream);

/* Device pointer of the context's state vector (interleaved re, im). */
void *qaoa_state_ptr(qaoa_ctx *ctx);

/*
 * Fills `out` (host, cap bytes) with a text description of the pass plan the
 * context would use for depth p (one line per pass and round). Host-only; for
 * inspection and tests. Returns the number of bytes needed (excluding NUL).
 */
int qaoa_describe_plan(int n, int precision, int p, int adjoint, char *out, int cap);

/*
 * Per-kernel timing (CUDA events recorded on the context's stream around every
 * launch of the library's kernels while enabled). kind: 0 forward pass
 * kernel, 1 adjoint pass kernel, 2 cost diagonal / extremes, 3 sampling,
 * 4 small-n whole-circuit kernels; kind 5 returns only the count of every
 * kernel launch (all kinds, including reduction and scan helpers) since
 * enabling. qaoa_profile_enable(ctx, 1) clears the
 * counters and starts recording; 0 stops. qaoa_profile_read synchronises the
 * stream and returns, for `kind`, the number of launches, their summed device
 * time in ms and the algorithmic bytes they moved (state reads and writes, plus
 * the int32 diagonal in stream mode). Errors: EINVAL (bad kind), ECUDA.
 */
int qaoa_profile_enable(qaoa_ctx *ctx, int enable);
int qaoa_profile_read(qaoa_ctx *ctx, int kind, int64_t *launches, double *ms, double *bytes);

/* Message of the last failure on ctx (or of the last failed qaoa_init_graph
 * when ctx is NULL). Never NULL. */
const char *qaoa_last_error(const qaoa_ctx *ctx);

/* Releases the context and every buffer the library allocated for it. */
void qaoa_free(qaoa_ctx *ctx);

/* ------------------------------------------------------------------------
 * Batched instances: many independent LR-QAOA MaxCut problems (complex64) in
 * one persistent kernel replayed from a CUDA graph. Each instance i has n[i]
 * qubits (2..24), depth p[i] (1..64), edges u/v/w[edge_off[i] .. edge_off[i+1])
 * (vertex indices local to the instance; the checks of qaoa_init_graph apply),
 * and the LR schedule of Sec. II-B with its own dgamma[i], dbeta[i]. Outputs
 * per instance: <C>, r (exhaustive C_min / C_max, Eq. r), the norm, and with
 * with_grad the exact adjoint gradient d<C>/d(gamma_k, beta_k) and its chain
 * rule to d<C>/d(dgamma, dbeta). The paper has no batched interface; it runs
 * its instances one at a time (Sec. III).
 */
typedef struct qaoa_batch qaoa_batch;

/* Scheduling knobs (0 = default). solo_max_n: instances below this many
 * qubits run all their passes in one CTA (default 16); window_items / window_mb:
 * large instances are interleaved pass by pass until their next passes hold at
 * least this many work items (default 2 per CTA) or their states this many MiB
 * (default 96, sized for L2); max_units: super-tiles per work item (default 8);
 * ctas_per_sm: persistent CTAs per SM (default: occupancy, at most 2);
 * wait_ns: limit of each device-side dependency wait in nanoseconds (default
 * 2e9). A wait that reaches the limit sets the batch's error flag and skips
 * its item, so the run ends and qaoa_batch_results returns ETIMEOUT; a limit
 * of 1 ns makes any wait give up (a test of that path). cost_mode: as at
 * qaoa_init_graph (AUTO and RECOMPUTE recompute C(x) in each tile; STREAM
 * reads an int32 diagonal per instance, computed once by qaoa_batch_create:
 * 2^n * 4 more bytes of device memory per instance with HBM passes).
 * fwd_shape: tile of the forward passes, QAOA_SHAPE_5x3 (default) or
 * QAOA_SHAPE_4x3. */
typedef struct qaoa_batch_opts {
  int solo_max_n, window_items, window_mb, max_units, ctas_per_sm;
  int64_t wait_ns;
  int cost_mode, fwd_shape;
} qaoa_batch_opts;

/* Validates and plans the batch, allocates its device memory (all states, and
 * the adjoint vectors with with_grad), uploads weights, phase and cost tables,
 * and captures one run (counter resets, the persistent kernel, the per-instance
 * finalisation) into a CUDA graph. Host arrays are copied; opts may be NULL.
 * Errors: EINVAL (sizes, graphs, angles), ENOMEM, ECUDA. On failure *out is
 * NULL and qaoa_batch_last_error(NULL) describes it. */
int qaoa_batch_create(qaoa_batch **out, int count, const int32_t *n, const int32_t *p,
                      const int64_t *edge_off, const int32_t *u, const int32_t *v, const int32_t *w,
                      const double *dgamma, const double *dbeta, double weight_scale, int with_grad,
                      const qaoa_batch_opts *opts, void *cuda_stream);

/* Replays the batch's graph on its stream (asynchronous). Each run recomputes
 * every instance from |+>. */
int qaoa_batch_run(qaoa_batch *b);

/* Waits for the stream and copies results to host arrays (either may be NULL):
 * out[9 i + 0..8] = {<C>, r, norm, C_min, C_max, argmin, argmax,
 * d<C>/d dgamma, d<C>/d dbeta} (the last two are 0 without gradient);
 * grads = per instance g_gamma[p_i] then g_beta[p_i], concatenated in instance
 * order (sum of 2 p_i doubles). Returns ETIMEOUT if a dependency wait in the
 * persistent kernel gave up (results are then invalid), ESTATE before a run. */
int qaoa_batch_results(qaoa_batch *b, double *out, double *grads);

/* Device pointer to instance i's final state (2^n[i] complex64); ESTATE for a
 * gradient batch, whose states have been walked back by the adjoint sweep. */
int qaoa_batch_state(qaoa_batch *b, int i, void **state_dev);

/* Human-readable plan summary (instances per mode, items, grid, bytes). */
int qaoa_batch_describe(const qaoa_batch *b, char *out, size_t cap);

/* Algorithmic HBM-or-L2 bytes of one run (state reads and writes of all passes). */
double qaoa_batch_bytes(const qaoa_batch *b);

const char *qaoa_batch_last_error(const qaoa_batch *b);
void qaoa_batch_free(qaoa_batch *b);

/* ------------------------------------------------------------------------
 * Noisy LR-QAOA (Sec. II-C): a two-qubit depolarizing channel of rate eps
 * after every ZZ gate, E(rho) = (1 - eps) rho + eps (I/4 (x) Tr_ij rho), i.e.
 * with probability eps one of the 16 two-qubit Paulis on (i, j), uniformly.
 * ------------------------------------------------------------------------ */

/*
 * Monte Carlo trajectories of the noisy circuit with explicit angles gamma,
 * beta (p each, host; the LR schedule is qaoa_run's) on the context's graph,
 * n <= QAOA_NOISY_MAX_QUBITS, in the context's precision (complex64: FP32
 * phases and butterflies; <C>_t always summed in FP64). Trajectory t draws, for
 * gate g = k m + e (layer k, edge e in the order given to qaoa_init_graph),
 * draw t (p m) + g of SplitMix64 stream `seed`: an error when its top 53 bits
 * times 2^-53 are below eps, then Pauli (draw & 3) on u_e and ((draw >> 2) & 3)
 * on v_e (0 I, 1 X, 2 Y, 3 Z). exp_c_dev (device, `trajectories` doubles, or
 * NULL): each trajectory's <C>_t; *mean_exp_c (host, or NULL): their mean, the
 * noisy <C> estimate; *r_noisy (host, or NULL): (mean - C_min)/(C_max - C_min).
 * The context's state is not touched. Returns after the kernels finished.
 * Errors: EINVAL (n too large, p < 0, eps outside [0, 1], trajectories < 1,
 * non-finite angles), ENOMEM, ECUDA.
 */
#define QAOA_NOISY_MAX_QUBITS 12
int qaoa_noisy_expect(qaoa_ctx *ctx, int p, const double *gamma, const double *beta, double eps,
                      int trajectories, uint64_t seed, double *exp_c_dev, double *mean_exp_c, double *r_noisy);

/* r_ovl = (r_noisy - r_random) / (r_ideal - r_random) (Sec. II-C); host only. */
double qaoa_overlap_ratio(double r_noisy, double r_ideal, double r_random);

/*
 * k0 of Eq. noise, r_ovl = 2^(-k0 eps_acc) with eps_acc = N_2q eps: the least
 * squares slope of log2 r_ovl = -k0 eps_acc through the origin over the
 * `count` points (host arrays) with r_ovl > 0; NaN when none remains.
 */
double qaoa_fit_k0(int count, const double *eps_acc, const double *r_ovl);

/* ------------------------------------------------------------------------
 * Sampling methodology (Sec. II-D): the approximation ratio of individual
 * bitstrings, the uniform random sampler, the mean of subsample means and the
 * three performance regimes. Random draws are SplitMix64 stream draws (the
 * definition given at qaoa_sample).
 * ------------------------------------------------------------------------ */

/*
 * Cut value C(x) (Sec. II-B) and approximation ratio r(x) = (C(x) - C_min) /
 * (C_max - C_min) (Eq. r with one bitstring; 1 when C_max = C_min) of `count`
 * bitstrings on the context's graph. x_dev: device array of `count` indices
 * < 2^n, or NULL for the random sampler: x_i = the top n bits of draw i of
 * stream `seed`. Outputs are device arrays of `count` entries, each optional:
 * x_out_dev (the bitstrings), c_out_dev (int32 C), r_out_dev (double r).
 * C_min / C_max are those of qaoa_expect (computed first when not known).
 * Ordered on the context's stream; returns after the kernel finished.
 * Errors: EINVAL (count < 0, an index >= 2^n), ENOMEM, ECUDA.
 */
int qaoa_sample_cuts(qaoa_ctx *ctx, int64_t count, const uint64_t *x_dev, uint64_t seed,
                     uint64_t *x_out_dev, int32_t *c_out_dev, double *r_out_dev);

/*
 * Mean of subsample means (Sec. II-D). From the pool r_dev[0..m) (device,
 * read only), `reps` subsamples of `ns` distinct entries are drawn uniformly
 * without replacement, each by a partial Fisher-Yates shuffle: step j of
 * subsample i takes draw k = i*ns + j of stream `seed` and swaps position j
 * with position j + floor(z_k (m - j) / 2^64); the entry moved to position j
 * joins the subsample. means_dev[i] (device, reps doubles) = the entries'
 * FP64 sum in draw order / ns. stats_dev (device, 3 doubles) = {grand mean
 * <r_bar> (sum of the means in order / reps), sigma (square root of the mean
 * squared deviation, 1/reps), random threshold <r_bar> + 3 sigma}. No device
 * memory is allocated. Limits: 1 <= ns <= min(m, 4096), m < 2^32 - 1,
 * 1 <= reps <= 65535. Asynchronous on `cuda_stream`. Errors: EINVAL, ECUDA.
 */
#define QAOA_MOM_MAX_NS 4096
int qaoa_mean_of_means(const double *r_dev, int64_t m, int ns, int reps, uint64_t seed, double *means_dev,
                       double *stats_dev, void *cuda_stream);

/*
 * Performance regime of an observed mean ratio r_obs (Sec. II-D), host only.
 * QAOA_REGIME_RANDOM when r_obs is within or below the random sampler's
 * interval (r_obs <= rand_mean + 3 rand_sigma); otherwise, with a noiseless
 * reference (have_ideal != 0), QAOA_REGIME_NOISE_TOLERANT when r_obs reaches
 * its interval (r_obs >= ideal_mean - 3 ideal_sigma), else
 * QAOA_REGIME_TRANSITION; without one, QAOA_REGIME_ABOVE_RANDOM (the result is
 * statistically meaningful at 99.73% confidence). Returns the regime, or -1
 * for a NaN or negative sigma.
 */
enum { QAOA_REGIME_RANDOM = 0, QAOA_REGIME_TRANSITION = 1, QAOA_REGIME_NOISE_TOLERANT = 2,
       QAOA_REGIME_ABOVE_RANDOM = 3 };
int qaoa_classify_regime(double r_obs, double rand_mean, double rand_sigma, int have_ideal, double ideal_mean,
                         double ideal_sigma);

#ifdef __cplusplus
}
#endif
#endif /* QAOA_H */
