/*
 * fdcore -- GB300 (sm_103a) library for batched Monte Carlo evaluation of
 * compiled self-energy Feynman graphs (arXiv 2403.18840).
 *
 * The paper states the problem as I_f = int dx f(x) over the unit hypercube
 * (Sec. IV) with f the order-n self-energy integrand (Sec. II.A, Eq.
 * sigma_integration) and its counterterm derivatives Sigma^(n,m,l)
 * (Sec. VI.A, Eq. sigma_xi_dmu_dlambda).  This header is the whole boundary:
 * plain pointers and sizes, no framework types.
 *
 * Conventions shared by every call
 *  - Device buffers are owned by the caller and passed as raw device pointers;
 *    `stream` is a cudaStream_t cast to void* (NULL = legacy default stream).
 *  - Opaque handles are owned by the library (create/free pairs).
 *  - Calls are asynchronous on `stream` unless stated otherwise.
 *  - No exception crosses the boundary: every failure returns a status other
 *    than FD_OK and sets a thread-local message readable by fd_last_error().
 *    Arguments are validated before any launch; on error nothing is launched.
 *  - Host threads: calls on distinct handles may come from several host
 *    threads at once (launch descriptors are built in thread-local storage);
 *    one handle is not to be used by two threads at the same time, and the
 *    no-allocation entry point's shared scratch array is serialised on the
 *    stream by the caller (see fd_integrand_eval_stats_noalloc).
 *  - Hypercube points are structure-of-arrays: x[d * n + i] for dimension d
 *    and sample i (FP32).
 *  - Units: Rydberg, hbar^2/2m = 1, e^2 = 2: eps_k = k^2 - mu and
 *    V(q) = 8 pi / (q^2 + Lambda) (Eq. ueg_action with Yukawa screening,
 *    Eq. interaction_ct).
 */
#ifndef FDCORE_H
#define FDCORE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FD_OK = 0,
    FD_EINVAL = 1,    /* bad argument (null pointer, size, range, NaN parameter) */
    FD_EFORMAT = 2,   /* malformed graph tape */
    FD_ENOMEM = 3,    /* device or host allocation failed */
    FD_ECUDA = 4,     /* CUDA runtime error */
    FD_ETIMEOUT = 5,  /* a bounded device wait gave up (kernel returned early) */
    FD_ENOTSUP = 6    /* valid request the library does not support */
} fd_status;

typedef struct fd_graph fd_graph;
typedef struct fd_vegas fd_vegas;
typedef struct fd_flow fd_flow;

/* Physical parameters of one instance (Sec. VI.A).  k_ext: external momentum
 * |k| (along z); mu: renormalised chemical potential mu_R = E_F; beta = 1/T;
 * Lambda: Yukawa screening lambda^2; k_cut: radius cutoff of every loop
 * momentum.  k_F is informational (post-processing uses it). */
typedef struct {
    double k_ext, k_F, mu, beta, Lambda, k_cut;
    int32_t order;   /* must equal the order of the instance's graph */
    int32_t reserved;
} fd_params;

/* Sample-tile size of the reduction: partial sums are kept per instance and
 * per tile of consecutive samples.  The tile is the smallest power of two
 * >= n_per_inst / 4096, at least 1024 and at most FD_TILE_SAMPLES: many work
 * items per SM, so the last wave of the persistent CTAs leaves little idle
 * time; fd_tile_samples(n) returns it. */
#define FD_TILE_SAMPLES 16384
int64_t fd_tile_samples(int64_t n_per_inst);

/* Message of the last failed call on this thread ("" if none). */
const char *fd_last_error(void);

/* ---- graphs (Sec. V.A: the compiled computational graph) -----------------
 * fd_graph_load parses and validates a tape produced by the graph compiler
 * (format in paper_2403_18840_gb300/fdgraph.py: header, root table
 * (n, m, l, dk) per root, 64-bit instructions), checks every slot index and
 * opcode against the declared sizes, and uploads it to the current device.
 * Synchronous.  FD_EFORMAT on any inconsistency; the buffer is not retained. */
fd_status fd_graph_load(const void *buf, size_t len, fd_graph **out);
/* n_roots: number of roots; dim: hypercube dimension 4N-1; n_instr: tape
 * length; n_slots: per-sample state size in 4-byte slots. Any pointer may be NULL. */
fd_status fd_graph_info(const fd_graph *g, int32_t *n_roots, int32_t *dim,
                        int64_t *n_instr, int32_t *n_slots);
/* roots[4*r + {0,1,2,3}] = (n, m, l, dk) of root r (host array of 4*n_roots). */
fd_status fd_graph_roots(const fd_graph *g, int32_t *roots);
void fd_graph_free(fd_graph *g);
/* Preferred CTA shape of evaluation launches whose first graph is g:
 * (threads, samples per thread) in {(128,2), (256,1), (128,1), (64,2), (64,1)},
 * or (0,0) for the automatic choice (most samples in flight per SM).
 * A preference that does not fit in shared memory falls back to automatic. */
fd_status fd_graph_set_launch(fd_graph *g, int32_t threads, int32_t samples_per_thread);

/* ---- specialised kernels (Sec. VI.A: graphs compiled once, evaluated in batches)
 * fd_graph_jit translates the graph's validated tape into straight-line CUDA
 * (the backward slice of every root-accumulate instruction, intermediates in
 * registers), compiles it for the current device with NVRTC (modules
 * compiled in parallel and linked with nvJitLink when the graph is large) and
 * from then on evaluates the graph's instances with it (one launch per graph;
 * graphs without one keep the interpreter).  Options:
 *  threads      CTA size, 64, 128 or 256;
 *  min_blocks   1..8, launch bounds; registers capped at 65536 / (threads * min_blocks);
 *  max_modules  1..64, modules compiled in parallel for a large graph;
 *  root_units   != 0: a split graph gets one function per root (its slices
 *               share their leaves) instead of one per slice;
 *  sync_every   > 0: a block barrier after about that many generated
 *               arithmetic statements (warps share instruction-cache lines);
 *               with spt > 1: a block barrier after every unit call;
 *  leaf_calls   != 0: leaf families are calls to one out-of-line function per
 *               (Taylor order, d/dk) shape instead of inlined code;
 *  spt          1..16 samples per thread per pass; with spt > 1 every
 *               compilation unit loops over the spt samples, so its code is
 *               re-executed from the instruction cache;
 *  unit_cap     with spt > 1: consecutive slices of a root share a unit while
 *               its cost (FMAs + 30 per distinct leaf) stays within the cap;
 *  pair         != 0 (even spt, inlined leaves): every unit evaluates two of
 *               the thread's samples at once in packed two-lane FP32
 *               arithmetic (the same operations per lane, one instruction for
 *               both samples);
 *  sv_smem      != 0 (spt > 1): the per-sample inputs of the thread's spt
 *               samples (momenta, times) in shared memory instead of local
 *               memory; FD_EINVAL from fd_graph_jit when they do not fit;
 *  cross_roots  != 0 (spt > 1): units pack consecutive slices across root
 *               boundaries, so leaves that neighbouring roots share are
 *               computed once per unit.
 *  leaf_cache   0..4096 floats per sample (scalar, inlined leaves): leaf
 *               families used by several units are computed once per sample
 *               into shared memory ([float][sample][thread], threads x spt x
 *               4 bytes per float) and read there by the units, the families
 *               that save the most work per float first, up to this many
 *               floats; any spt (spt = 1 takes the sample-loop kernel);
 *  lc_global    != 0 (leaf_cache > 0): the leaf cache in a global scratch
 *               array the graph owns (one region per resident CTA, freed
 *               with the graph or the next fd_graph_jit) instead of shared
 *               memory; evaluations of such a graph must not overlap on the
 *               GPU (they share the array).
 * cache_dir (may be NULL): directory for compiled images, keyed by a hash of
 * the generated source and options.  Synchronous; FD_ENOTSUP when the
 * run-time compiler is unavailable or fails (fd_last_error holds its log).
 * Results agree with the interpreter up to FP32 rounding order. */
typedef struct {
    int32_t threads, min_blocks, max_modules, root_units, sync_every, leaf_calls, spt, unit_cap, pair, sv_smem,
        cross_roots, leaf_cache, lc_global;
} fd_jit_options;
fd_status fd_graph_jit(fd_graph *g, const fd_jit_options *opt, const char *cache_dir);
/* Switch evaluation of g between its specialised kernel (on != 0) and the interpreter. */
fd_status fd_graph_jit_enable(fd_graph *g, int32_t on);
/* info[6] = threads, min_blocks, registers per thread, local bytes per thread,
 * modules, enabled; compile_s (may be NULL) = seconds of the last fd_graph_jit. */
fd_status fd_graph_jit_info(const fd_graph *g, int32_t *info, double *compile_s);
/* The generated source of module `module` for a serialised tape (no device
 * needed): copies at most cap - 1 bytes plus a terminating 0 into buf (may be
 * NULL), *len = full length, *n_modules = module count. */
fd_status fd_jit_emit(const void *tape, size_t tape_len, const fd_jit_options *opt, int32_t module, char *buf,
                      int64_t cap, int64_t *len, int32_t *n_modules);

/* ---- VEGAS map (Sec. IV, separable map q(x) = prod q_k(x_k)) ---------------
 * A map owns FP64 bin edges [dim][n_bins+1] (uniform at creation), their FP32
 * copy used by the sampling kernels, and an FP64 training histogram
 * [dim][n_bins] that fd_integrand_eval accumulates (sum of (f J)^2 per bin)
 * and fd_vegas_update consumes.  create/free/set/get are synchronous. */
fd_status fd_vegas_create(int32_t dim, int32_t n_bins, fd_vegas **out);
void fd_vegas_free(fd_vegas *m);
/* host FP64 edges [dim][n_bins+1]; must be strictly increasing from 0 to 1 */
fd_status fd_vegas_set_edges(fd_vegas *m, const double *edges);
fd_status fd_vegas_get_edges(const fd_vegas *m, double *edges);
/* host FP64 copy of the histogram [dim][n_bins] */
fd_status fd_vegas_get_hist(const fd_vegas *m, double *hist);
/* overwrite the histogram from host FP64 [dim][n_bins] (entries >= 0) */
fd_status fd_vegas_set_hist(fd_vegas *m, const double *hist);
/* zero the histogram (async) */
fd_status fd_vegas_clear_hist(fd_vegas *m, void *stream);
/* Lepage's update (3-point smoothing, damping exponent alpha, equal-share
 * redistribution of the edges) in FP64 on the device, then zero the
 * histogram. */
fd_status fd_vegas_update(fd_vegas *m, double alpha, void *stream);
/* The same update for n_maps (<= 256) maps of equal bin count in one launch. */
fd_status fd_vegas_update_batch(fd_vegas *const *maps, int32_t n_maps, double alpha, void *stream);

/* ---- sample generation ---------------------------------------------------
 * Philox4x32-10 stream of sample i of instance `inst` at iteration `iter`:
 * counter (i_lo, i_hi, iter, (inst << 8) | block), key (seed_lo, seed_hi);
 * u = ((w >> 9) + 0.5) 2^-23.  map == NULL: x = u, w = 1; otherwise the VEGAS
 * map, w = its Jacobian.  x: device [dim][n], w: device [n] (may be NULL).
 * dim must equal the map's dimension when map != NULL. */
fd_status fd_map_samples(const fd_vegas *map, uint64_t seed, uint64_t iter, int32_t inst,
                         int64_t n, int32_t dim, float *x, float *w, void *stream);

/* ---- integrand evaluation (Eqs. sigma_integration, sigma_xi_dmu_dlambda) --
 * One launch over n_inst instances; instance j evaluates graph
 * graphs[graph_of_inst[j]] with params[j] on n_per_inst samples drawn as in
 * fd_map_samples with maps[j] (NULL entry = identity) -- or, when `points`
 * is not NULL, on the given points instead (points: device
 * [n_inst][dim_max][n_per_inst] with dim_max the largest graph dimension,
 * point_w: device [n_inst][n_per_inst] sample weights).  Given points with a
 * map are coordinates of the map's input space: the map and its Jacobian are
 * applied (a proposal that lives on top of an adapted VEGAS grid).
 * For each sample and root r it computes
 *   f_r = w * J(x) * sum_t s_t d^m_mu d^l_Lambda (d_k)^dk [prod G0 prod V] e^{i pi x_out}
 * in FP32 (J: loop-momentum and time Jacobians of the roots' own variables).
 * Outputs
 *  partials (device, required): FP64 [n_inst][n_tiles][R_max][2][2] with
 *    n_tiles = ceil(n_per_inst / fd_tile_samples(n_per_inst)), R_max the largest root
 *    count; entry (.., r, c, 0) = sum of f (c = 0 real, 1 imaginary) over the
 *    tile, (.., r, c, 1) = sum of f^2.  Tiles are summed in a fixed order
 *    inside the tile, so results are bitwise reproducible.
 *  per_sample_f (device, optional): FP32 [n_inst][R_max][2][n_per_inst].
 *  VEGAS maps accumulate their histograms only when `points` is NULL.
 * params and graph_of_inst are host arrays; graphs/maps host arrays of handles.
 * FD_ETIMEOUT if a bounded wait for a tape copy gave up. */
fd_status fd_integrand_eval(const fd_graph *const *graphs, int32_t n_graphs,
                            const fd_params *params, const int32_t *graph_of_inst,
                            int32_t n_inst, fd_vegas *const *maps, const float *points,
                            const float *point_w, uint64_t seed, uint64_t iter,
                            int64_t n_per_inst, double *partials, float *per_sample_f,
                            void *stream);

/* As fd_integrand_eval (sampler maps or identity, no per-sample output) with
 * the Philox iteration taken as iter_base + *d_iter, read on the device when
 * the kernel runs, so that a captured CUDA graph advances the sample stream
 * on every replay (d_iter: device uint32, advanced with fd_counter_add). */
fd_status fd_integrand_eval_iter_dev(const fd_graph *const *graphs, int32_t n_graphs,
                                     const fd_params *params, const int32_t *graph_of_inst,
                                     int32_t n_inst, fd_vegas *const *maps, uint64_t seed,
                                     uint64_t iter_base, const uint32_t *d_iter, int64_t n_per_inst,
                                     double *partials, void *stream);
/* As fd_integrand_eval without the per-sample roots, writing instead the
 * learned proposal's training target (App. A: the flow is fitted by forward
 * KL to |f| on points the method itself draws, each weighted by 1/q of the
 * sampler that drew it): abs_f [n_inst][n_per_inst] (device FP32) receives,
 * per sample, the sum over the value roots (no d/dk) of |Re| + |Im| of the
 * weighted integrand (the point weight, e.g. 1/q, and the map's Jacobian
 * included), 0 where that sum is not finite.  The same sum feeds the VEGAS
 * histogram.  FD_EINVAL for a null abs_f, otherwise as fd_integrand_eval. */
fd_status fd_integrand_eval_target(const fd_graph *const *graphs, int32_t n_graphs, const fd_params *params,
                                   const int32_t *graph_of_inst, int32_t n_inst, fd_vegas *const *maps,
                                   const float *points, const float *point_w, uint64_t seed, uint64_t iter,
                                   int64_t n_per_inst, double *partials, float *abs_f, void *stream);

/* *d_counter += v on the device (async). */
fd_status fd_counter_add(uint32_t *d_counter, uint32_t v, void *stream);

/* Synchronise `stream`; FD_ETIMEOUT if a kernel recorded a bounded wait
 * that gave up since the last call (the record is cleared). */
fd_status fd_device_status(void *stream);

/* Test hook for the bounded waits (the paper has no counterpart; failure
 * handling of this library).  The tape interpreter stages its instruction
 * chunks into shared memory with bulk copies and waits on an mbarrier for
 * each, polling at most a fixed number of times (2^24) before it gives up,
 * records FD_ETIMEOUT for fd_device_status, waits (at the full limit) for the
 * copies still in flight and returns early, leaving its unfinished tiles
 * unwritten.  This call sets that poll count for the evaluations issued
 * after it from any host thread: polls = 0 gives up at the first wait (the
 * timeout path runs without a fault or a hang), polls < 0 restores the
 * default.  FD_EINVAL for polls >= 2^32. */
fd_status fd_debug_set_wait_polls(int64_t polls);

/* Number of doubles of the `partials` buffer for this launch shape: the tile
 * partial sums followed by one word the launch uses as its work counter. */
int64_t fd_partials_count(int32_t n_inst, int32_t r_max, int64_t n_per_inst);

/* ---- reduction (FP64, fixed order) ---------------------------------------
 * From partials [n_inst][n_tiles][r_max][2][2] compute, per instance, root
 * and real/imaginary part, the mean and the variance of the mean over
 * n_per_inst samples: out (device) [n_inst][r_max][2][2] = (mean, var).
 * Tiles are combined in index order with Neumaier compensation. */
fd_status fd_accumulate(const double *partials, int32_t n_inst, int32_t r_max,
                        int64_t n_per_inst, double *out, void *stream);

/* ---- evaluation without device allocation ---------------------------------
 * The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory (a host process whose allocations are all made up
 * front, a replayed CUDA graph that may not allocate, a caller without an
 * allocator in reach).  It does what fd_integrand_eval followed by
 * fd_accumulate do, with the same arguments except that the tile partial
 * sums live in one fixed device array inside this library (holding
 * FD_NOALLOC_MAX_PARTIALS doubles, 4 MiB, present on every device that loads
 * the library until the process exits) instead of a caller buffer, and the
 * result goes straight to `out` (device FP64 [n_inst][R_max][2][2], mean and
 * variance of the mean).  It calls no allocator.
 *  - Requests needing more than FD_NOALLOC_MAX_PARTIALS partial sums
 *    (fd_partials_count) are rejected with FD_EINVAL before any launch.
 *  - The first call on a device resolves the array's device address; make
 *    that first call before any stream capture on that device.
 *  - All calls share the one array: calls whose kernels overlap on the GPU
 *    (different streams, no ordering between them) race and give wrong
 *    results.  Each call first fills the part it uses with NaN, so a tile a
 *    kernel could not finish shows up as NaN in `out`.
 *  - A bounded wait that gives up is not recorded for fd_device_status on
 *    this path; it appears as NaN in `out`. */
#define FD_NOALLOC_MAX_PARTIALS (1 << 19)
fd_status fd_integrand_eval_stats_noalloc(const fd_graph *const *graphs, int32_t n_graphs,
                                          const fd_params *params, const int32_t *graph_of_inst,
                                          int32_t n_inst, fd_vegas *const *maps,
                                          const float *points, const float *point_w,
                                          uint64_t seed, uint64_t iter, int64_t n_per_inst,
                                          double *out, float *per_sample_f, void *stream);

/* ---- affine coupling flow (Appendix A, Eqs. NFtransform, coupling_layer) --
 * A flow of n_layers affine coupling layers over [0,1]^dim in logit space,
 * each conditioned by an MLP (in -> hidden -> hidden -> out, ReLU), BF16
 * weights/activations on tensor cores with FP32 accumulation, FP32 master
 * weights and Adam state.  Parameter blob layout (FP32, host): per layer
 * W1 [H][a], b1 [H], W2 [H][H], b2 [H], W3 [2b][H], b3 [2b] with a/b the
 * sizes of the conditioning/transformed halves (first ceil(dim/2)
 * coordinates condition on even layers). */
fd_status fd_flow_create(int32_t dim, int32_t n_layers, int32_t hidden, uint64_t seed,
                         fd_flow **out);
void fd_flow_free(fd_flow *f);
int64_t fd_flow_param_count(const fd_flow *f);
fd_status fd_flow_set_params(fd_flow *f, const float *blob, int64_t n);
fd_status fd_flow_get_params(const fd_flow *f, float *blob, int64_t n);
/* z ~ U(0,1)^dim from the Philox stream (as fd_map_samples), x = T(z) and
 * w = 1/q(x).  x: device [dim][n], w: device [n]. */
fd_status fd_flow_sample(const fd_flow *f, uint64_t seed, uint64_t iter, int32_t inst,
                         int64_t n, float *x, float *w, void *stream);
/* Defensive mixture proposal q_mix = (1 - a) q + a (a uniform share on the
 * hypercube; Hesterberg's defensive importance sampling): samples
 * [0, n - n_u) as fd_flow_sample, samples [n - n_u, n) uniform from the same
 * Philox stream, where the flow share n - n_u is n - floor(alpha n) rounded up
 * to a multiple of 512 (at most n), and every sample weighted w = 1 / q_mix(x)
 * with a = n_u / n (written to *alpha_used, may be NULL).  The weights never exceed 1 / a, so the proposal's tails are
 * bounded by those of the uniform (or, on a VEGAS grid's coordinates, of
 * VEGAS).  alpha in [0, 0.5]. */
fd_status fd_flow_sample_defensive(const fd_flow *f, uint64_t seed, uint64_t iter, int32_t inst,
                                   int64_t n, double alpha, float *x, float *w, double *alpha_used,
                                   void *stream);
/* log q(x) for given points (inverse pass).  x: device [dim][n], logq: device [n]. */
fd_status fd_flow_log_density(const fd_flow *f, const float *x, int64_t n, float *logq,
                              void *stream);
/* Tensor-core path of the sampling and density passes: 2 (default) =
 * tcgen05.mma with TMEM accumulators, warp-specialised: four 128-sample tiles
 * in flight per SM, one thread issuing the GEMMs, one streaming the layers'
 * weights by bulk copies, epilogue warps owning one sample per thread (the
 * hidden biases enter the accumulators on the tensor core); 1 = tcgen05.mma
 * with two tiles in flight and block barriers between the GEMMs; 0 =
 * warp-level mma.sync m16n8k16 with the activations kept in registers.  All
 * compute the same BF16 contract (BF16 weights and GEMM inputs, FP32
 * accumulation); training always uses the mma.sync kernels.  FD_EINVAL for
 * another path. */
fd_status fd_flow_set_tensor_path(fd_flow *f, int32_t path);
/* Weighted forward-KL loss L = -sum w log q(x) / sum w and its gradient in
 * blob layout.  x: device [dim][n]; w: device [n] (>= 0); loss: device [1];
 * grad: device [param_count]. */
fd_status fd_flow_grad(fd_flow *f, const float *x, const float *w, int64_t n, float *loss,
                       float *grad, void *stream);
/* `steps` Adam steps (lr, beta = (0.9, 0.999), eps = 1e-8) on the batch
 * (x, w).  loss_out: host array [steps] of losses (synchronous readback at
 * the end), may be NULL. */
fd_status fd_flow_train(fd_flow *f, const float *x, const float *w, int64_t n, int32_t steps,
                        float lr, float *loss_out, void *stream);

/* ---- pipe throughput probes -------------------------------------------------
 * Measured throughput of one pipe of the current device, used as roofline
 * denominators next to the unit-count peaks: kind 0 = FP32 FMA (flops per
 * second, FMA = 2), 1 = SFU exp2 (results per second), 2 = SFU reciprocal,
 * 3 = packed two-lane FP32 FMA (flops per second, 4 per instruction).
 * Synchronous; allocates a small scratch buffer. */
fd_status fd_measure_peak(int32_t kind, double *ops_per_s);

/* ---- neural spline flow, sampling and density (App. A) --------------------
 * x = T(z), z uniform on [0, 1]^dim, T = n_layers rational-quadratic coupling
 * layers (K = 8 bins on [0, 1]: widths and heights from softmax of the
 * conditioner's outputs, each at least 1e-3; derivative 1e-3 + softplus at the
 * 7 internal knots, 1 at both ends), layer l keeping the first floor(dim/2)
 * coordinates when l is even and the others when odd; the conditioner maps
 * the kept coordinates linearly to width 32, applies two residual blocks
 * h += W_b relu(W_a relu(h) + b_a) + b_b and maps linearly to 23 parameters
 * per transformed coordinate (8 width, 8 height, 7 derivative logits).
 * Parameters (host FP32, fd_nsf_param_count of them), layer after layer:
 * W0 [n_keep][32], b0 [32], for each block W_a [32][32], b_a [32], W_b [32][32],
 * b_b [32], then W1 [32][n_move * 23], b1 [n_move * 23] (row-major, inputs
 * first).  The flow owns its device copy; create/free are synchronous. */
typedef struct fd_nsf fd_nsf;
fd_status fd_nsf_create(int32_t dim, int32_t n_layers, fd_nsf **out);   /* 2 <= dim <= 24; all parameters 0 */
void fd_nsf_free(fd_nsf *f);
int64_t fd_nsf_param_count(const fd_nsf *f);
/* Synchronous; FD_EINVAL if any is non-finite.  Also resets the training
 * state (Adam moments and step count, fd_nsf_train). */
fd_status fd_nsf_set_params(fd_nsf *f, const float *params, int64_t n);
/* The current parameters into host params [n == fd_nsf_param_count];
 * synchronous (waits for the device). */
fd_status fd_nsf_get_params(const fd_nsf *f, float *params, int64_t n);
/* x = T(z) for device z [dim][n]: x (device FP32 [dim][n]) and log q(x)
 * (device FP32 [n]); 1 <= n <= 2^36 (FD_EINVAL otherwise).  Asynchronous on
 * stream. */
fd_status fd_nsf_forward(const fd_nsf *f, const float *z, int64_t n, float *x, float *logq, void *stream);
/* The same with z from the sample stream (Philox counter (i_lo, i_hi, iter,
 * inst << 8 | block), u = ((w >> 9) + 0.5) 2^-23). */
fd_status fd_nsf_sample(const fd_nsf *f, uint64_t seed, uint64_t iter, int32_t inst, int64_t n, float *x,
                        float *logq, void *stream);
/* The sampler's draws as importance-sampling proposals (App. A: the flow
 * proposes configurations for the integral of Sec. IV and for the NF-MCMC
 * chains of Sec. V): the same stream and points as fd_nsf_sample, with w
 * (device FP32 [n]) = 1 / q(x), the weight fd_integrand_eval takes as
 * point_w and the chains take through the integrand's weighted values. */
fd_status fd_nsf_sample_w(const fd_nsf *f, uint64_t seed, uint64_t iter, int32_t inst, int64_t n, float *x,
                          float *w, void *stream);
/* Density at given points: z = T^-1(x) (device FP32 [dim][n], the layers in
 * reverse order, each spline inverted through its bin's quadratic) and
 * log q(x) (device FP32 [n]) for device x [dim][n] in [0, 1]^dim.
 * Asynchronous on stream. */
fd_status fd_nsf_log_density(const fd_nsf *f, const float *x, int64_t n, float *z, float *logq, void *stream);
/* Where the sampling and density passes (fd_nsf_forward, fd_nsf_sample,
 * fd_nsf_sample_w, fd_nsf_log_density) evaluate the conditioner: 1 (default)
 * = BF16 tensor cores (mma.sync tiles; the weights and every GEMM input
 * rounded to BF16, FP32 accumulation and residual stream: the BF16 contract
 * of the affine flow's sampler), 0 = FP32 CUDA cores.  The splines are FP32
 * on both paths; the training gradient (fd_nsf_kl_grad, fd_nsf_train) is
 * FP32.  FD_EINVAL for another path. */
fd_status fd_nsf_set_tensor_path(fd_nsf *f, int32_t path);
/* Forward-KL training loss of the flow (App. A) and its gradient:
 * loss = -sum_i w_i log q(x_i) / sum_i w_i over device points x [dim][n] in
 * [0, 1]^dim with device weights w [n] (e.g. |f|/q of the proposal that drew
 * them; sum w > 0), and grad = d loss / d parameters (device FP32
 * [fd_nsf_param_count], the parameter layout above, overwritten).  Reverse
 * mode through the inverse pass with the splines' closed-form partials, FP32
 * per sample; loss (device FP64 [1], overwritten) and grad are sums over
 * samples by atomics, so their last bits depend on the order of arrival.
 * n_layers <= 16 (FD_EINVAL otherwise); 1 <= n <= 2^36.  Asynchronous on
 * stream; calls on one flow must not overlap on different streams (they share
 * the flow's weight-sum scratch word). */
fd_status fd_nsf_kl_grad(const fd_nsf *f, const float *x, const float *w, int64_t n, float *grad, double *loss,
                         void *stream);
/* Training on one batch (App. A): `steps` Adam steps (Kingma and Ba: beta =
 * (0.9, 0.999), eps = 1e-8, bias-corrected; the moments live in the flow and
 * persist across calls), each on the gradient of fd_nsf_kl_grad over (x, w)
 * at the current parameters.  loss_out: host FP64 [steps], the loss before
 * each step, or NULL; with it the call waits for the stream.
 * 1 <= steps <= 4096, lr > 0 (FD_EINVAL otherwise). */
fd_status fd_nsf_train(fd_nsf *f, const float *x, const float *w, int64_t n, int32_t steps, float lr,
                       double *loss_out, void *stream);

/* ---- NF-MCMC / VEGAS-MCMC chains (Sec. V, Eqs. target_distr and
 * nf_mcmc_estimator) --------------------------------------------------------
 * Independence Metropolis-Hastings over proposals x ~ q that were already
 * evaluated.  w: device FP32 [n_out][ld], the importance weights
 * w_o = f_o(x)/q(x) of the proposals (e.g. the per-sample output of
 * fd_integrand_eval: on a VEGAS grid q = 1/J, for flow points on the grid
 * q = q_flow/J; rows = (root, Re/Im)); proposal k of chain c is column
 * k * n_chains + c, so ld >= n_chains * n_steps.  The chains sample
 * pi = alpha q + (1 - alpha) |f| with |f| = sum over o < n_sel of |w_o|
 * (0 < alpha <= 1), accept a proposal when u g_t < g' with g = pi/q =
 * alpha + (1 - alpha)|f|/q and u from Philox4x32-10 with counter
 * (chain_lo, chain_hi, iter, 0x40000000 | (step >> 2)), word step & 3, key
 * (seed_lo, seed_hi), u = ((word >> 9) + 0.5) 2^-23; a chain with g_t = 0
 * has no state yet and accepts its first proposal.
 * state: device FP64 [n_out + 1][n_chains], in/out: the chains' current
 *        weights, then g (zero-fill it before the first call).
 * sums:  device FP64 [n_out + 2][n_chains], out: per chain the sums over the
 *        steps k >= n_therm of w_o (1/g) (= f/pi) and of 1/g (= q/pi), then
 *        the number of accepted proposals.
 * FP64 throughout, each operation rounded as written (reproducible bit for
 * bit).  Asynchronous on stream; FD_EINVAL for sizes or alpha out of range
 * (n_out <= 32). */
fd_status fd_mcmc_chains(const float *w, int32_t n_out, int64_t ld, int32_t n_sel, int64_t n_chains,
                         int32_t n_steps, double alpha, uint64_t seed, uint64_t iter, int32_t n_therm,
                         double *state, double *sums, void *stream);
/* Estimates from the chains' sums (Eq. nf_mcmc_estimator): out (device FP64
 * [n_out + 1][2]) row o = (I_o = sum_c A_oc / sum_c B_c, its variance by the
 * delta method over the independent chains: sum_c (A_oc - I_o B_c)^2 /
 * (C (C - 1)) / mean(B)^2), last row = (accepted fraction of the n_chains x
 * n_steps proposals, 0).  Fixed reduction order.  Asynchronous on stream. */
fd_status fd_mcmc_estimate(const double *sums, int32_t n_out, int64_t n_chains, int32_t n_steps, double *out,
                           void *stream);

/* ---- renormalisation post-processing (host, FP64; Sec. VI.A) -------------
 * sigma_re/sigma_im/dsigma_re: FP64 [N+1][N+1][N+1] indexed (n, m, l) holding
 * Sigma^(n,m,l)(k_F, i w0) and d_k Re Sigma^(n,m,l) for n + m + l <= N.
 * Solves dmu(xi) = Re Sigma(xi)|_FS order by order and returns the xi-series
 * coefficients dmu, a, b [N+1] and partial sums meff [N+1] of the series of
 * (1 - b) / (1 + a) (Eq. eff_mass_ratio).  Synchronous, host memory only. */
fd_status fd_postprocess(int32_t N, const double *sigma_re, const double *sigma_im,
                         const double *dsigma_re, double k_F, double beta, double Lambda,
                         double *dmu, double *a, double *b, double *meff);

#ifdef __cplusplus
}
#endif
#endif /* FDCORE_H */
