/*
 * ptsdf.h -- C ABI of the points-as-tori signed-distance library (libptsdf.so).
 *
 * The library evaluates the signed distance of "Points as Tori: Fast Pointwise
 * Signed Distance for Point Clouds" on one NVIDIA B300 (sm_103a):
 *
 *   phi(x) = sum_i g_i(x) w_i(x) / sum_i w_i(x),
 *   w_i(x) = exp(-lambda_x (||x - p_i|| - sigma_x)),
 *   sigma_x = max_i ||x - p_i|| / 2,   lambda_x = C / sigma_x,   C = 64,
 *
 * (Sec. 4.2, Eqs. BasicFormulaShifted and RelationshipBetweenLambdaAndRadius;
 * Algorithm 1, "Inference"), where g_i is the signed distance of a torus fitted
 * at p_i from six coefficients (Sec. 4.1, Eq. SingleTorusSDF).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Pointers named d_* are DEVICE pointers on the current CUDA device; h_*
 *    pointers are HOST pointers (pageable or pinned).  float arrays are
 *    contiguous, row-major, 4-byte aligned; "Q x 3" means x0 y0 z0 x1 y1 z1 ...
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls on device pointers are stream-ordered and return once
 *    the work is enqueued; results are valid after the stream synchronises.
 *  - The caller owns every input and output buffer.  A cloud owns its packed
 *    torus records (device memory) until sdf_destroy.
 *  - Every call returns an sdf_status.  Nothing aborts or exits.  On failure
 *    sdf_last_error() returns a thread-local message.  Kernels that detect a
 *    fault (a bounded wait that ran out) set a per-cloud device status word
 *    instead of trapping; sdf_device_status() reads and clears it.
 *  - Work is not thread-safe per cloud for concurrent *builds*; queries on
 *    one cloud from several host threads/streams are safe (read-only).
 *  - Every call that computes cites the passage of the paper it implements.
 *    The calls that manage resources, report status or measure the device
 *    (sdf_destroy, sdf_cloud_info, sdf_cloud_forms, sdf_device_status, the
 *    sdf_serve_* bookkeeping, sdf_probe_rates, sdf_probe_timing,
 *    sdf_selftest_wait_timeout, sdf_selftest_soft_sqrt,
 *    sdf_profile_*, sdf_kernel_name, sdf_last_error, sdf_version) have no
 *    counterpart in the paper.
 */
#ifndef PTSDF_H
#define PTSDF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PTSDF_API __attribute__((visibility("default")))
#else
#define PTSDF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdf_cloud_s* sdf_cloud;

typedef enum {
    SDF_OK = 0,
    SDF_EINVAL = 1,    /* bad argument (null pointer, negative size, bad option, bad input) */
    SDF_ENOMEM = 2,    /* device or host allocation failed */
    SDF_ECUDA = 3,     /* a CUDA runtime call failed (message has the CUDA error string) */
    SDF_EBUSY = 4,     /* resource in use (serving: no slot / admission refused) */
    SDF_ETIMEOUT = 5,  /* a host-side wait ran out */
    SDF_EDEVICE = 6    /* a kernel reported a fault through the device status word */
} sdf_status;

/* Arithmetic of the weights exp(-lambda_x (d_i - d_min)) in sdf_query (and
 * the calls built on it).  SDF_F32: FP32 throughout.  SDF_F16X2 / SDF_BF16X2:
 * the exponents of a lane's two queries are packed into one register of
 * half / bfloat16 values and evaluated by one packed exp2; distances, the
 * torus SDF and all sums stay FP32.  Gradients are FP32 only. */
typedef enum { SDF_F32 = 0, SDF_F16X2 = 1, SDF_BF16X2 = 2 } sdf_precision;

/* Which units evaluate the pairs of direct-form tori in sdf_query (and in
 * sdf_query_host, the distance steps of sdf_trace, and serving QUERY,
 * Boolean and TRACE_STEP requests).  SDF_ENGINE_AUTO: the
 * tensor cores when precision is SDF_F32, else the FP32 units.
 * SDF_ENGINE_TENSOR: the tensor cores (SDF_EINVAL unless precision is
 * SDF_F32).  SDF_ENGINE_ALU: the FP32 units for every pair.  The tensor-core
 * loop forms |x - p|^2, <x - c, u> and |x - c|^2 as products of split-f16
 * features on the tensor cores and finishes each pair in FP32; pairs where
 * that loses accuracy (query near a torus axis, or far outside the cloud) are
 * recomputed by the FP32 formula.  Points of the kappa form always use the
 * FP32 units.  sdf_query_grad, sdf_backward_params and sdf_query_noalloc
 * (and the normals of sdf_trace) use the FP32 units; the first three reject
 * SDF_ENGINE_TENSOR. */
typedef enum { SDF_ENGINE_AUTO = 0, SDF_ENGINE_ALU = 1, SDF_ENGINE_TENSOR = 2 } sdf_engine;

typedef enum {
    SDF_LAMBDA_GLOBAL = 0,  /* lambda_x = C / sigma_x, sigma_x = max_i ||x - p_i|| / 2 (the paper's rule) */
    SDF_LAMBDA_FIXED = 1,   /* lambda_x = fixed_lambda for every query (Sec. 4.2, "Acceleration and
                               adaptive lambda", without the radius cut-off) */
    SDF_LAMBDA_RADIUS = 2   /* Sec. 4.2, "Acceleration and adaptive lambda": lambda = fixed_lambda (> 0)
                               for every query, and only the points within R_eval = 2 C / lambda of the
                               query are summed; a query with none of them sums over its
                               SDF_RADIUS_FALLBACK_K nearest points.  The paper's lambda is
                               10^3 / D with D from sdf_knn_mean_distance(cloud, 64).  FP32 only;
                               no gradients. */
} sdf_lambda_mode;

enum { SDF_RADIUS_FALLBACK_K = 32 };

typedef enum {
    SDF_FORMULA_BLEND = 0,  /* phi = sum_i A_i w_i g_i / sum_i A_i w_i: Eq. BasicFormulaShifted (the
                               self-normalised blend of the torus SDFs), A_i = 1 unless the cloud
                               was built with weights */
    SDF_FORMULA_LSE = 1,    /* d~ = -(1/lambda) log sum_i A_i exp(-lambda ||x - p_i||): the log-sum-exp
                               distance, Eq. ConvolutionalDistanceFormula with h = 1 (unsigned; the
                               tori are not used).  lambda is the blend's: lambda_x under
                               SDF_LAMBDA_GLOBAL (d~ = d_min where lambda_x = 0, every point at x),
                               fixed_lambda (> 0) under FIXED and RADIUS (the RADIUS set's sum).
                               sdf_query, and sdf_query_grad (d~ and grad d~ = sum A_i w_i n_i / W
                               + (mean distance - d~) / lambda grad lambda_x; d_saved must be
                               NULL); no parameter gradients, Laplacian, level-set sampling or
                               sphere tracing. */
    SDF_FORMULA_SSPD = 2,   /* phi_SSPD = sum_i A_i <x - p_i, n_i> e_i / sum_i A_i e_i: the smoothed signed
                               planar distance, Eq. SmoothedSignedPlanarDistance (Sec. 5's first
                               baseline), e_i = exp(-lambda (||x - p_i|| - sigma_x)), n_i the unit input
                               normal; the tori are not used.  lambda is the blend's (lambda_x under
                               GLOBAL, fixed_lambda >= 0 under FIXED). */
    SDF_FORMULA_SHC = 3     /* phi_SHC = sign(w) (-(1/lambda) log|w| + sigma_x) with the screened
                               double-layer sum w = sum_i A_i (lambda d_i + 1) <x - p_i, n_i> e_i /
                               (2 pi d_i^3): the signed Hopf-Cole distance (screened winding number),
                               Eq. ScreenedWindingNumber (Sec. 5's second baseline).  lambda_x under
                               GLOBAL, fixed_lambda > 0 under FIXED.  A point at the query adds
                               nothing to w; w = 0 gives +inf; a query at every point gives 0.
                               SSPD and SHC: sdf_query and sdf_query_host only; FP32, GLOBAL or
                               FIXED lambda, on the FP32 units (SDF_ENGINE_TENSOR is refused). */
} sdf_formula;

typedef struct {
    int32_t lambda_mode;   /* sdf_lambda_mode */
    int32_t precision;     /* sdf_precision (SDF_F32 is the reference path) */
    float C;               /* screening constant C of Eq. RelationshipBetweenLambdaAndRadius (64) */
    float fixed_lambda;    /* lambda for SDF_LAMBDA_FIXED, >= 0 */
    float offset;          /* returned value is phi(x) - offset (offset surfaces, Sec. 6) */
    int32_t split_n;       /* number of point chunks per query block; 0 = automatic.  The
                              automatic choice depends only on (Q, N, SM count), so a query's
                              result does not depend on what else runs.  An explicit split also
                              makes a batch too small for the one-thread-per-query pruned
                              prepass take the point-split full scan rather than the
                              warp-per-query pruned one (the same d_max, d_min bit for bit). */
    int32_t engine;        /* sdf_engine (SDF_ENGINE_AUTO) */
    int32_t formula;       /* sdf_formula (SDF_FORMULA_BLEND) */
} sdf_query_opts;

/* Fills *opts with the paper's defaults: GLOBAL lambda, C = 64, F32, offset 0,
 * automatic split, automatic engine, the blend.  Returns SDF_EINVAL for NULL. */
PTSDF_API sdf_status sdf_opts_default(sdf_query_opts* opts);

/* ---------------------------------------------------------------------------
 * sdf_build -- fit one torus per point and pack the cloud for querying.
 *   Sec. 4.1 (Eqs. BivariatePolynomial, MeanAndGaussCurvatures,
 *   PrincipalDirections, TorusSigns; App. C); Algorithm 1, "Precomputation"
 *   with the per-point coefficients given as input.
 *
 *   d_points   N x 3 float, point positions p_i.
 *   d_normals  N x 3 float, oriented normals n_i (normalised here; need not
 *              be unit).  The local frame (s_i, t_i) of n_i is the branchless
 *              orthonormal basis of Duff et al. 2017.
 *   d_params   N x 6 float per point: a00, a01, a10, a11, a02, a20 of
 *              Q(s,t) = a00 + a10 s + a01 t + a11 s t + a20 s^2 + a02 t^2.
 *   n          number of points, 1 <= n <= 2^31 - 1.
 *   out        receives the new cloud handle.
 *   The fit runs in double precision on the device; the cloud copies what it
 *   needs (inputs may be freed after the stream synchronises).  The call
 *   synchronises `stream` once (to size the packed layout).
 *   Errors: SDF_EINVAL for n < 1, NULL pointers, or a zero / non-finite
 *   normal or non-finite input (detected on the device, reported here);
 *   SDF_ENOMEM; SDF_ECUDA.
 * ------------------------------------------------------------------------- */
PTSDF_API sdf_status sdf_build(const float* d_points, const float* d_normals, const float* d_params,
                     int64_t n, void* stream, sdf_cloud* out);

/* sdf_build with per-point weights A_i: every sum over points (the blend,
 * its gradients and Laplacian, the parameter gradient, the radius-limited
 * sum and the log-sum-exp distance) weighs point i by A_i.  They are the
 * area weights of the discretised surface integral of Eq.
 * SelfNormalizedConvolutionalDistanceFormula, which Eq. BasicFormulaShifted
 * leaves out (sdf_build: all A_i = 1).
 *   d_weights  N float on the device, each in [2^-64, 2^64] (else SDF_EINVAL,
 *              detected on the device; the range keeps every FP32 sum finite
 *              and non-zero); NULL is sdf_build.
 *   With the tensor engine, a weighted cloud's direct-form tiles take the
 *   tensor cores (the weight scales the per-point constants of their B tiles)
 *   and its curvature-form tiles the FP32 units. */
PTSDF_API sdf_status sdf_build_weighted(const float* d_points, const float* d_normals, const float* d_params,
                              const float* d_weights, int64_t n, void* stream, sdf_cloud* out);

/* ---------------------------------------------------------------------------
 * Checkpoint of a built cloud (no counterpart in the paper; its precomputation
 * is Algorithm 1 "Precomputation": the tori fitted from the per-point
 * coefficients, Sec. 4.1).
 *
 * sdf_export -- writes the cloud into a host buffer: its inputs (points,
 *   normals, the six coefficients, the weights of a weighted cloud) and the
 *   fitted torus records, so that sdf_import rebuilds it without fitting.
 *   buf == NULL: *size receives the bytes needed and nothing else happens.
 *   Else cap must be at least that size (SDF_EINVAL otherwise) and *size
 *   receives the bytes written.  Synchronous (device-wide copies).  The
 *   layout is this library's: a 24-byte header ("PTSDFCK", version 1, the
 *   weighted flag, n), then the arrays in host byte order.
 * sdf_import -- builds a cloud on the current device from an sdf_export
 *   buffer of `size` bytes; every query of the imported cloud equals that of
 *   the exported one bit for bit.  SDF_EINVAL (before any CUDA call) for a
 *   buffer that is not an export of version 1 or whose size does not match
 *   its header; the records are taken as written (the export checked them).
 *   Synchronises `stream` before returning.
 * ------------------------------------------------------------------------- */
PTSDF_API sdf_status sdf_export(sdf_cloud cloud, void* buf, int64_t cap, int64_t* size);
PTSDF_API sdf_status sdf_import(const void* buf, int64_t size, void* stream, sdf_cloud* out);

/* Releases a cloud (synchronises the device first).  NULL is a no-op. */
PTSDF_API sdf_status sdf_destroy(sdf_cloud cloud);

/* Cloud facts: number of points, the diagonal of the points' axis-aligned
 * bounding box (the error scale of the FP32 tolerance), and how many points
 * use the direct (radius) torus form vs the curvature (kappa) form. */
PTSDF_API sdf_status sdf_cloud_info(sdf_cloud cloud, int64_t* n, float* aabb_diag, int64_t* n_direct,
                          int64_t* n_kappa);

/* More cloud facts, for cost accounting: how many curvature-form points have
 * kappa_min = 0 (planes, cylinders; they take the shorter formula of the
 * form, Sec. 4.1), and how many 32-record tiles of the tensor-core loop
 * take the FP32 record formula because a coefficient (e.g. kappa_max times
 * the coordinate scale, above 2^15) leaves its f16 split's range.  Either
 * pointer may be NULL; exact_tiles synchronises the device. */
PTSDF_API sdf_status sdf_cloud_forms(sdf_cloud cloud, int64_t* n_kappa_flat, int64_t* exact_tiles);

/* ---------------------------------------------------------------------------
 * sdf_query -- phi at Q query points (Algorithm 1, "Inference"; Eqs.
 *   BasicFormulaShifted, RelationshipBetweenLambdaAndRadius, SingleTorusSDF).
 *
 *   d_x     Q x 3 float query positions.
 *   q       number of queries, >= 0 (0 is a no-op).
 *   d_phi   Q float, receives phi(x) - opts->offset.
 *   opts    NULL = sdf_opts_default.
 *   Under SDF_LAMBDA_GLOBAL and SDF_LAMBDA_FIXED every (query, point) pair
 *   is evaluated (no cut-off); SDF_LAMBDA_RADIUS sums each query's radius set
 *   only (see sdf_lambda_mode).  Scratch memory is taken from the
 *   stream-ordered allocator and returned on the stream.
 *   Errors: SDF_EINVAL (NULL pointers with q > 0, bad opts); SDF_ENOMEM;
 *   SDF_ECUDA.  Kernel faults show up in sdf_device_status.
 * ------------------------------------------------------------------------- */
PTSDF_API sdf_status sdf_query(sdf_cloud cloud, const float* d_x, int64_t q, float* d_phi,
                     const sdf_query_opts* opts, void* stream);

/* As sdf_query (Algorithm 1, "Inference") with HOST buffers: copies h_x to the device, evaluates, copies
 * phi back into h_phi, and synchronises `stream` before returning (so h_phi
 * is valid on return).  Large batches are cut into chunks whose copies
 * overlap the evaluation of the previous chunk.  Pinned host memory gives
 * the fastest copies; pageable memory works. */
PTSDF_API sdf_status sdf_query_host(sdf_cloud cloud, const float* h_x, int64_t q, float* h_phi,
                          const sdf_query_opts* opts, void* stream);

/* Reads and clears the cloud's device status word (synchronises `stream`).
 * *code = 0 when no kernel reported a fault; otherwise a bit set of
 * SDF_DEV_* codes.  Returns SDF_EDEVICE when *code != 0. */
enum { SDF_DEV_WAIT_TIMEOUT = 1, SDF_DEV_BAD_INPUT = 2 };
PTSDF_API sdf_status sdf_device_status(sdf_cloud cloud, void* stream, int32_t* code);

/* ---------------------------------------------------------------------------
 * sdf_query_grad -- phi and d phi / d x (App. D, "Gradient expressions",
 *   plus the x-dependence of lambda_x through the farthest point).
 *
 *   d_phi      Q float (phi - offset).
 *   d_grad     Q x 3 float, d phi / d x.
 *   d_saved    Q x 8 float or NULL: per-query statistics for
 *              sdf_backward_params {x, y, z, L, A0, W, phi, 0} where the
 *              weights are w_i = 2^(A0 - L |x - p_i|) (L = lambda_x log2 e,
 *              A0 = L d_min), W = sum_i w_i and phi excludes the offset.
 *   Where two points tie for the farthest, lambda_x has a kink; the
 *   gradient then uses one of them.
 *   Errors as sdf_query.
 * ------------------------------------------------------------------------- */
PTSDF_API sdf_status sdf_query_grad(sdf_cloud cloud, const float* d_x, int64_t q, float* d_phi,
                          float* d_grad, float* d_saved, const sdf_query_opts* opts, void* stream);

/* ---------------------------------------------------------------------------
 * sdf_backward_params -- d L / d(a00..a20) for L = sum_q G_q phi(x_q): the
 *   weights do not depend on the coefficients, so
 *   dL/da_i = sum_q G_q (w_qi / W_q) d g_i(x_q) / d a_i, chained through the
 *   fit of Sec. 4.1.
 *
 *   d_saved        Q x 8 float written by sdf_query_grad for the same d_x.
 *   d_grad_phi     Q float, G_q.
 *   d_grad_params  N x 6 float in the ORIGINAL point order; overwritten
 *                  (zeros when q == 0).
 *   opts           must equal the options of the sdf_query_grad call.
 *   The chain through the fit runs in double precision.  At a zero
 *   curvature the derivative is that of the curvature form's smooth
 *   continuation through zero.
 *   Errors as sdf_query.
 * ------------------------------------------------------------------------- */
PTSDF_API sdf_status sdf_backward_params(sdf_cloud cloud, const float* d_x, int64_t q, const float* d_saved,
                               const float* d_grad_phi, float* d_grad_params,
                               const sdf_query_opts* opts, void* stream);

/* ---------------------------------------------------------------------------
 * sdf_trace -- sphere tracing of the level set phi = offset (Sec. 6, "Direct
 *   visualization of point cloud surfaces").  From t = 0 each step evaluates
 *   f = phi(o + t d) - offset; a ray hits when f < eps (t_hit = t), else
 *   t += f; it misses when t > t_max or after max_steps evaluations
 *   (t_hit = -1).  Each step is one query batch over the rays still live.
 *
 *   d_origins, d_dirs  R x 3 float (dirs unit length).
 *   d_t_hit            R float; d_steps R int32 (evaluations used).
 *   d_normals          R x 3 float or NULL: unit grad phi at hits (0 at misses).
 *   The call synchronises `stream` once per step (the live-ray count sizes
 *   the next batch) and returns when the results are written.
 *   Errors as sdf_query; SDF_EINVAL for nrays < 0, max_steps < 1, eps <= 0 or
 *   t_max <= 0.
 * ------------------------------------------------------------------------- */
PTSDF_API sdf_status sdf_trace(sdf_cloud cloud, const float* d_origins, const float* d_dirs, int64_t nrays,
                     int32_t max_steps, float eps, float t_max, float* d_t_hit, int32_t* d_steps,
                     float* d_normals, const sdf_query_opts* opts, void* stream);

/* Booleans of two phi arrays (Sec. 6, "Offset surfaces and Booleans"):
 * union min(a, b), intersection max(a, b), difference max(a, -b). */
typedef enum { SDF_UNION = 0, SDF_INTERSECT = 1, SDF_DIFFERENCE = 2 } sdf_bool_op;
PTSDF_API sdf_status sdf_combine(int32_t op, const float* d_a, const float* d_b, int64_t q, float* d_out,
                       void* stream);

/* ---------------------------------------------------------------------------
 * sdf_query_noalloc -- sdf_query (Algorithm 1, "Inference") that allocates
 *   nothing.  The allocation-free form has no counterpart in the paper; it
 *   is a service of this library.
 *
 *   For callers that must not touch the CUDA allocator once they are running:
 *   latency-bound loops (a renderer asking for phi every frame, a controller
 *   checking clearance every cycle), where cudaMalloc / cudaMallocAsync can
 *   block, synchronise or fail at the worst moment, and services that reserve
 *   all of their device memory at start-up and treat any later allocation as
 *   an error.
 *
 *   Same arguments as sdf_query, and the same option checks and errors,
 *   with these refused as well (SDF_EINVAL): SDF_LAMBDA_RADIUS, the
 *   packed-half precisions (SDF_F16X2, SDF_BF16X2) and SDF_ENGINE_TENSOR.
 *   Every pair is evaluated on the FP32 units (SDF_ENGINE_AUTO included),
 *   while sdf_query's default engine uses the tensor cores, so the two
 *   results agree within the FP32 tolerance (1e-4 x the cloud's bounding-box
 *   diagonal), not bit for bit.  The scratch lives in one fixed 8 MiB array
 *   compiled into the library.  Every GPU that loads the library holds that
 *   array until the process exits.
 *   - Limit: q <= 1,048,576 queries per call; larger q returns SDF_EINVAL with
 *     a message (split the batch).  For small batches the number of point
 *     chunks is reduced until the chunk partials fit.
 *   - The first call on each device looks up the array's device address
 *     (with that device current); make that first call before any stream
 *     capture.
 *   - Every call on a device shares the one array and it keeps the last
 *     call's contents (every entry is written before it is read, so nothing
 *     needs clearing).  Calls whose kernels overlap on the GPU (different
 *     streams, or several host threads) race on it: serialise them.
 * ------------------------------------------------------------------------- */
PTSDF_API sdf_status sdf_query_noalloc(sdf_cloud cloud, const float* d_x, int64_t q, float* d_phi,
                                       const sdf_query_opts* opts, void* stream);

/* ---------------------------------------------------------------------------
 * Serving: a request loop over several resident clouds (Sec. 6 uses of the
 * SDF: query batches of uneven size, sphere-tracing steps, offsets and
 * Booleans).  A scheduler thread admits queued requests (in arrival order, or
 * smallest first) when a slot (max_inflight) and enough of the memory budget are free and
 * launches each at once on one of n_streams streams (the least loaded of its
 * priority class), so work that arrives while other requests run overlaps
 * with them on the device.  A request's
 * result depends only on its own inputs, cloud and options: it is the same
 * alone and in a mix.
 * ------------------------------------------------------------------------- */
typedef struct sdf_server_s* sdf_server;

typedef enum {
    SDF_SERVE_FIFO = 0,            /* admit in arrival order */
    SDF_SERVE_SMALLEST_FIRST = 1   /* admit the queued request with the fewest (query, point) pairs
                                      first; a request queued longer than starve_ms goes first */
} sdf_serve_policy;

typedef struct {
    int64_t mem_budget_bytes;   /* device bytes the server may hold for staging and scratch */
    int32_t max_inflight;       /* requests on the GPU at once (slots) */
    int32_t n_streams;          /* CUDA streams the requests are spread over */
    int32_t device;             /* CUDA device of the clouds */
    int32_t policy;             /* sdf_serve_policy */
    int32_t starve_ms;          /* SMALLEST_FIRST: age after which a request is admitted first */
    int32_t split_gpairs;       /* requests of more (query, point) pairs than split_gpairs x 1e9 run as
                                   query chunks that are admitted one after another, each queued
                                   behind the requests waiting when the previous one started (0:
                                   never split).  A chunk keeps at least 2 x 4 x SMs x 512 queries,
                                   so every query's result is exactly that of the unsplit request;
                                   GRAD requests are not split. */
    float express_gpairs;       /* > 0: requests (and chunks) of at most express_gpairs x 1e9 pairs
                                   run on the first half of the streams, created at the device's
                                   highest stream priority, the others on the second half at the
                                   lowest, so the block scheduler starts a small request's blocks
                                   before the queued blocks of large ones; and the larger requests
                                   hold at most max_inflight - max_inflight / 2 slots at once, so
                                   a small one never waits for a slot behind them.  0: one
                                   priority, no reservation.  Either way a request goes to the
                                   stream of its class with the least work in flight.  Needs
                                   n_streams >= 2 when > 0. */
} sdf_serve_config;

typedef enum {
    SDF_REQ_QUERY = 0,       /* out[q]      = phi(x) - offset */
    SDF_REQ_GRAD = 1,        /* out[4q]     = phi (q floats) then grad phi (q x 3) */
    SDF_REQ_UNION = 2,       /* out[q]      = min(phi_a, phi_b) */
    SDF_REQ_INTERSECT = 3,   /* out[q]      = max(phi_a, phi_b) */
    SDF_REQ_DIFFERENCE = 4,  /* out[q]      = max(phi_a, -phi_b) */
    SDF_REQ_TRACE_STEP = 5   /* out[q]      = phi(x + t dirs) - offset (one sphere-tracing step) */
} sdf_request_kind;

typedef struct {
    int32_t kind;            /* sdf_request_kind */
    int32_t cloud_id;        /* from sdf_serve_register */
    int32_t cloud_id_b;      /* second cloud of a Boolean */
    int32_t host_buffers;    /* 1: x, dirs, t, out are host pointers (staged by the server); 0: device */
    const float* x;          /* q x 3 positions (TRACE_STEP: ray origins) */
    const float* dirs;       /* TRACE_STEP: q x 3 directions; else NULL */
    const float* t;          /* TRACE_STEP: q ray parameters; else NULL */
    int64_t q;               /* >= 1 */
    float* out;              /* see sdf_request_kind */
    sdf_query_opts opts;
} sdf_request;

typedef struct {
    int32_t status;          /* sdf_status of the request */
    int32_t chunks;          /* query chunks it ran as (1 unless split, see split_gpairs) */
    int64_t arrive_ns;       /* host steady-clock times: submit, */
    int64_t admit_ns;        /*   admission (of the first chunk), */
    int64_t start_ns;        /*   launch (of the first chunk), */
    int64_t done_ns;         /*   completion of the request's last operation */
    double device_ms;        /* CUDA-event time of the request's work on its stream (summed over chunks) */
} sdf_request_stats;

/* Creates a server (and its scheduler thread and streams). */
PTSDF_API sdf_status sdf_serve_create(const sdf_serve_config* cfg, sdf_server* out);
/* Makes a built cloud addressable by requests; the cloud must outlive the server. */
PTSDF_API sdf_status sdf_serve_register(sdf_server srv, sdf_cloud cloud, int32_t* cloud_id);
/* Queues a request (any host thread).  Buffers must stay valid until the
 * request is polled.  SDF_ENOMEM if the request alone exceeds the memory
 * budget; SDF_EINVAL for bad arguments; SDF_EBUSY after shutdown began. */
PTSDF_API sdf_status sdf_serve_submit(sdf_server srv, const sdf_request* req, uint64_t* ticket);
/* Waits up to timeout_us (negative: without limit) for a request;
 * SDF_ETIMEOUT if it is not finished (the ticket stays valid), else the
 * request's status (the ticket is released) and its timestamps in *stats. */
PTSDF_API sdf_status sdf_serve_poll(sdf_server srv, uint64_t ticket, int64_t timeout_us, sdf_request_stats* stats);
/* Current queue length, requests in flight and bytes charged to the budget. */
PTSDF_API sdf_status sdf_serve_stats(sdf_server srv, int32_t* queued, int32_t* inflight, int64_t* mem_in_use);
/* Finishes every queued request, joins the scheduler and frees the server. */
PTSDF_API sdf_status sdf_serve_shutdown(sdf_server srv);

/* ---------------------------------------------------------------------------
 * sdf_project_level_set -- samples of a level set of phi with normals, the
 *   first half of the paper's morphological operations (Sec. 6,
 *   "Morphological operations": sample the -c level set of phi and take the
 *   normals at the moved points from grad phi; the re-fit of tori at those
 *   points needs the paper's network and is not done here).
 *
 *   Each seed x0 moves by Newton steps along the gradient,
 *     x <- x - (phi(x) - level) grad phi(x) / |grad phi(x)|^2,
 *   at most max_iter of them (0..100); a seed stops once |phi - level| <= tol
 *   or its gradient vanishes.  Then phi and grad phi are evaluated once more.
 *   d_x0       Q x 3 seeds (for erosion, the cloud's own points).
 *   d_x        Q x 3 out: the moved points (may be d_x0: in place).
 *   d_normals  Q x 3 out: grad phi / |grad phi| at the moved points.
 *   d_residual Q out: phi - level there.
 *   opts: as sdf_query_grad (FP32, GLOBAL or FIXED lambda, the blend); the
 *   offset is ignored (level takes its part).  Costs max_iter + 1 gradient
 *   evaluations of Q queries.
 * ------------------------------------------------------------------------- */
PTSDF_API sdf_status sdf_project_level_set(sdf_cloud cloud, const float* d_x0, int64_t q, float level,
                                 int32_t max_iter, float tol, float* d_x, float* d_normals, float* d_residual,
                                 const sdf_query_opts* opts, void* stream);

/* ---------------------------------------------------------------------------
 * sdf_query_laplacian -- phi, grad phi and the Laplacian lap phi at Q points
 * (App. D, "Laplacian"): the divergence of the gradient of the blend, with
 * lap g_i of each torus in closed form (lap D = 1/D + (rho - R)/(rho D) for
 * D the distance to the tube's centre circle, and the same quantity in the
 * curvature form) and, for SDF_LAMBDA_GLOBAL, the terms of lambda_x(x)
 * (lambda_x = 2C / d_max(x) is harmonic, so only its gradient enters).
 * Diagnostics of the SDF: |grad phi| - 1 (eikonal residual) and lap phi
 * (twice the mean curvature of the level set on the surface).
 *   d_phi, d_grad (Q x 3) may be NULL; d_lap (Q) is required.  FP32;
 *   GLOBAL or FIXED lambda; the same point-chunk plan as sdf_query_grad.
 *   Accuracy: about 1e-2 (1 + |lap phi|) at worst, because the FP32 sums
 *   include terms of size lambda sum w / d that cancel exactly.
 * ------------------------------------------------------------------------- */
PTSDF_API sdf_status sdf_query_laplacian(sdf_cloud cloud, const float* d_x, int64_t q, float* d_phi, float* d_grad,
                                         float* d_lap, const sdf_query_opts* opts, void* stream);

/* ---------------------------------------------------------------------------
 * sdf_orient -- orientation repair of an inconsistently oriented cloud
 * (Sec. 6, "Orienting inconsistently oriented point clouds").  Each
 * iteration builds the cloud, evaluates grad phi at its points, and for every
 * point i forms n~_i = sum over its k nearest other points j of
 * exp(-M_i(p_i - p_j)) grad phi(p_j), with the curvature-scaled length
 * M_i(r) = sqrt(kmin^2 <r, v_min>^2 + kmax^2 <r, v_max>^2 + eps^2 <r, n_i>^2)
 * (principal curvatures and directions of point i's fit, eps = 1 / the mean
 * distance to the k nearest).  Points with <n_i, n~_i> < 0 are flipped: n_i
 * is negated and its six coefficients re-expressed, for the same quadratic
 * patch, in the frame of -n_i (so its torus is the same torus with the
 * opposite sign).  All points decide from the same cloud; iterations stop
 * when nothing flips or after max_iter.
 *   d_points N x 3 (read), d_normals N x 3 and d_params N x 6 (device, read
 *   and overwritten).  k in [1, 64] (16 is a reasonable default); opts as for
 *   sdf_query_grad (GLOBAL or FIXED lambda, FP32).  flips (host, max_iter
 *   entries) receives the flip count of each iteration run, *iterations their
 *   number.  Synchronous on `stream`.
 * ------------------------------------------------------------------------- */
PTSDF_API sdf_status sdf_orient(const float* d_points, float* d_normals, float* d_params, int64_t n, int32_t k,
                                int32_t max_iter, const sdf_query_opts* opts, int32_t* flips, int32_t* iterations,
                                void* stream);

/* ---------------------------------------------------------------------------
 * sdf_knn_mean_distance -- D of the lambda heuristic of Sec. 4.2
 * ("Acceleration and adaptive lambda"): for every point of the cloud the
 * mean of the distances to its k nearest other points (all of them when the
 * cloud has k or fewer other points), averaged over the points, in FP64 from
 * FP32 distances.  k in [1, 64] (the paper uses 64).  The paper then sets
 * lambda = 10^3 / D and R_eval = 2 C / lambda (SDF_LAMBDA_RADIUS).
 * Synchronous on `stream`; a one-point cloud gives D = 0.
 * ------------------------------------------------------------------------- */
PTSDF_API sdf_status sdf_knn_mean_distance(sdf_cloud cloud, int32_t k, double* D, void* stream);

/* The paper's constant lambda of the radius-limited evaluation (Sec. 4.2,
 * "Acceleration and adaptive lambda"): *lambda = 10^3 / D with D =
 * sdf_knn_mean_distance(cloud, 64) (also returned in *D unless D is NULL).
 * Synchronous on `stream`.  SDF_EINVAL when D = 0 (one point, or all points
 * coincide). */
PTSDF_API sdf_status sdf_paper_lambda(sdf_cloud cloud, double* lambda, double* D, void* stream);

/* ---------------------------------------------------------------------------
 * sdf_mesh_level_set -- the level-`level` surface of a phi grid (offset
 * surfaces and morphological operations, Sec. 6), by marching tetrahedra.
 *   d_phi: nz x ny x nx FP32 values (x fastest) on the device, node (i, j, k)
 *   at origin + (i, j, k) * spacing (origin, spacing: 3 host floats each).
 *   Every grid cube is split into the six tetrahedra of its Kuhn
 *   triangulation, so the surface is watertight; a node is inside when
 *   phi < level.  Vertices (one per cut edge of the triangulation, FP32
 *   x, y, z) are numbered by (lower node index, edge direction x, y, z, xy,
 *   xz, yz, xyz); triangles (3 int32 vertex numbers) are listed cube by cube
 *   with normals pointing from phi < level to phi >= level.
 *   Always sets *n_vertices and *n_triangles.  With d_vertices and
 *   d_triangles NULL it only counts; with both given and large enough
 *   (cap_* entries) it also writes them; otherwise SDF_EINVAL.  Synchronous
 *   on `stream`.  SDF_EINVAL for a dimension below 2 or more than 2^31
 *   nodes, vertices or triangles.
 * ------------------------------------------------------------------------- */
PTSDF_API sdf_status sdf_mesh_level_set(const float* d_phi, int32_t nx, int32_t ny, int32_t nz, const float* origin,
                                        const float* spacing, float level, float* d_vertices, int64_t cap_vertices,
                                        int32_t* d_triangles, int64_t cap_triangles, int64_t* n_vertices,
                                        int64_t* n_triangles, void* stream);

/* ---------------------------------------------------------------------------
 * Kernel timing (a tracing aid, not part of the method).  While enabled,
 * every kernel the library launches is bracketed by two CUDA events recorded
 * on the stream it is launched on.  sdf_profile_read waits for the recorded
 * events and returns, for one kernel family, the number of launches and
 * their total device time in milliseconds since the last enable.  Enabling
 * clears earlier records; disabling stops recording and keeps them.
 * ------------------------------------------------------------------------- */
/* Measures, on the current device, the sustained throughput of the
 * operations that bound the pair loops, in results per SM per SM clock
 * (per SM, its CTAs' results over the union of their %globaltimer windows,
 * at the SM clock measured in the kernel):
 * rates[0] sqrt.approx, rates[1] rsqrt.approx, rates[2] ex2.approx (the
 * special-function unit), rates[3] FP32 FMA and rates[4] rcp.approx; and,
 * in pairs per SM per clock, the special-function work of one pair as the
 * pair loops issue it: rates[5] direct form (3 sqrt + 1 exp2), rates[6]
 * curvature form with kappa_min = 0 (2 sqrt + 1 rcp + 1 exp2), rates[7]
 * other curvature form (3 sqrt + 2 rcp + 1 exp2).  A measurement aid for
 * roofline reporting (about 20 ms of kernels on every SM); it does not touch
 * any cloud.  rates must hold 8 doubles. */
PTSDF_API sdf_status sdf_probe_rates(double* rates);

/* Three readings of one rate of sdf_probe_rates (a measurement aid, no
 * counterpart in the paper): runs probe `op` (0..7, the index into rates
 * above) once more and returns out[0] the rate per SM clock over the longest
 * single CTA's clock64 window of each SM (overstates when an SM's CTAs do not
 * run in lockstep), out[1] the rate over the union of the SM's CTA windows
 * timed by %globaltimer and converted to SM clocks with the clock measured in
 * the kernel (what sdf_probe_rates reports), out[2] results per SM per ns
 * from the launch's CUDA-event time (all SMs), and out[3] that measured SM
 * clock in GHz (clock64 cycles over %globaltimer ns, mean over the CTAs).
 * out[2] / out[3] is the event-timed rate per clock.  out must hold 4
 * doubles. */
PTSDF_API sdf_status sdf_probe_timing(int32_t op, double* out);

/* Self-test of the failure path (not part of the method): launches one
 * kernel whose thread waits, through the same bounded mbarrier wait the pair
 * loops use but with a limit of limit_us microseconds (1 .. 1e6), on a phase
 * that nothing completes.  The wait gives up, the kernel records
 * SDF_DEV_WAIT_TIMEOUT in its own status word and returns: *status_bits
 * receives that word (SDF_DEV_WAIT_TIMEOUT expected) and *waited_ms the time
 * the wait took.  Nothing faults or hangs, and the context stays usable. */
PTSDF_API sdf_status sdf_selftest_wait_timeout(int32_t limit_us, int32_t* status_bits, double* waited_ms);

/* Self-test of the square root the tensor-core epilogue computes on the FMA
 * pipe (no counterpart in the paper): over 2^25 positive normal floats from
 * 1e-30 up, the largest relative difference from CUDA's correctly rounded
 * sqrtf (about 4.7e-6 expected: two Newton steps from a bit-level
 * estimate). */
PTSDF_API sdf_status sdf_selftest_soft_sqrt(double* max_rel_err);

enum { SDF_K_PREPASS = 0, SDF_K_FWD = 1, SDF_K_MERGE = 2, SDF_K_BUILD = 3, SDF_K_FWD_GRAD = 4, SDF_K_BWD = 5,
       SDF_K_FWD_TC = 6, SDF_K_RADIUS = 7, SDF_K_KNN = 8, SDF_K_PLANE = 9, SDF_K_COUNT_ = 10 };
PTSDF_API sdf_status sdf_profile_enable(int32_t on);
PTSDF_API sdf_status sdf_profile_read(int32_t kernel, int64_t* launches, double* total_ms);
/* Name of a kernel family (NULL for an id out of range). */
PTSDF_API const char* sdf_kernel_name(int32_t kernel);

/* Thread-local description of the last failure on this thread ("" if none). */
PTSDF_API const char* sdf_last_error(void);

/* Library version string. */
PTSDF_API const char* sdf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PTSDF_H */
