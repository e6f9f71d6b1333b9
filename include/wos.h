/*
 * wos.h -- C ABI of the GB300 walk-on-ellipsoids operator library.
 *
 * The library builds, on one GPU, the Monte Carlo estimate of the discretised
 * direct operator of the Cauchy / data-completion problem of Cimpean, Grecu
 * & Marin, "Numerical spectral analysis of Cauchy-type inverse problems: a
 * probabilistic approach" (arXiv:2409.03686), then its FP64 SVD and the
 * truncated-SVD reconstruction of the Dirichlet data on Gamma_1.
 *
 * Conventions for every entry point
 *   - Array arguments marked "device" are pointers to memory of the device
 *     the context was created on; "host" arrays are read during the call and
 *     may be freed when it returns.  The caller owns every array it passes.
 *   - Descriptor structs are copied during the call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Device work is enqueued on it; unless stated otherwise a call
 *     returns without waiting for that work.
 *   - Errors are returned as wos_status and never abort the process.  On an
 *     error other than a warning nothing was enqueued.
 *   - Matrices are row-major.  Element (boundary cell) indices run over the
 *     outer boundary component first, then hole 0, hole 1, ...
 */
#ifndef WOS_H
#define WOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WOS_OK = 0,
    WOS_INVALID_ARG = 1,        /* a size, pointer or descriptor field is bad */
    WOS_K_NOT_SPD = 2,          /* K is not symmetric positive definite */
    WOS_POINT_OUTSIDE = 3,      /* an observation point lies outside D */
    WOS_EPS_BELOW_FP32_FLOOR = 4, /* FP32 walks need eps >= the floor below */
    WOS_COUNT_OVERFLOW = 5,     /* a count could exceed 2^32 - 1 */
    WOS_STEP_CAP_HIT = 6,       /* warning: some walks hit the step cap; the
                                   counts are valid and unterminated > 0 */
    WOS_DEVICE_TIMEOUT = 7,     /* a bounded device-side wait gave up */
    WOS_OOM = 8,                /* a device allocation failed */
    WOS_CUDA_ERROR = 9,         /* a CUDA runtime call failed */
    WOS_NO_CONVERGENCE = 10,    /* Jacobi SVD did not converge in max sweeps */
    WOS_TRUNCATION_IN_CLUSTER = 11, /* warning: sigma_r / sigma_{r+1} < 1.5 */
    WOS_NOT_READY = 12,         /* a queued request is not finished yet */
    WOS_NOALLOC_LIMIT = 13      /* the problem needs more than the fixed scratch
                                   of wos_build_operator_noalloc */
} wos_status;

#define WOS_MAX_VERTICES 64
#define WOS_MAX_HOLES 16

typedef enum {
    WOS_OUTER_SPHERE = 1,  /* disc (dim 2) or ball (dim 3) */
    WOS_OUTER_BOX = 2,     /* axis-aligned rectangle (dim 2) or box (dim 3) */
    WOS_OUTER_POLYGON = 3  /* simple polygon, vertices counter-clockwise (dim 2) */
} wos_outer_kind;

/* D = outer body minus disjoint closed holes (discs in 2-D, balls in 3-D).
 * Unused fields are ignored. */
typedef struct {
    int32_t dim;        /* 2 or 3 */
    int32_t outer_kind; /* wos_outer_kind */
    double center[3];   /* sphere / box centre */
    double radius;      /* sphere radius */
    double half[3];     /* box half-extents */
    int32_t n_vertices; /* polygon vertex count, 3..WOS_MAX_VERTICES */
    double vertices[2 * WOS_MAX_VERTICES]; /* (x, y) pairs, counter-clockwise */
    int32_t n_holes;    /* 0..WOS_MAX_HOLES */
    double hole_center[WOS_MAX_HOLES][3];
    double hole_radius[WOS_MAX_HOLES];
} wos_domain;

/* Partition of dD into boundary elements (the cells of the intrinsic Voronoi
 * weights, paper App. A, Ex. A.3, or of the extrinsic ones, Ex. A.2).
 *   circle (2-D sphere / hole): m arcs counter-clockwise from theta0,
 *       arc j = [theta0 + 2 pi j/m, theta0 + 2 pi (j+1)/m).
 *   polygon / 2-D box: edge e (v_e -> v_{e+1}; for a box the edges are
 *       bottom, right, top, left from the corner c - h) in edge_m[e] equal
 *       cells.
 *   3-D sphere / hole: nb equal-height z-bands (band 0 at the south pole)
 *       times ns phi-sectors from phi = 0; cell = band * ns + sector.
 *   3-D box: faces -x, -y, -z, +x, +y, +z, each face_n1 x face_n2 cells over
 *       its two other axes in increasing axis order.
 * A point is assigned through its nearest boundary point (the projection pi
 * of App. A); ties go to the lowest element index (Ex. A.3).
 * voronoi_n > 0 replaces all of the above by the extrinsic Voronoi cells of
 * the given sites (nearest site, lowest index on ties, Ex. A.2). */
typedef struct {
    int32_t outer_m;
    double outer_theta0;
    int32_t edge_m[WOS_MAX_VERTICES];
    int32_t outer_nb, outer_ns;
    int32_t face_n1, face_n2;
    int32_t hole_m[WOS_MAX_HOLES];
    double hole_theta0[WOS_MAX_HOLES];
    int32_t hole_nb[WOS_MAX_HOLES];
    int32_t hole_ns[WOS_MAX_HOLES];
    int32_t voronoi_n;            /* 0 = use the cells above */
    const double *voronoi_sites;  /* host, voronoi_n x dim */
} wos_partition;

typedef enum { WOS_FP32 = 0, WOS_FP64 = 1 } wos_precision;

/* Options of a build; zero-initialise and set what you need. */
typedef struct {
    int32_t precision;   /* wos_precision of the walk arithmetic */
    uint32_t step_cap;   /* 0 = 1,000,000; walks reaching it stay unterminated */
    uint32_t stream_id;  /* fourth Philox counter word (instance id) */
    uint32_t k0, k1;     /* walk range [k0, k1) of every point; k1 = 0 -> N */
    int32_t accumulate;  /* 0: counts/unterminated are zeroed first; 1: added */
    int32_t block_size;  /* 0 = tuned default; else a multiple of 32, <= 1024 */
    int32_t blocks_per_sm; /* 0 = as many as fit */
    int32_t tile_walks;  /* walks per warp tile (0 = automatic) */
    int32_t hist_slots;  /* shared-memory histogram slots per warp: 0 = auto,
                            1 or 2; -1 = tally straight to global memory */
    int32_t refill_min;  /* refill granularity: finished lanes wait until at
                            least this many lanes of the warp need a walk
                            (0 or 1 = refill at every group of steps) */
    int32_t tiles_per_warp; /* target tiles per warp when tile_walks = 0
                            (0 = 16); walks per lane per tile follow */
    int32_t *trace_elem; /* device, optional: M_D x (k1-k0) exit element of
                            every walk (-1 = unterminated); for tests */
    uint32_t *trace_steps; /* device, optional: same shape, N_eps per walk */
    double *trace_x;     /* device, optional: M_D x (k1-k0) x dim exit points */
    void *kernel_events[2]; /* optional cudaEvent_t pair (caller-created):
                               recorded on `stream` right before and after
                               the walk kernel, to time it alone */
    int32_t mapped;      /* 1: the chain of Sec. 4.2 with larger steps: the
                            ellipsoid X + rho S B(0,1) of each step is the
                            largest inside D, i.e. rho = dist_y(S^{-1} X) in
                            y = S^{-1} x (instead of dist_x).  Boxes and convex
                            counter-clockwise polygons of at most 8 edges
                            without holes: walk-on-spheres in y with the
                            exact distance to the polytope S^{-1} D, stop at
                            dist_y <= eps.  Discs / balls minus disc / ball
                            holes: rho = a lower bound of dist_y that is
                            exact to first order at dD and >= dist_x (one
                            quadratic majorant per boundary component), stop
                            at rho <= eps.  Either way dist_x <= eps at the
                            stop and exits are classified in x; other
                            domains: WOS_INVALID_ARG */
    int32_t group_blocks; /* Philox blocks per group of steps (0 = about 16
                            steps, at most 16 blocks): a group is
                            group_blocks x (4 / words per step) steps, the
                            lanes whose walk ended are refilled once per
                            group; results do not depend on it (the counter
                            of step n is n / steps per block) */
} wos_opts;

/* Per-build statistics (filled after the build's device work finished). */
typedef struct {
    uint64_t walks;        /* walks run */
    uint64_t steps;        /* sum over walks of N_eps (moves of the chain) */
    uint64_t unterminated; /* walks stopped by the step cap */
    uint32_t max_steps;    /* largest N_eps seen */
    int32_t grid, block, tile_walks, hist_slots; /* launch configuration */
    float kernel_ms;       /* device time of the walk kernel */
} wos_stats;

typedef struct wos_context wos_context;

/* Create a context on CUDA device `device` (sets it current for the calling
 * thread).  The context owns small device scratch buffers (work counters,
 * statistics, descriptor tables) and frees them in wos_destroy.
 * Errors: WOS_INVALID_ARG (no such device), WOS_OOM, WOS_CUDA_ERROR. */
wos_status wos_create(int32_t device, wos_context **ctx);
wos_status wos_destroy(wos_context *ctx);

/* Number of kernels this context has launched so far (all entry points). */
uint64_t wos_kernel_launches(const wos_context *ctx);

/* Human-readable name of a status code (static string). */
const char *wos_status_string(wos_status s);

/* Instance set-up of the chain (paper Sec. 4.2, "lambda_max(K) = 1 without
 * loss of generality"): S = (K / lambda_max(K))^{1/2}, the symmetric square
 * root.  K, S: host, dim x dim row-major.  Host only (no device work).
 * Errors: WOS_INVALID_ARG (dim not 2 or 3), WOS_K_NOT_SPD. */
wos_status wos_conductivity_sqrt(int32_t dim, const double *K, double *S);

/* Number of boundary elements M_tot of a partition, or -1 if invalid. */
int32_t wos_num_elements(const wos_domain *domain, const wos_partition *part);

/* sigma(omega_j) of every element (arc length, edge-cell length or patch
 * area: the surface measure of the cell, paper Sec. 3.1, Eq.
 * (boundary_weights)).  out: host, M_tot doubles.  Host only.
 * Extrinsic Voronoi partitions (App. A, Ex. A.2) are supported when every
 * site lies on a circle / sphere of D (the outer sphere or a hole, within
 * 1e-9 of its radius), each such surface shared among its own sites: 2-D
 * cells are arcs between the bisectors of angular neighbours, 3-D cells
 * spherical Voronoi polygons (built by half-plane clipping in the central
 * projection at the site; areas from spherical triangles); identical sites
 * give the lowest index the cell and the others 0.  Errors: WOS_INVALID_ARG
 * (bad descriptors; Voronoi sites on a box or polygon, off every circle /
 * sphere, or a cell reaching 89.9 degrees from its site). */
wos_status wos_element_measures(const wos_domain *domain,
                                const wos_partition *part, double *out);

/* The FP32 safety floor of eps: 128 * 2^-24 * max |coordinate| over the
 * domain's bounding box.  Above it FP32 rounding of the distance and of a
 * move stays far inside the eps-shell, so no walk can cross dD unstopped. */
double wos_fp32_eps_floor(const wos_domain *domain);

/* MC-REM (paper Sec. 5.1, Algorithm MC-REM; Sec. 4.2, Eq. (wos chain) and
 * Eq. (N epsilon x); Sec. 4.3, Eq. (WoE_matrix_MC)).
 *
 * For every observation point x_i (i < M_D) and walk k in [k0, k1), runs the
 * walk-on-ellipsoids chain X_{n+1} = X_n + dist(X_n, dD) S U_n from X_0 = x_i,
 * S = (K / lambda_max(K))^{1/2}, U_n uniform on the unit sphere drawn from
 * Philox4x32-10 (key = seed, counter = (block, walk lo, walk hi, stream_id),
 * walk = i * N + k; step n reads block n / G: G = 5 for FP32 2-D walks, whose
 * step takes the 23-bit window (n mod 5) of the block's 128 bits; G = 2 for
 * FP32 3-D walks (23-bit uniforms (w >> 9) 2^-23 from two words) and FP64
 * 2-D walks; G = 1 for FP64 3-D walks (53-bit uniforms from two words)),
 * stops at the first n with dist(X_n, dD) <= eps and adds
 * 1 to counts[i][j], j the element holding pi(X_n).  Walks reaching
 * opts->step_cap add 1 to unterminated[i] instead, so that
 * sum_j counts[i][j] + unterminated[i] = k1 - k0 exactly (per call).
 * A = counts / N estimates [mu_{x_i}(omega_j)].
 *
 *   K        host, dim x dim row-major, symmetric positive definite.
 *   points   device, M_D x dim doubles, strictly inside D.
 *   counts   device, M_D x M_tot uint32 (zeroed first unless accumulate).
 *   unterminated device, M_D uint32, or NULL (then capped walks are only
 *            counted in stats).
 *   stats    host or NULL.  If non-NULL the call waits for the device work
 *            and fills it; if NULL the call is asynchronous.
 * Errors: WOS_INVALID_ARG, WOS_K_NOT_SPD, WOS_EPS_BELOW_FP32_FLOOR (FP32
 * walks only), WOS_COUNT_OVERFLOW, WOS_CUDA_ERROR; WOS_STEP_CAP_HIT is
 * returned as a warning when stats is non-NULL and a walk was capped.
 * WOS_POINT_OUTSIDE: the points are tested on the device before the walks
 * (FP64, the test of wos_check_points: dist(x_i, dD) > 0, and inside a
 * polygon by the crossing number); if one lies outside D or on dD no walk
 * runs, so counts and unterminated keep their values after the zeroing (all
 * zero unless accumulate).  The status itself needs the device result: it
 * is returned when stats is non-NULL (the call waits); an asynchronous call
 * (stats NULL) returns WOS_OK and leaves the zero row sums as the sign --
 * use wos_check_points on host copies of the points to test them up front. */
wos_status wos_build_operator(wos_context *ctx, const wos_domain *domain,
                              const double *K, const double *points,
                              int32_t M_D, const wos_partition *partition,
                              uint32_t N, double eps, uint64_t seed,
                              const wos_opts *opts, uint32_t *counts,
                              uint32_t *unterminated, wos_stats *stats,
                              void *stream);

/* The operator build of wos_build_operator for callers that cannot allocate
 * device memory.  The paper has no counterpart: this is an interface for
 * callers that run under a device-memory budget reserved up front (work is
 * admitted by its footprint) or inside a host framework that owns every
 * device allocation, so that neither cudaMalloc nor cudaMallocAsync may be
 * called on their behalf.
 *
 * Arguments, results and errors are those of wos_build_operator, plus
 * WOS_NOALLOC_LIMIT.  The call allocates nothing: its scratch (the work-queue
 * and statistics counters, and the site table of an extrinsic Voronoi
 * partition) lives in one 64 KiB array of device memory defined by the
 * library, which every GPU that loads the library holds until the process
 * exits.  Limits: at most 2048 Voronoi sites (more returns WOS_NOALLOC_LIMIT);
 * everything else as in wos_build_operator.  stats->kernel_ms is left 0 (use
 * opts->kernel_events to time the kernel).
 *
 * The first call on each device looks up that array's device address (with
 * the context's device current); make that first call before any stream
 * capture.  All calls on a device share the array and it keeps the last
 * call's contents: each call clears the counters it needs at zero, but calls
 * whose device work may overlap (other streams, no event ordering) race on
 * it and must be serialised by the caller.  The looked-up address, like a
 * context, does not survive cudaDeviceReset.
 *
 * Differences from wos_build_operator: an extrinsic Voronoi partition is
 * classified by a scan of all its sites per exit (no candidate grid, which
 * would need scratch), so such builds are slower; its site table is copied
 * from a host stack buffer with a pageable cudaMemcpyAsync, and a call with
 * stats waits for the stream -- neither may run under stream capture. */
wos_status wos_build_operator_noalloc(wos_context *ctx, const wos_domain *domain,
                                      const double *K, const double *points,
                                      int32_t M_D, const wos_partition *partition,
                                      uint32_t N, double eps, uint64_t seed,
                                      const wos_opts *opts, uint32_t *counts,
                                      uint32_t *unterminated, wos_stats *stats,
                                      void *stream);

/* One operator build of a batch (see wos_build_operators_batched).  Host
 * descriptors are read during the call; device arrays as in
 * wos_build_operator. */
typedef struct {
    const wos_domain *domain;
    const wos_partition *partition;
    const double *K;          /* host, dim x dim */
    const double *points;     /* device, M_D x dim */
    int32_t M_D;
    uint32_t N;               /* walks per point */
    double eps;
    uint32_t stream_id;       /* fourth Philox counter word of this problem */
    uint32_t step_cap;        /* 0 = 1,000,000 */
    uint32_t *counts;         /* device, M_D x M_tot */
    uint32_t *unterminated;   /* device, M_D, or NULL */
    uint32_t k0, k1;          /* walk range [k0, k1) of every point; k1 = 0 -> N */
} wos_problem;

/* Many MC-REM builds (paper Sec. 5.1, Algorithm MC-REM, applied to each
 * problem) in one persistent launch per class (dimension x kernel kind:
 * plain disc/ball, box, box with equal half-extents, disc/ball with holes,
 * disc/ball with one concentric hole, mapped walks, other): the walks of all the
 * problems of a class share a global tile queue, so problems of very
 * different sizes and walk lengths keep the whole GPU busy.  All problems
 * share `seed` and opts->precision; each problem's walks use counter
 * (block, walk lo, walk hi, stream_id), so its counts are bit-identical to
 * the same problem built alone with wos_build_operator (same stream_id).
 * opts may set precision, accumulate and the launch fields (block_size,
 * blocks_per_sm, tile_walks, hist_slots, kernel_events); opts->k0 / k1 and
 * traces must be zero (each problem has its own walk range).  stats (host or NULL): totals over the batch; non-NULL waits.
 * Errors: those of wos_build_operator, for the first failing problem, except
 * that the points are not tested here (wos_check_points tests them). */
wos_status wos_build_operators_batched(wos_context *ctx, int32_t n,
                                       const wos_problem *problems, uint64_t seed,
                                       const wos_opts *opts, wos_stats *stats,
                                       void *stream);

/* A launch configuration chosen by wos_autotune. */
typedef struct {
    int32_t block_size, blocks_per_sm, tiles_per_warp, hist_slots, refill_min;
    int32_t group_blocks;
    int32_t trials;        /* configurations timed */
    float best_ms;         /* walk-kernel time of the sample, best config */
    float default_ms;      /* the same with the built-in defaults */
} wos_tuning;

/* Autotuner (no paper counterpart: it only picks launch parameters, which
 * never change results since every walk's random numbers are fixed by its
 * Philox counter).  Times the walk kernel of `sample` (its first points, at
 * most sample_walks walks in all) with CUDA events under a coordinate search
 * over block size {256, 128}, resident blocks per SM {max, 3, 2}, tiles per
 * warp {16, 4, 64}, histogram slots {auto, none} and refill granularity
 * {1, 4, 8}; keeps the fastest in the context for problems of the same
 * precision, dimension and kernel kind (plain disc/ball, box, box with equal
 * half-extents, disc/ball with holes, disc/ball with one concentric hole,
 * mapped walks, other).  Later wos_build_operator / wos_build_operators_batched calls
 * whose opts leave all launch fields 0 use it.  Synchronises `stream`.
 * Errors: those of wos_build_operator. */
wos_status wos_autotune(wos_context *ctx, const wos_problem *sample, uint64_t seed,
                        int32_t precision, uint64_t sample_walks, wos_tuning *out,
                        void *stream);

/* Forget every tuned configuration of the context. */
wos_status wos_autotune_reset(wos_context *ctx);

/* ---------------------------------------------------------------------------
 * Serving: a request queue with continuous batching (spec serving
 * pattern; no paper counterpart).  A request is one Cauchy problem end to
 * end: MC-REM operator build, FP64 SVD and TSVD reconstruction (paper
 * Algorithm Main).  A worker thread admits queued requests in arrival order
 * while the device-memory budget and the slot count allow, keeps their counts
 * resident on the device, and advances every admitted request by a slice of
 * walks per point in one batched launch per slice, so requests arriving while
 * others run join at the next slice.  A request whose walks are done gets its
 * SVD and reconstruction on a side stream, overlapping other requests' walks.
 * Results are bit-identical to running the same request alone (the walks of a
 * request are fixed by the queue seed and the request's stream_id).
 * ------------------------------------------------------------------------- */
typedef struct wos_queue wos_queue;

typedef struct {
    int32_t max_inflight;   /* requests admitted at once (0 = 64) */
    uint64_t device_budget; /* device bytes for admitted requests (0 = 8 GiB) */
    uint32_t slice_walks;   /* walks per point per slice (0 = 4096) */
    int32_t precision;      /* walk precision of every request (wos_precision) */
    uint64_t seed;          /* Philox key of the queue */
    int32_t side_streams;   /* concurrent SVD / reconstruction pipelines (0 = 8) */
} wos_queue_opts;

/* One request.  Every pointer is host memory: inputs are copied at submit
 * time; outputs must stay valid until the request completes. */
typedef struct {
    const wos_domain *domain;
    const wos_partition *partition;
    const uint8_t *gamma1;  /* M_tot labels (1 = Gamma_1) */
    const double *K;        /* dim x dim */
    const double *points;   /* M_D x dim */
    int32_t M_D;
    uint32_t N;
    double eps;
    uint32_t stream_id;     /* Philox counter word: distinct per request */
    const double *nu;       /* M_D, or NULL (1/sqrt(M_D)) */
    const double *uD;       /* M_D measurements */
    const double *u0;       /* M_0 Gamma_0 data, or NULL (zero) */
    int32_t r;              /* truncation; 0 = first gap S_r/S_{r+1} >= 1.5
                               after S_r/S_1 < 1e-3 (else the last gap) */
    double tikhonov_alpha;  /* 0 = plain truncation */
    double *u_gamma1;       /* out: M_1 reconstructed Gamma_1 data */
    double *S;              /* out: k singular values, or NULL */
    uint32_t *counts;       /* out: M_D x M_tot counts, or NULL */
    int32_t *r_used;        /* out: the truncation used, or NULL */
} wos_request;

typedef struct {
    uint64_t submitted, admitted, completed, failed;
    uint64_t slices;        /* batched walk launches */
    uint64_t walks;         /* walks run */
    int32_t inflight;       /* admitted, not completed */
    int32_t queued;         /* waiting for admission */
} wos_queue_stats;

/* Create / destroy a queue on the context's device.  destroy waits for every
 * submitted request to finish.  Errors: WOS_INVALID_ARG, WOS_CUDA_ERROR. */
wos_status wos_queue_create(wos_context *ctx, const wos_queue_opts *opts,
                            wos_queue **q);
wos_status wos_queue_destroy(wos_queue *q);

/* Submit a request; *ticket identifies it.  Validates it first (errors of
 * wos_build_operator; WOS_INVALID_ARG if it can never fit the budget). */
wos_status wos_submit(wos_queue *q, const wos_request *req, uint64_t *ticket);

/* WOS_OK when the request completed (outputs written), WOS_NOT_READY while
 * it runs, else the error it failed with. */
wos_status wos_poll(wos_queue *q, uint64_t ticket);

/* Wait up to timeout_ms (< 0: forever) for a request; returns as wos_poll. */
wos_status wos_wait(wos_queue *q, uint64_t ticket, int32_t timeout_ms);

wos_status wos_queue_get_stats(wos_queue *q, wos_queue_stats *stats);

/* Check that every point (host, M_D x dim) lies strictly inside D.  Returns
 * WOS_OK or WOS_POINT_OUTSIDE (first offending index in *bad if non-NULL). */
wos_status wos_check_points(const wos_domain *domain, const double *points,
                            int32_t M_D, int32_t *bad);

/* One-sided Jacobi SVD of the scaled operator (paper Sec. 4.3, Eq. (A_r_MC);
 * Sec. 2, Eq. (SVD)):
 *     B = diag(nu) (counts[:, Gamma_1] / N) diag(sigma_{Gamma_1})^{-1/2}
 *       = U diag(S) V^T,
 * M_1 = number of Gamma_1 elements, k = min(M_D, M_1), S descending, each
 * right vector signed so that its largest-magnitude entry is positive.
 * eig(Lambda^nu) = S^2 (Prop. coro:B-Lambda).  FP64 throughout.
 *   counts   device, M_D x M_tot uint32.
 *   gamma1   host, M_tot bytes: 1 = element on Gamma_1, 0 = on Gamma_0.
 *   nu       device, M_D doubles, or NULL for nu_i = 1/sqrt(M_D) (Sec. 5.2).
 *   sigma    device, M_tot doubles (wos_element_measures).
 *   U        device, M_D x k;  S  device, k;  V  device, M_1 x k.
 *   sweeps   host or NULL; if non-NULL the call waits and stores the FP64
 *            sweep count (when FP32 sweeps ran first -- 257 to 768 columns,
 *            see wos_set_svd_path -- only the FP64 sweeps after them), and
 *            returns WOS_NO_CONVERGENCE if max sweeps were used, or
 *            WOS_DEVICE_TIMEOUT if a grid-wide wait of the QR or of the
 *            sweeps gave up.
 * Errors: WOS_INVALID_ARG, WOS_OOM, WOS_CUDA_ERROR, WOS_NO_CONVERGENCE,
 * WOS_DEVICE_TIMEOUT. */
wos_status wos_op_svd(wos_context *ctx, const uint32_t *counts, int32_t M_D,
                      int32_t M_tot, uint32_t N, const uint8_t *gamma1,
                      const double *nu, const double *sigma, double *U,
                      double *S, double *V, int32_t *sweeps, void *stream);

/* Many SVDs of wos_op_svd in one pass (one cooperative QR launch, one FP32
 * sweep launch, one launch per GEMM step and one Jacobi launch per class of
 * problem size, their CTAs split among the problems, each synchronising
 * only its own CTAs): independent operators of
 * a benchmark step or of the serving queue share the GPU instead of queueing
 * one latency-bound launch after another.  Every field as the argument of
 * the same name of wos_op_svd (counts, nu, sigma, U, S, V on the device;
 * gamma1 on the host).  Results equal wos_op_svd's for each problem, bit for
 * bit.  sweeps: host, n entries, or NULL (as wos_op_svd). */
typedef struct {
    const uint32_t *counts;
    int32_t M_D, M_tot;
    uint32_t N;
    const uint8_t *gamma1;
    const double *nu, *sigma;
    double *U, *S, *V;
} wos_svd_problem;

wos_status wos_op_svd_batched(wos_context *ctx, int32_t n,
                              const wos_svd_problem *problems, int32_t *sweeps,
                              void *stream, void *const *jacobi_events);
/* jacobi_events: NULL, or two cudaEvent_t recorded on the stream before the
 * first and after the last factorisation launch (the QR, the FP32 sweeps
 * and their Newton-Schulz products when they run, and the FP64 Jacobi
 * sweeps; for profiling). */

/* Which kernels factor an SVD problem (a setting of the context, read by
 * wos_op_svd, wos_op_svd_batched and the serving queue):
 *   WOS_SVD_AUTO     the cluster kernel when the worked matrix fits it (at
 *                    most 256 columns and the shared memory of the cluster),
 *                    else the grid-wide kernels (default);
 *   WOS_SVD_GRID     always the grid-wide kernels (cooperative QR and Jacobi
 *                    launches synchronised through global memory);
 *   WOS_SVD_CLUSTER  as AUTO (a problem that does not fit still runs on the
 *                    grid-wide kernels);
 *   WOS_SVD_FP64_SWEEPS  as AUTO, but a problem of more than 256 columns
 *                    runs every Jacobi sweep in FP64.  By default (up to 896
 *                    columns) its sweeps first run on an FP32 copy of
 *                    X = R^T in one thread-block cluster, and the FP64 sweeps
 *                    start from X Q, Q the product of those rotations made
 *                    orthogonal to FP64 rounding by Newton-Schulz steps: the
 *                    same singular values and vectors to FP64 rounding, in a
 *                    few FP64 sweeps instead of about ten.
 * The cluster kernel factors one problem in one thread-block cluster of up
 * to 16 CTAs: the matrix stays in distributed shared memory and the Jacobi
 * rounds are ordered by cluster barriers.  Both compute the same
 * factorisation (QR with column pivoting, then one-sided Jacobi on R^T in
 * the same round-robin order) with different summation orders, so their
 * results agree to rounding, not bit for bit; each is deterministic.
 * Errors: WOS_INVALID_ARG (unknown path or NULL ctx). */
enum { WOS_SVD_AUTO = 0, WOS_SVD_GRID = 1, WOS_SVD_CLUSTER = 2, WOS_SVD_FP64_SWEEPS = 3 };
wos_status wos_set_svd_path(wos_context *ctx, int32_t path);

/* Measured throughput of the execution pipes the kernels lean on, from
 * microbenchmark kernels on the context's device (a few milliseconds; SMs x
 * 8 CTAs of 256 threads, eight independent chains of one PTX operation per
 * thread, CUDA events around a launch after a warm-up launch):
 *   out[WOS_PIPE_FFMA]       fma.rn.f32 per second (lanes)
 *   out[WOS_PIPE_MUFU]       sin.approx.f32 and cos.approx.f32 per second
 *   out[WOS_PIPE_IMAD_WIDE]  mul.wide.u32 (each followed by the xor of its
 *                            halves: a Philox half-round) per second
 *   out[WOS_PIPE_LOP3]       lop3.b32 per second
 *   out[WOS_PIPE_DFMA]       fma.rn.f64 per second
 *   out[WOS_PIPE_ISSUE]      instructions per second of an fma.rn.f32 /
 *                            lop3.b32 alternation (two pipes: the issue limit)
 * out: host, WOS_PIPE_COUNT doubles; stream as elsewhere (the call waits).
 * Errors: WOS_INVALID_ARG, WOS_OOM, WOS_CUDA_ERROR. */
enum {
    WOS_PIPE_FFMA = 0, WOS_PIPE_MUFU = 1, WOS_PIPE_IMAD_WIDE = 2, WOS_PIPE_LOP3 = 3,
    WOS_PIPE_DFMA = 4, WOS_PIPE_ISSUE = 5, WOS_PIPE_COUNT = 6
};
wos_status wos_measure_pipes(wos_context *ctx, double *out, void *stream);

/* r-TSVD reconstruction (paper Sec. 2, Eq. (u1r); Sec. 4.3, Eq.
 * (u_omega_M1_r_MC A); Sec. 5.1, Rem. (b and u0 simulations), Eq. (tsvd
 * solution simulations)):
 *     b      = uD - A_{Gamma_0} u0                (A = counts / N)
 *     u_g1   = diag(sigma_{Gamma_1})^{-1/2} V_r F_r U_r^T diag(nu) b
 * with F_r = diag(1 / S_i) (i < r), or the Tikhonov filter
 * S_i / (S_i^2 + alpha) when tikhonov_alpha > 0; and the fitted interior
 * data uD_hat = A_{Gamma_1} u_g1 + A_{Gamma_0} u0 (Sec. 5.2, item (iv)).
 *   U, S, V  device, from wos_op_svd (k columns).
 *   uD       device, M_D;  u0 device, M_0 (= M_tot - M_1) or NULL (= 0).
 *   u_gamma1 device, M_1;  uD_hat device, M_D, or NULL.
 * The truncation r is the caller's; wos_truncation_gap tells whether it
 * sits at a gap of the spectrum.
 * Errors: WOS_INVALID_ARG (r outside 1..k), WOS_OOM, WOS_CUDA_ERROR. */
wos_status wos_reconstruct(wos_context *ctx, const double *U, const double *S,
                           const double *V, int32_t M_D, int32_t k,
                           const uint32_t *counts, int32_t M_tot, uint32_t N,
                           const uint8_t *gamma1, const double *nu,
                           const double *sigma, const double *uD,
                           const double *u0, int32_t r, double tikhonov_alpha,
                           double *u_gamma1, double *uD_hat, void *stream);

/* Spectral diagnostics of one operator from its SVD (paper Sec. 5.2 items
 * (i)-(iv); Eq. (Lambda_tilde_nu), (rho omega1 MC), (eigenfunctions_MC),
 * (tsvd solution simulations)), FP64:
 *   lambda[j]            = S_j^2, the eigenvalues of Lambda^nu (Prop.
 *                          coro:B-Lambda), j < k;
 *   eigfun[l * k + j]    = the eigenfunction estimator u~_j on Gamma_1
 *                          element l: S_j^{-1} sum_i nu_i U_ij A_il / sigma_l;
 *   density[l]           = (1 / M_D) sum_i A_il / sigma_l, the averaged
 *                          estimator of the elliptic densities on Gamma_1;
 *   u_sweep[(r-1) * M_1 + l]  = the r-TSVD solution on element l, r = 1..r_max
 *                          (equal to wos_reconstruct at truncation r, bit for bit);
 *   uD_sweep[(r-1) * M_D + i] = A_Gamma_1 u^(r) + A_Gamma_0 u0 at point i
 *                          (the fitted interior data of item (iv)).
 * Inputs as wos_reconstruct (U, S, V from wos_op_svd; counts, gamma1, nu,
 * sigma, uD, u0).  Every output is a device buffer or NULL (not computed);
 * u_sweep is required when uD_sweep is given; r_max in 0..k.
 * Errors: WOS_INVALID_ARG, WOS_OOM, WOS_CUDA_ERROR. */
wos_status wos_spectral(wos_context *ctx, const double *U, const double *S,
                        const double *V, int32_t M_D, int32_t k,
                        const uint32_t *counts, int32_t M_tot, uint32_t N,
                        const uint8_t *gamma1, const double *nu,
                        const double *sigma, const double *uD, const double *u0,
                        int32_t r_max, double *lambda, double *eigfun,
                        double *density, double *u_sweep, double *uD_sweep,
                        void *stream);

/* Truncation rule for degenerate spectra: returns WOS_OK when
 * S[r-1] / S[r] >= 1.5 (or r = k), else WOS_TRUNCATION_IN_CLUSTER.
 * S: host, k doubles. */
wos_status wos_truncation_gap(const double *S, int32_t k, int32_t r);

#ifdef __cplusplus
}
#endif

#endif /* WOS_H */
