/*
 * hbsqp: fast direct solver for quasi-periodic Dirichlet scattering from a
 * grating of obstacles (Gillman & Barnett, "A fast direct solver for
 * quasi-periodic scattering problems"), GB300 (sm_103a) CUDA library.
 *
 * C ABI.  All complex numbers are complex128 stored as interleaved (re, im)
 * pairs of doubles.  Matrices are column-major.  Device pointers are plain
 * CUDA global-memory addresses; `stream` is a cudaStream_t passed as void*
 * (NULL = legacy default stream).  Every call returns an hbs_status;
 * hbs_last_error() gives a human-readable message for the last failure on
 * the calling thread.  Nothing here falls back to the CPU: a call that
 * cannot run its kernels fails with HBS_ERR_CUDA.
 */
#ifndef HBSQP_H
#define HBSQP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hbs_status {
  HBS_OK = 0,
  HBS_ERR_INVALID_ARG = 1, /* bad size, pointer, angle or geometry */
  HBS_ERR_OOM = 2,         /* device allocation failed */
  HBS_ERR_CUDA = 3,        /* a CUDA call or kernel launch failed */
  HBS_ERR_RANK = 4,        /* a skeleton rank exceeded the supported maximum */
  HBS_WARN_ILLCOND = 5,    /* a Schur system was numerically singular (guided mode, Remark 2.1) */
  HBS_ERR_TIMEOUT = 6,     /* a bounded device wait gave up */
  HBS_ERR_IO = 7,          /* file could not be read or written */
  HBS_ERR_INTERNAL = 8
} hbs_status;

typedef struct hbs_handle hbs_handle; /* compressed inverse of A + periodizer precompute */
typedef struct hbs_result hbs_result; /* Bragg amplitudes of a batch of incident angles */

/*
 * Obstacle boundary sampled by the N-point periodic trapezoid rule (Sec. 2.3):
 * nodes z(t_j) = (x_j, y_j) and derivatives z'(t_j) = (dx_j, dy_j) at
 * t_j = 2 pi j / N, counter-clockwise, with the obstacle inside the unit
 * cell |x| < d/2 (Sec. 2.1).  The arrays are copied at build time; the
 * caller keeps ownership.
 */
typedef struct hbs_geometry {
  int64_t n;
  double d;
  const double* x;
  const double* y;
  const double* dx;
  const double* dy;
  int on_device; /* 0: host pointers, 1: device pointers */
} hbs_geometry;

#define HBS_PRECISION_FP64 0
/* Dense products (the telescoping applies, the level products E, F*, G and the
 * periodizer projections) in double-float arithmetic: each FP64 operand is split into
 * two floats and multiplied and accumulated error-free on the FP32 pipes (about 48
 * significant bits, relative error near 1e-14 per product).  Kernel evaluations, the
 * interpolative decompositions, the inversions and the Schur solves stay in FP64. */
#define HBS_PRECISION_DOUBLE_FLOAT 1
/* As HBS_PRECISION_DOUBLE_FLOAT, and the large dense products (inner dimension >= 4096,
 * at least 64 rows) run on the tcgen05 tensor cores: every FP64 row of op(A) and column
 * of B is scaled by a power of two and cut into seven 7-bit integer digits held exactly
 * in bf16; the digit products are accumulated exactly in FP32 tensor memory over 64
 * values of k and recombined in double-float arithmetic (relative error about 2^-46 of
 * max|a_ik| max|b_kj| per product term). */
#define HBS_PRECISION_TENSOR 2

typedef struct hbs_options {
  int leaf_size;        /* maximum points per leaf of the binary tree (default 64) */
  int n_proxy_min;      /* minimum proxy points on each node's proxy circle (default 64) */
  double proxy_rho;     /* node proxy circle radius / node radius (default 1.5) */
  double nb_radius;     /* neighbour proxy circle radius, Sec. 3.2 (0: automatic) */
  int nb_proxies;       /* neighbour proxy points (0: automatic) */
  int m;                /* Sommerfeld nodes per wall density type (0: automatic) */
  double contour_h;     /* trapezoid spacing in Re k (0: automatic, 0.2) */
  double contour_c;     /* contour height c in k = t - i c tanh((t - t0)/w) (0: 2) */
  double contour_w;     /* contour width w (0: 2) */
  double contour_k;     /* truncation |Re k - t0| <= K (0: automatic) */
  double wood_shift;    /* crossing point t0 of the second contour (0: automatic, < 0: none) */
  int n_bragg_samples;  /* samples per line for the Bragg DFT (0: automatic) */
  double y0;            /* Bragg sampling height (0: max |y| + d/4) */
  int precision;        /* HBS_PRECISION_FP64 (default), _DOUBLE_FLOAT or _TENSOR */
  double index;         /* refractive index n of the obstacles, Sec. 5 (0, the default:
                           sound-soft obstacles, Sec. 2).  n > 0 selects the transmission
                           problem: two unknowns per boundary node, interlaced
                           [s_1; tau_1; s_2; ...] (s = sigma / omega the single-layer and tau
                           the double-layer density), rows in the same order (sigma row:
                           minus the normal derivative of the field over omega, tau row: its
                           value).  Its kernel functions are evaluated in FP64 in every
                           precision mode. */
} hbs_options;

typedef struct hbs_info_t {
  int64_t n;             /* boundary nodes */
  int levels;            /* tree levels below the root */
  int max_rank;          /* largest skeleton size over all nodes */
  int nb_rank;           /* neighbour interaction rank l (Sec. 3.2) */
  int m;                 /* Sommerfeld nodes per density type */
  int n_contours;        /* 1, or 2 when a Wood's-anomaly contour is precomputed */
  size_t device_bytes;   /* device memory held by the handle */
  double build_seconds;  /* wall time of hbs_build */
  double factor_bytes;   /* bytes of the compressed inverse (E, F*, G over all nodes) */
  double apply_flops_per_rhs; /* real flops of one A^{-1} apply per right-hand side */
  double contour_h, contour_c, contour_w; /* Sommerfeld contour actually used */
  double wood_t0;        /* crossing point of the second contour (0 if none) */
  int n_bragg_samples;   /* S */
  double y0;             /* Bragg sampling height */
  double nb_radius;      /* neighbour proxy circle radius */
  int nb_proxies;        /* neighbour proxy points */
  int pid_col_rank;      /* skeleton columns kept of the wall blocks B_L, B_R (all contours) */
  int pid_row_rank;      /* skeleton rows kept of C_L, C_R and of the Bragg sampling rows */
  double pid_residual;   /* relative error of those decompositions on an independent point sample */
  double nb_residual;    /* relative error of the neighbour ID (Sec. 3.2) on nodes between its candidates */
  int64_t unknowns;      /* n (sound-soft) or 2 n (transmission): the size of A */
  double index;          /* refractive index (0: sound-soft) */
} hbs_info_t;

/* Fill `opts` with the defaults listed above. */
void hbs_default_options(hbs_options* opts);

/*
 * Pre-computation (Sec. 6, first step): HBS compression and inversion of the
 * isolated-obstacle matrix A = I/2 + D - i w S (Sec. 4), the neighbour-image
 * factors A_{+-1} = L R (Sec. 3.2) and the angle-independent products with
 * the periodizing blocks (Secs. 2.2-2.4).  `tol` is the relative ID
 * tolerance.  On success *out owns device memory until hbs_free.
 * Errors: INVALID_ARG (n < 64, d <= 0, omega <= 0, tol outside (0, 1),
 * obstacle touching a wall), OOM, CUDA, RANK.
 */
hbs_status hbs_build(const hbs_geometry* geom, double omega, double tol, const hbs_options* opts,
                     void* stream, hbs_handle** out);

/*
 * The pre-computation of hbs_build for `count` independent solvers at once (gratings of
 * different obstacles, sizes and frequencies; geoms[i] with omegas[i], one tol and one
 * options struct for all).  The HBS compression and inversion run level-synchronously
 * from the leaves: at every stage each kernel covers the current level of every solver
 * in one launch.  Each out[i] is the same solver hbs_build would return for geoms[i]
 * (up to the rounding of a different batch split) and is freed with hbs_free; its
 * build_seconds is the time of the whole batch.  `out` has `count` entries.
 * Errors: as hbs_build, for the first failing solver; on any error every out[i] is NULL.
 */
hbs_status hbs_build_batch(const hbs_geometry* geoms, const double* omegas, int64_t count, double tol,
                           const hbs_options* opts, void* stream, hbs_handle** out);

/*
 * Block solve (Sec. 3 and Sec. 6, second step) for incident angles
 * theta[0..n_theta) in (-pi, 0) (host array).  Angles are grouped by Bloch
 * phase alpha = exp(i w d cos theta) (Remark 3.1) and each group is solved
 * with one multi-right-hand-side apply of the compressed inverse.  Returns
 * a result holding Bragg amplitudes for every angle.  Errors: INVALID_ARG,
 * OOM, CUDA; WARN_ILLCOND when a Schur system was singular to working
 * precision (the result is still produced).
 */
hbs_status hbs_solve(hbs_handle* h, const double* theta, int64_t n_theta, void* stream,
                     hbs_result** out);

/*
 * Same result as hbs_solve, computed the way the paper counts it: for each
 * Bloch phase the compressed inverse is applied to q + 2M + 2Pl vectors
 * (Remark 3.2) instead of using the angle-independent precompute.  This is
 * the plain FP64 per-angle path used as a reference.
 */
hbs_status hbs_solve_plain(hbs_handle* h, const double* theta, int64_t n_theta, void* stream,
                           hbs_result** out);

/*
 * The same Bragg amplitudes with a second periodizer: proxy points and wall discrepancies
 * instead of the Sommerfeld-contour wall potentials of Secs. 2.2-2.4 (the paper's Sec. 7
 * points to this family of schemes without defining one).  The handle's compressed
 * inverse and neighbour factors (Secs. 3.2, 4) are reused; the unit cell is cut to the box
 * |x| <= d/2, |y| <= h (h = max|y| + d/8), the images beyond the neighbours are represented by
 * combined-field sources on a circle around it, and the radiation condition by outgoing
 * Rayleigh-Bloch expansions matched on y = +-h.  Each Bloch phase's rectangular system is
 * solved in the least-squares sense; every step is FP64.  The amplitudes are referred to
 * y = +-y0 as hbs_solve's are (n_wood = 0, t0 = 0 in hbs_result_angle_info).  Meant to
 * cross-check hbs_solve, not tuned for speed.  Transmission solvers (options.index > 0) use
 * the same scheme with the pair of densities (Sec. 5): their obstacle rows are the interlaced
 * transmission rows.  theta must lie in (-pi, 0), else HBS_ERR_INVALID_ARG; OOM and CUDA as
 * hbs_solve.  Synchronizes the stream.
 */
hbs_status hbs_solve_proxy(hbs_handle* h, const double* theta, int64_t n_theta, void* stream,
                           hbs_result** out);

/*
 * Bragg amplitudes of angle i of a result (Remarks 2.2, 2.3): propagating
 * orders n_min..n_max (|kappa_n| <= w), upward c_n and downward d_n as in
 * Eqs. (rbu), (rbd), and the flux error |sum_n (k_n/k_0)(|c_n|^2 +
 * |d_n + delta_n0 e^{i k_0 y0}|^2) - 1|.  c and d are caller-allocated host
 * arrays of 2 (n_max - n_min + 1) doubles, or NULL to query the orders only.
 */
hbs_status hbs_bragg_amplitudes(const hbs_result* r, int64_t i, int* n_min, int* n_max, double* c,
                                double* d, double* flux_err);

/* Extra per-angle facts of a result: Wood's-anomaly modes added (count) and the
 * contour crossing point used. */
hbs_status hbs_result_angle_info(const hbs_result* r, int64_t i, int* n_wood, double* t0);

/* Sizes and timings of a built handle. */
hbs_status hbs_info(const hbs_handle* h, hbs_info_t* info);

/*
 * Persistence of a built handle.  The pre-computation (Sec. 6, first step) depends
 * only on the geometry, w and the options, and the block solves (second step) reuse
 * it for any number of angles, so a process may write it once and later processes
 * read it instead of rebuilding.
 *
 * hbs_save writes every factor, skeleton, interpolation matrix and precomputed product
 * of `h` to `path` (native byte order, a private binary format with a version tag) and
 * returns when the file is complete.  It copies device data to the host through
 * `stream`.  Errors: HBS_ERR_INVALID_ARG (NULL argument), HBS_ERR_IO (cannot open or
 * write the file), HBS_ERR_CUDA.
 *
 * hbs_load reads such a file into a new handle on the current device (allocations and
 * copies on `stream`); the handle is owned by the caller (hbs_free) and solves exactly
 * like the one that was saved.  The file's tag is checked before any device memory is
 * touched.  Errors: HBS_ERR_INVALID_ARG, HBS_ERR_IO (missing, foreign, truncated or
 * corrupt file), HBS_ERR_OOM, HBS_ERR_CUDA.  On error *out is NULL.
 */
hbs_status hbs_save(const hbs_handle* h, const char* path, void* stream);
hbs_status hbs_load(const char* path, void* stream, hbs_handle** out);

/*
 * Serving: built solvers kept resident and solved for a stream of requests.  The block
 * solve (Sec. 6, second step) of one geometry handles any number of angles at once and
 * groups them by Bloch phase (Remark 3.1); a server turns a stream of single-angle
 * requests into such batches.  `slots` worker threads, each on its own CUDA stream of
 * the device current at creation, take all requests queued for one geometry (up to
 * `max_batch`) when they become free; requests arriving while other batches run join
 * the next batch, so batches grow with the load and up to `slots` of them overlap on
 * the device.  Results are those of hbs_solve for the same angles (to rounding).
 *
 * hbs_server_create: `hbm_budget_bytes` (0: no limit) bounds the device bytes of the
 *   admitted geometries.  Errors: INVALID_ARG (slots outside 1..64, max_batch < 1),
 *   CUDA (no device), OOM.
 * hbs_server_add: admits a built handle (borrowed: it must outlive its membership) and
 *   returns its geometry id; OOM if its hbs_info device_bytes do not fit the budget.
 * hbs_server_remove: waits until no queued or running request refers to the geometry,
 *   then releases its share of the budget.
 * hbs_server_submit: queues one angle theta in (-pi, 0) for a geometry; returns at once
 *   with a request id.  Thread-safe.
 * hbs_server_wait: waits up to timeout_s seconds for a request and hands over its result
 *   (one angle; read it with hbs_bragg_amplitudes(res, 0, ...), free with
 *   hbs_result_free).  Each request can be waited for once.  Errors: TIMEOUT (not
 *   finished yet; the request stays pending), or the solve's own status.
 * hbs_server_stats: counts, per-request latency percentiles (submit to completion) and
 *   completed requests per second since the first submission.
 * hbs_server_free: finishes every queued request, stops the workers and frees the server
 *   (not the admitted handles).
 */
typedef struct hbs_server hbs_server;
typedef struct hbs_server_stats_t {
  int64_t submitted, completed, batches;
  double mean_batch;      /* requests per solve call */
  double p50_latency_s, p99_latency_s, max_latency_s;
  double solves_per_s;
  size_t resident_bytes;  /* device bytes of the admitted geometries */
} hbs_server_stats_t;
hbs_status hbs_server_create(size_t hbm_budget_bytes, int slots, int max_batch, hbs_server** out);
hbs_status hbs_server_add(hbs_server* sv, const hbs_handle* h, int64_t* geometry_id);
hbs_status hbs_server_remove(hbs_server* sv, int64_t geometry_id);
hbs_status hbs_server_submit(hbs_server* sv, int64_t geometry_id, double theta, int64_t* request_id);
hbs_status hbs_server_wait(hbs_server* sv, int64_t request_id, double timeout_s, hbs_result** out);
hbs_status hbs_server_stats(hbs_server* sv, hbs_server_stats_t* st);
void hbs_server_free(hbs_server* sv);

/*
 * x = A^{-1} b with the compressed inverse (Sec. 4, telescoping apply),
 * for nrhs columns at once.  b and x are device arrays of N x nrhs complex128,
 * column-major with leading dimension N (N = hbs_info_t.unknowns: interlaced
 * [sigma; tau] per node for the transmission problem); they may not alias.
 */
hbs_status hbs_apply_inverse(const hbs_handle* h, const void* b, void* x, int64_t nrhs,
                             void* stream);

/*
 * Kernel block fill, the building block of every matrix in the method
 * (Sec. 2.3 entry formula): out[r + nr c] = entry(rows[r], cols[c]) for
 * device index arrays rows (nr) and cols (nc) into the boundary nodes of a
 * device geometry.  kind 0: A_ij (with I/2 and Kapur-Rokhlin weights);
 * kind 1: image block A_s with the source obstacle shifted by shift_x.
 * out is device complex128, nr x nc column-major.
 */
hbs_status hbs_kernel_block(const hbs_geometry* geom, double omega, int kind, double shift_x,
                            const int64_t* rows, int64_t nr, const int64_t* cols, int64_t nc,
                            void* out, void* stream);

/*
 * The same for the transmission problem (Sec. 5) with refractive index `index` > 0:
 * rows and cols index the 2 n interlaced unknowns (2p: s_p = sigma_p / omega, single
 * layer; 2p + 1: tau_p, double layer) and rows (2p: minus the normal derivative of the
 * outside minus the inside field, over omega; 2p + 1: its value).  kind 0: the operator A
 * (identity plus kernel differences between wavenumbers omega and index * omega,
 * Kapur-Rokhlin weights); kind 1: the image block of the pair shifted by shift_x
 * (outside wavenumber only).
 * Errors: INVALID_ARG (as hbs_kernel_block, or index <= 0), CUDA.
 */
hbs_status hbs_kernel_block_transmission(const hbs_geometry* geom, double omega, double index, int kind,
                                         double shift_x, const int64_t* rows, int64_t nr,
                                         const int64_t* cols, int64_t nc, void* out, void* stream);

/*
 * Interpolative decomposition (Def. 3.1) by column-pivoted QR of a device
 * matrix Mt = M^T (m x n, column-major, overwritten): M ~ P M(J, :).
 * On return *rank = l, perm[0..n) (device int32) lists J = perm[0..l) first,
 * and T (device, l x (n - l) column-major, capacity min(m,n) x n) holds
 * R11^{-1} R12 so that P(perm[l + j], :) = T(:, j)^T.
 */
hbs_status hbs_row_id(void* mt, int64_t m, int64_t n, double tol, int* rank, int* perm, void* t,
                      void* stream);

/*
 * Batched in-place inverse of `count` complex128 blocks of size n x n (column-major,
 * back to back in device memory `a`), the per-node inversion step of Sec. 4 (D_tau^{-1}
 * in Eqs. def_muhD..def_muG): Gauss-Jordan elimination with partial pivoting, all
 * blocks in one launch (a persistent multi-CTA kernel for up to 128 blocks, one CTA per
 * block otherwise).  precision as for hbs_zgemm: _DOUBLE_FLOAT and _TENSOR run the
 * eliminations in double-float arithmetic.  1 <= n <= 4096, 1 <= count <= 2^20, else
 * HBS_ERR_INVALID_ARG.  Returns HBS_WARN_ILLCOND when a pivot is exactly zero (the
 * blocks' contents are then undefined) and HBS_ERR_TIMEOUT if a bounded barrier wait
 * of the persistent kernel gave up.  Synchronizes the stream.
 */
hbs_status hbs_batched_inverse(void* a, int64_t n, int64_t count, int precision, void* stream);

/*
 * Complex GEMM on device arrays (complex128, column-major):
 *   C = alpha op(A) B + beta C,
 * op(A) = A (m x k, lda >= m) or, with trans_a = 1, A^T (A stored k x m, lda >= k);
 * B is k x n (ldb >= k) and C m x n (ldc >= m); alpha and beta point to two host doubles
 * (re, im).  precision selects the arithmetic of the library's dense products:
 * HBS_PRECISION_FP64, _DOUBLE_FLOAT or _TENSOR (see above; products below the tensor
 * size limits use double-float).  Returns HBS_ERR_INVALID_ARG for negative sizes, short
 * leading dimensions, null pointers with nonzero sizes or an unknown precision, and
 * HBS_ERR_TIMEOUT if a tensor-core completion wait gave up.  Synchronizes the stream.
 */
hbs_status hbs_zgemm(int64_t m, int64_t n, int64_t k, const double* alpha, const void* a, int64_t lda, int trans_a,
                     const void* b, int64_t ldb, const double* beta, void* c, int64_t ldc, int precision,
                     void* stream);

/*
 * Profiling.  hbs_launch_count() is the number of kernels this library has
 * launched since it was loaded.  With hbs_profile_enable(1) every launch is also
 * bracketed by CUDA events on its stream; hbs_profile_get copies up to `max`
 * per-kernel records (launches, summed device milliseconds, summed algorithmic
 * flops and bytes; entries named "phase:..." are host wall time of build and
 * solve phases; entries named "in:<phase>:<kernel>" are the launches and device
 * milliseconds of one kernel inside one phase, charged to the innermost phase open on
 * the launching host thread) and returns the number of records.  hbs_profile_reset
 * clears them.
 */
typedef struct hbs_kernel_stat {
  char name[80];
  int64_t launches;
  double ms;
  double flops;
  double bytes;
} hbs_kernel_stat;
void hbs_profile_enable(int on);
void hbs_profile_reset(void);
int hbs_profile_get(hbs_kernel_stat* out, int max);
int64_t hbs_launch_count(void);

/*
 * Allocation-free interpolative decomposition.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory during the
 * call (a fixed, pre-reserved memory budget; code that cannot wait for cudaMalloc /
 * cudaFree, which synchronize the device; a foreign allocator in charge of memory).
 *
 * Same inputs, outputs and result as hbs_row_id, computed by the multi-CTA pivoted
 * QR, but its working arrays live in one fixed device array that the library
 * reserves on every GPU that loads it (about 4 MiB, kept until the process exits).
 * It calls no cudaMalloc, cudaFree or allocating library routine.
 *  - n may not exceed HBS_ROW_ID_STATIC_MAX_N columns; larger n returns
 *    HBS_ERR_INVALID_ARG.
 *  - The first call on a device looks up the array's device address (with that
 *    device current); make that first call before any CUDA graph capture.
 *  - Every call waits for `stream` before it returns: it steps the pivot search
 *    from the host and reads the rank back.  No call may therefore run while the
 *    stream is being captured into a CUDA graph.
 *  - All calls share the one array and it keeps the last call's contents: two
 *    calls that overlap on the GPU (different streams, or different host threads)
 *    race and give wrong results.  Serialise them.
 */
#define HBS_ROW_ID_STATIC_MAX_N 262144
hbs_status hbs_row_id_static(void* mt, int64_t m, int64_t n, double tol, int* rank, int* perm,
                             void* t, void* stream);

/*
 * Error-path testing (the paper has no counterpart).  Nothing here makes a GPU fault,
 * trap or hang.
 *
 * hbs_fault_inject(kind, value) arms a host-side fault for the library's later calls
 * (process-wide, all threads):
 *  - HBS_INJECT_CLEAR: disarm everything (value ignored);
 *  - HBS_INJECT_ALLOC_FAILURE: the device allocation `value` allocations from now
 *    (0 = the next one) fails before cudaMallocAsync is called; the call that made
 *    it returns HBS_ERR_OOM and frees what it had allocated.  One failure per arming;
 *  - HBS_INJECT_RANK_CAP: interpolative decompositions of the persistent QR (tree
 *    levels of at most 128 nodes, the neighbour and periodizer IDs, hbs_row_id with
 *    n > 4096) may reach rank `value` at most (0 = no cap); one that needs more
 *    returns HBS_ERR_RANK, as an overflow of the supported maximum would.
 * Returns HBS_ERR_INVALID_ARG for an unknown kind or a negative value.
 *
 * hbs_barrier_selftest runs the library's bounded grid barrier (the one the
 * persistent QR, Gauss-Jordan and Schur kernels use) in a cooperative launch of
 * `ctas` CTAs (1..64) passing three barriers; CTA `absent_cta` (if in [0, ctas))
 * leaves before the second, so the others give up after `limit_s` seconds (0 < limit_s
 * <= 10) and return.  *passed (host int) = CTAs that passed all three.  Returns
 * HBS_ERR_TIMEOUT when a wait gave up, HBS_OK otherwise.  Synchronizes the stream.
 */
#define HBS_INJECT_CLEAR 0
#define HBS_INJECT_ALLOC_FAILURE 1
#define HBS_INJECT_RANK_CAP 2
hbs_status hbs_fault_inject(int kind, int64_t value);
hbs_status hbs_barrier_selftest(int ctas, int absent_cta, double limit_s, int* passed, void* stream);

void hbs_free(hbs_handle* h);
void hbs_result_free(hbs_result* r);
const char* hbs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HBSQP_H */
