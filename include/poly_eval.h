/*
 * poly_eval.h -- C ABI of the GB300 (sm_103a) partial modular polynomial
 * evaluation library.
 *
 * Problem (paper Sect. 2.1 and Sect. 2.3, Eq. 1): a prime p, a polynomial
 *     f = sum_{i=1..s} a_i x1^{d_i} x2^{e_i} M_i(x3, ..., xn)  over F_p,
 * a base point beta = (beta_3, ..., beta_n) in F_p^{n-2} and T points.  The
 * library computes the T bivariate images
 *     b_t(x1, x2) = f(x1, x2, beta^t),   t = t0, t0+1, ..., t0+T-1,
 * by the matrix method (Sect. 2.3, Algorithm 1): monomial values
 * m_i = M_i(beta) from per-variable power tables (Step A), then T rounds of
 * v_i <- v_i * m_i mod p with a segmented sum over each (x1, x2) group
 * (Step B, the "coefficient reductions").
 *
 * Output layout: a dense row-major T x G array of uint64, row r holding image
 * b_{t0+r}; column g is the g-th distinct (d, e) pair in descending
 * lexicographic order (Sect. 2.3: lex order with x1 > x2 > ...).  Every value
 * is canonical, in [0, p).  Zero coefficients are kept (Algorithm 1 skips
 * them; the dense layout does not).
 *
 * Conventions common to every call:
 *  - p is a run-time value, never a compile-time constant (Sect. 3.1 footnote).
 *  - Primality of p is the caller's contract; the library checks its width
 *    and parity only.
 *  - The input is a list of terms: repeated monomials are allowed (the images
 *    are linear in the terms) and zero coefficients are accepted.
 *  - Streams are passed as `void*` holding a cudaStream_t (NULL = legacy
 *    default stream).
 *  - No call ever falls back to a CPU computation.  Errors are returned as a
 *    pe_status; poly_eval_last_error() gives a message for the calling thread.
 *  - All handles are owned by the library and freed by their destroy call.
 */
#ifndef POLY_EVAL_H
#define POLY_EVAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PE_OK = 0,
    PE_ERR_ARG = 1,           /* a null pointer, a size out of range, beta_j not in [1, p) */
    PE_ERR_PRIME = 2,         /* p even, below 3, or too wide for the chosen modular product */
    PE_ERR_NOT_REDUCED = 3,   /* a coefficient a_i >= p */
    PE_ERR_EXP_RANGE = 4,     /* an exponent above 65535 */
    PE_ERR_NOMEM = 5,         /* device or host allocation failed */
    PE_ERR_ADMISSION = 6,     /* server: request larger than the memory cap, or queue full */
    PE_ERR_CUDA = 7,          /* a CUDA runtime error (message in poly_eval_last_error) */
    PE_ERR_TIMEOUT = 8,       /* server poll: not finished within the timeout */
    PE_PENDING = 9,           /* server poll with zero timeout: still running */
    PE_ERR_NOT_FOUND = 10,    /* server: unknown ticket or resident polynomial */
    PE_ERR_SINGULAR = 11      /* interpolation: repeated monomial values, or a zero one with t0 > 0 */
} pe_status;

/*
 * Modular product used in Step B (the T x s Hadamard products).
 *   PE_MODMUL_BARRETT64: Barrett's product (Sect. 3.1) specialised to a fixed
 *       multiplier: per term the quotient floor(m_i 2^64 / p) is precomputed,
 *       so v*m_i mod p costs one high and two low 64-bit products.  p odd,
 *       3 <= p < 2^62.
 *   PE_MODMUL_MONT64: Montgomery reduction (Sect. 3.1) with R = 2^64, m_i kept
 *       in Montgomery form.  p odd, 3 <= p < 2^62.
 *   PE_MODMUL_FP64: the floating-point FMA product of Algorithm 2 and the
 *       addition of Algorithm 3, in IEEE binary64.  p odd, 3 <= p < 2^50.
 *   PE_MODMUL_BARRETT32: the fixed-multiplier Barrett product in 32-bit
 *       words (one high and two low 32-bit multiplies), for the smaller primes
 *       the paper names as future work (Sect. 6).  p odd, 3 <= p < 2^30.
 *   PE_MODMUL_AUTO: BARRETT32 when p < 2^30, else BARRETT64 (the fastest on
 *       this GPU at each width), unless the autotuner has recorded otherwise.
 * All variants give identical, canonical results.
 */
typedef enum {
    PE_MODMUL_AUTO = 0,
    PE_MODMUL_MONT64 = 1,
    PE_MODMUL_FP64 = 2,
    PE_MODMUL_BARRETT64 = 3,
    PE_MODMUL_BARRETT32 = 4
} pe_variant;

/* pe_poly_desc.flags */
#define PE_FLAG_DEVICE_PTRS 0x1u  /* coeffs and exps are device pointers */
#define PE_FLAG_SORTED      0x2u  /* hint: terms already in descending (d, e) order */
#define PE_FLAG_BORROW      0x4u  /* server submit: the arrays stay valid and unchanged until the
                                     request's ticket completes, so they are not copied */

#define PE_MAX_VARS 66            /* n <= 66, i.e. at most 64 evaluated variables */

/*
 * A polynomial in term-list form (Eq. 1).
 *   p        : the prime modulus.
 *   n        : number of variables x1..xn, 2 <= n <= PE_MAX_VARS.
 *   exp_bytes: width of one exponent in `exps`: 1 (uint8), 2 (uint16) or 4 (uint32).
 *   s        : number of terms (0 allowed).
 *   coeffs   : s values a_i, each < p.
 *   exps     : s x n exponents, row-major: exps[i*n + 0] = d_i (x1),
 *              exps[i*n + 1] = e_i (x2), exps[i*n + k-1] = exponent of x_k.
 *   flags    : PE_FLAG_* bits.
 *   variant  : modular product used by poly_eval_run.
 * The descriptor and the arrays are read during the create call only.
 */
typedef struct {
    uint64_t p;
    uint32_t n;
    uint32_t exp_bytes;
    uint64_t s;
    const uint64_t *coeffs;
    const void *exps;
    uint32_t flags;
    pe_variant variant;
} pe_poly_desc;

typedef struct pe_poly pe_poly;

/*
 * Validates the terms, groups them by (d, e) (a stable sort into descending
 * lexicographic order unless they already are, Sect. 2.3), packs them into a
 * structure-of-arrays layout and copies them to the current CUDA device.
 * The returned handle owns that device memory until poly_eval_destroy.
 * Errors: PE_ERR_ARG, PE_ERR_PRIME, PE_ERR_NOT_REDUCED, PE_ERR_EXP_RANGE,
 * PE_ERR_NOMEM, PE_ERR_CUDA.  On error *out is set to NULL.
 */
pe_status poly_eval_create(const pe_poly_desc *desc, pe_poly **out);

/*
 * The same terms modulo another prime (multi-prime evaluation for Chinese
 * remaindering, the smaller primes of the paper's concluding remarks): a new
 * handle that shares `layout`'s exponents, groups and term order on the
 * device and owns only its coefficients.  `coeffs` holds the s coefficients
 * reduced mod p, in the order of the terms given to poly_eval_create for
 * `layout` (host, or device with PE_FLAG_DEVICE_PTRS in `flags`).  The shared
 * exponents live until the last handle that uses them is destroyed, so
 * `layout` may be destroyed first.
 * Errors: PE_ERR_ARG, PE_ERR_PRIME, PE_ERR_NOT_REDUCED, PE_ERR_NOMEM, PE_ERR_CUDA.
 */
pe_status poly_eval_create_like(const pe_poly *layout, uint64_t p, const uint64_t *coeffs, uint32_t flags,
                                pe_variant variant, pe_poly **out);

/*
 * Number of nonempty (x1, x2) groups G and, if keys != NULL, their (d, e)
 * pairs in column order: keys[2g] = d, keys[2g+1] = e (host array of 2G).
 */
pe_status poly_eval_groups(const pe_poly *poly, uint64_t *G, uint32_t *keys);

/*
 * Evaluates the T bivariate images b_t = f(x1, x2, beta^t), t = t0..t0+T-1
 * (Sect. 2.1; t0 = 1 avoids the unlucky point beta^0, t0 = 0 is allowed).
 *   T    : at most 2^31 points, the last of them t0 + T - 1 below 2^64, and
 *          T x G at most 2^60 values (else PE_ERR_ARG); T = 0 does nothing.
 *   beta : host array of n-2 values, each in [1, p).
 *   out  : T x G uint64 (layout above), host or device memory.  With a device
 *          pointer the call is asynchronous on `stream`; with a host pointer it
 *          copies the result back and returns after the stream has finished.
 * Runs Step A (power tables, monomial values) and Step B (Hadamard products
 * and coefficient reductions) as CUDA kernels.  Scratch device memory is owned
 * by the handle and reused by later calls, so runs of one handle execute one
 * after another on the device even when issued on different streams (each
 * run's stream waits for the previous run); use separate handles for
 * concurrent evaluations.  The host-side call itself is not thread-safe per
 * handle.
 */
pe_status poly_eval_run(pe_poly *poly, const uint64_t *beta, uint64_t T, uint64_t t0,
                        uint64_t *out, void *stream);

/*
 * The same images by the asymptotically fast method (Sect. 2.3.1): for each
 * group, sum_t b_(t0+t) z^t = N(z)/D(z) with D = prod (1 - m_i z), from a
 * product tree of NTT polynomial products and a Newton inversion of D, in
 * O(s log^2 T) products instead of s*T.  Needs an NTT-friendly prime: p - 1
 * divisible by 2*Tp, Tp = T rounded up to a power of two (at least 64); and
 * T <= 4096.  Arguments, layout and ordering as poly_eval_run; the result is
 * identical.  Errors: PE_ERR_ARG, PE_ERR_PRIME (p - 1 lacks the power of
 * two), PE_ERR_NOMEM, PE_ERR_CUDA.
 */
pe_status poly_eval_run_fast(pe_poly *poly, const uint64_t *beta, uint64_t T, uint64_t t0, uint64_t *out,
                             void *stream);

/* Waits for the device to finish queued work (like cudaFree), then frees the
 * handle and returns its device memory to the library's pool (NULL: no-op). */
void poly_eval_destroy(pe_poly *poly);

/* Message for the last failed call on this thread ("" if none). */
const char *poly_eval_last_error(void);

/*
 * Testing aid for failure paths: the nth device allocation the library makes
 * from now on (in any thread) fails as if the device were out of memory, and
 * the call that made it returns PE_ERR_NOMEM; 0 cancels a pending failure.
 * No GPU fault is involved; handles stay usable afterwards.
 */
pe_status poly_eval_debug_fail_alloc(uint32_t nth);

/*
 * Tile shape of Step B.  A warp-lane owns a chunk of at most K consecutive
 * terms of one group and keeps their state in registers across a range of
 * points (the paper's dependent evaluations T_d, Sect. 4.1); 32 chunks form a
 * slab; a work item is `slabs` consecutive slabs over `tchunk` consecutive
 * points.  Zero fields mean "choose automatically".
 */
typedef struct {
    uint32_t K;               /* terms per lane: 1, 2, 4, 8, 12 or 16 */
    uint32_t slabs;           /* slabs per work item */
    uint32_t tchunk;          /* points per work item */
    uint32_t warps_per_block; /* 1..8 (the plain Step B kernel uses at most 4) */
    uint32_t tail;            /* with slabs and tchunk forced: final points run as a band of
                                 one-slab items issued after the others (0: none) */
} pe_tiles;

/* Forces tile parameters for later runs of this handle (NULL = automatic). */
pe_status poly_eval_set_tiles(pe_poly *poly, const pe_tiles *tiles);

/* Tile parameters chosen for a run with T points, and the work decomposition. */
typedef struct {
    pe_tiles tiles;
    pe_variant variant;
    uint64_t chunks;          /* lane chunks (padded K-term pieces of groups) */
    uint64_t items;           /* warp work items per run */
    uint64_t spans;           /* groups whose terms cross work-item boundaries */
    uint64_t padded_terms;    /* chunks * K */
    uint64_t tail_points;     /* last points run as one-slab items after the others (0: none) */
    uint32_t method;          /* what poly_eval_run uses for this T: 0 matrix method, 1 fast method
                                 (poly_eval_tune measured it faster; NTT-friendly p) */
} pe_plan_info;

pe_status poly_eval_plan_info(pe_poly *poly, uint64_t T, pe_plan_info *info);

/*
 * Kernel timing of later poly_eval_run calls: with timing enabled, each run
 * records CUDA events on its launch stream around every kernel.
 * poly_eval_kernel_times waits for the recorded runs, returns the summed
 * durations in milliseconds -- ms[0] power tables, ms[1] Step A, ms[2] Step B --
 * and the number of runs, then starts a new sum.
 */
pe_status poly_eval_set_timing(pe_poly *poly, int enable);
pe_status poly_eval_kernel_times(pe_poly *poly, double ms[3], uint64_t *runs);

/* Number of kernel launches one poly_eval_run issues (for launch accounting). */
pe_status poly_eval_launches_per_run(pe_poly *poly, uint64_t T, uint32_t *launches);

/*
 * Sparse images (Algorithm 1 adds a coefficient c to b_t only when c != 0):
 * turns dense T x G images (device, as written by poly_eval_run) into a CSR
 * structure on the device.
 *   row_ptr  : device, T+1 entries; image r's entries are [row_ptr[r], row_ptr[r+1]).
 *   cols     : device, nonzero column indices (group g), ascending within a row.
 *   vals     : device, the matching coefficients.
 *   capacity : entries available in cols and vals.
 *   nnz      : host; receives the number of nonzero coefficients.
 * Synchronizes `stream` once (to learn nnz).  If nnz > capacity nothing is
 * written to cols/vals and PE_ERR_ARG is returned with *nnz set, so the
 * caller can retry with larger arrays.
 */
pe_status poly_eval_compact(const uint64_t *dense, uint64_t T, uint64_t G, uint64_t *row_ptr, uint32_t *cols,
                            uint64_t *vals, uint64_t capacity, uint64_t *nnz, void *stream);

/*
 * Monomial values z_i = M_i(beta) (the m_i of Step A, Sect. 2.3), canonical
 * in [0, p), in the library's term order: terms stably sorted by (d, e) in
 * descending lexicographic order, so input that is already sorted keeps its
 * order.  The terms of column g of the images are [off[g], off[g+1]).
 *   beta : host, n-2 values in [1, p).
 *   z    : device, s values (written on `stream`).
 *   off  : host, G+1 values, or NULL.
 * Errors: PE_ERR_ARG, PE_ERR_CUDA.
 */
pe_status poly_eval_monomials(pe_poly *poly, const uint64_t *beta, uint64_t *z, uint64_t *off, void *stream);

/*
 * Interpolation from images at successive powers (Sect. 1: with the points
 * beta^t the linear systems of sparse interpolation are transposed
 * Vandermonde systems).  For every column g with n_g = off[g+1] - off[g]
 * terms, solves
 *     sum_{i < n_g} c[off[g] + i] * z[off[g] + i]^(t0 + k) = images[k * lda + g],  k = 0..n_g-1,
 * i.e. recovers the coefficients of one (x1, x2) coefficient of f from its
 * first n_g images b_t0, b_t0+1, ... and its monomial values.  O(n_g^2)
 * operations per column, all columns in parallel.
 *   p      : odd prime, 3 <= p < 2^62.
 *   off    : host, G+1 nondecreasing term offsets, off[0] = 0, off[G] < 2^32;
 *            at most 2^24 terms per column.
 *   z      : device, off[G] monomial values in [0, p), distinct within a column.
 *   images : device, rows x lda uint64 (lda >= G), e.g. poly_eval_run's output
 *            with lda = G; rows must be at least the largest n_g.
 *   c      : device, off[G] outputs in [0, p).
 * Synchronizes `stream` once (to read the status).  Errors: PE_ERR_PRIME,
 * PE_ERR_ARG, PE_ERR_NOT_REDUCED (a node >= p), PE_ERR_SINGULAR (two equal
 * nodes in a column, or a zero node with t0 > 0; the message names the
 * column), PE_ERR_CUDA.
 */
pe_status poly_eval_vandermonde_solve(uint64_t p, uint64_t G, const uint64_t *off, const uint64_t *z,
                                      const uint64_t *images, uint64_t rows, uint64_t lda, uint64_t t0,
                                      uint64_t *c, void *stream);

/*
 * Kernel timing of poly_eval_vandermonde_solve on the calling host thread.
 * enable > 0 turns event timing on for later calls, 0 turns it off, < 0
 * leaves it unchanged.  If ms != NULL it receives the kernel times in
 * milliseconds of the latest timed call: ms[0] leaves and image gather,
 * ms[1] product tree (all levels), ms[2] correlation, ms[3] Horner and solve.
 */
pe_status poly_eval_vandermonde_timing(int enable, double ms[4]);

/*
 * Step B for callers that cannot allocate device memory.  The paper has no
 * counterpart; it exists because some callers may not call cudaMalloc (code
 * inside another framework's memory pool, embedded runtimes without allocator
 * access, processes that must not grow after start-up).  It allocates
 * nothing: all scratch comes from one fixed 32 MiB device array that the
 * library reserves on every GPU where it is loaded, until the process exits.
 *   p         : odd, 3 <= p < 2^62 (Barrett product).
 *   coeffs    : device, s coefficients a_i < p, sorted so that each group's
 *               terms are contiguous, groups in output-column order.
 *   m         : device, s monomial values m_i = M_i(beta) in [0, p) (Step A).
 *   group_off : device, G+1 uint32 offsets: group g is terms
 *               group_off[g] .. group_off[g+1]-1 (nonempty, group_off[G] = s).
 *               The offsets stay on the device and are not checked: offsets
 *               that break this rule give unspecified images but no access
 *               outside the inputs, the output or the scratch array.
 *   out       : device, T x G, row r = image at point t0 + r.
 * Asynchronous on `stream`.  The first call on a device looks up the scratch
 * address with that device current; make it before any stream capture.
 * Every call shares the one array, so calls that overlap on the GPU race:
 * serialise them (one stream, or events).  Inputs whose s*T needs more than
 * the fixed scratch are rejected with PE_ERR_ARG and a message.
 */
pe_status poly_eval_stepb_noalloc(uint64_t p, uint64_t s, uint64_t G, const uint64_t *coeffs,
                                  const uint64_t *m, const uint32_t *group_off, uint64_t T, uint64_t t0,
                                  uint64_t *out, void *stream);

/*
 * The work decomposition poly_eval_stepb_noalloc would use for s terms and T
 * points, without running anything: shape[0] = work units U (each kslabs
 * whole slabs of 32 terms), shape[1] = T-chunks Q, shape[2] = points per
 * T-chunk Tc, shape[3] = kslabs.  Host-only; it reads the device's SM count.
 * All zero for s = 0 or T = 0.  Errors: PE_ERR_ARG for a NULL shape, sizes
 * out of range, or inputs too large for the fixed scratch (the same
 * rejection as poly_eval_stepb_noalloc).  The paper has no counterpart.
 */
pe_status poly_eval_stepb_noalloc_shape(uint64_t s, uint64_t T, uint32_t shape[4]);

/* -------------------------------------------------------------------------
 * Batched evaluation: many polynomials, each with its own beta, T, t0 and
 * prime, evaluated by one persistent kernel with a device-side work queue.
 * ---------------------------------------------------------------------- */
typedef struct {
    pe_poly *poly;
    const uint64_t *beta;     /* host, n-2 values in [1, p) */
    uint64_t T;
    uint64_t t0;
    uint64_t *out;            /* device, T x G */
} pe_job;

typedef struct pe_batch pe_batch;

/*
 * Plans a batch: per-job tiles (from the autotuner cache when present),
 * a work queue ordered by decreasing cost, and a CUDA graph of the batch
 * (power tables for every job, then one persistent kernel that runs Step A
 * fused into Step B for every work item).  Jobs of at least 2^28
 * term-points (s*T) fill the GPU on their own: they are left out of the
 * graph and run as plain runs (poly_eval_run's matrix method, with the
 * handle's scratch) after it.  Job descriptors are copied.
 */
pe_status poly_eval_batch_plan(const pe_job *jobs, size_t njobs, pe_batch **out);

/* Launches the planned batch's CUDA graph on `stream`, then its plain runs
 * (asynchronous; the handles of plain runs must not be run elsewhere
 * meanwhile, as for poly_eval_run). */
pe_status poly_eval_batch_launch(pe_batch *batch, void *stream);

/* Kernel launches per poly_eval_batch_launch (the graph's and the plain
 * runs') and the number of jobs that run as plain runs; either pointer may
 * be NULL. */
pe_status poly_eval_batch_launches(const pe_batch *batch, uint32_t *kernels, uint32_t *plain_jobs);

/* Replaces the beta values of job `j` for later launches (same T and t0). */
pe_status poly_eval_batch_set_beta(pe_batch *batch, size_t j, const uint64_t *beta);

void poly_eval_batch_destroy(pe_batch *batch);

/* One-shot convenience: plan, launch on `stream`, synchronize, destroy. */
pe_status poly_eval_batch(const pe_job *jobs, size_t njobs, void *stream);

/* -------------------------------------------------------------------------
 * Autotuner: times candidate tile shapes for a polynomial on the current
 * device and records the fastest under a shape bucket; later plans of any
 * polynomial in the same bucket use it.
 * ---------------------------------------------------------------------- */
pe_status poly_eval_tune(pe_poly *poly, uint64_t T, pe_tiles *best, double *best_ms);
pe_status poly_eval_tune_save(const char *path);   /* JSON lines */
pe_status poly_eval_tune_load(const char *path);

/* -------------------------------------------------------------------------
 * Server: continuous batching of evaluation requests.  Requests are
 * admitted by device memory, polynomials can stay resident across
 * requests, and admitted jobs are packed into persistent-kernel epochs
 * that overlap on up to four streams (four by default).  While other epochs
 * run, an epoch of fewer than 16 ready requests waits until 16 are ready or
 * its oldest request is 2 ms old (larger epochs use the GPU better).
 * ---------------------------------------------------------------------- */
typedef struct {
    uint64_t mem_cap_bytes;   /* cap on resident terms + scratch + outputs */
    uint32_t max_queue;       /* pending requests before PE_ERR_ADMISSION */
    uint32_t max_epoch_jobs;  /* jobs packed into one epoch */
    uint32_t streams;         /* epochs in flight (1..4; 0: 4) */
} pe_server_cfg;

typedef struct pe_server pe_server;

/*
 * One request.  Exactly one of `poly_desc` (a new polynomial, copied at
 * submit and uploaded by the server) and `resident_id` (a polynomial already
 * on the device, reused at a new beta) is used: resident_id = 0 selects
 * poly_desc.  `out` is a host buffer of T x G uint64 that must stay valid
 * until the ticket completes; page-locked buffers are filled by an
 * asynchronous copy, others through a staging buffer.
 */
typedef struct {
    const pe_poly_desc *poly_desc;
    uint64_t resident_id;
    const uint64_t *beta;
    uint64_t T;
    uint64_t t0;
    uint64_t *out;
    uint64_t *new_resident_id; /* optional: with poly_desc, receives (at submit) the id under which
                                  the uploaded polynomial stays resident; requests may use it once
                                  this request's ticket has completed (least recently used
                                  residents are evicted first when memory is needed) */
} pe_request;

typedef struct {
    uint64_t submitted, completed, rejected, epochs;
    double p50_ms, p99_ms, max_ms;      /* submit-to-completion latency */
    double term_points;                 /* sum of s*T over completed requests */
    double busy_s;                      /* wall time with at least one epoch in flight */
    uint64_t resident_bytes, resident_polys, evictions;
    double upload_s, plan_s, launch_s, finish_s;   /* worker time: uploads, batch planning,
                                                      enqueueing, completing tickets */
} pe_server_stats;

pe_status poly_eval_server_create(const pe_server_cfg *cfg, pe_server **out);
/* Uploads a polynomial into the resident store; returns its id (> 0). */
pe_status poly_eval_server_register(pe_server *srv, const pe_poly_desc *desc, uint64_t *resident_id);
/* Queues a request; PE_ERR_ADMISSION is backpressure (queue full or too large). */
pe_status poly_eval_server_submit(pe_server *srv, const pe_request *req, uint64_t *ticket);
/* PE_OK when done (result in req->out), PE_PENDING / PE_ERR_TIMEOUT otherwise. */
pe_status poly_eval_server_poll(pe_server *srv, uint64_t ticket, int64_t timeout_us);
pe_status poly_eval_server_stats(pe_server *srv, pe_server_stats *stats);
/* Stops (paused = 1) or resumes (0) the forming of new epochs; epochs already
 * in flight complete and submissions keep queueing up to max_queue. */
pe_status poly_eval_server_pause(pe_server *srv, int paused);
void poly_eval_server_destroy(pe_server *srv);

/* -------------------------------------------------------------------------
 * Roofline calibration: a register-only kernel that runs the Step B inner
 * operation (one modular product and one modular addition per term-point,
 * Algorithm 1) on independent chains at full occupancy; returns its rate in
 * term-points per second and the SM clock seen by the kernel.
 * ---------------------------------------------------------------------- */
pe_status poly_eval_modmul_peak(pe_variant variant, uint64_t p, double *term_points_per_s,
                                double *sm_clock_mhz);

/*
 * Measured issue rates of single 32-bit integer instructions, in thread
 * operations per SM per clock, from independent dependency chains at full
 * occupancy: rates[0] mad.lo.u32, rates[1] mad.hi.u32, rates[2] mad.wide.u32,
 * rates[3] add.u32.  They are the unit counts behind the integer roofline.
 */
pe_status poly_eval_int_pipe_rates(double rates[4]);

/*
 * Measured issue rates of single FP64 instructions, in thread operations per
 * SM per clock, from independent dependency chains at full occupancy:
 * rates[0] fma.rn.f64, rates[1] add.rn.f64.  They are the unit counts behind
 * the roofline of Algorithm 2's product (paper Sect. 3.2), which runs on the
 * FP64 pipe.
 */
pe_status poly_eval_fp64_pipe_rates(double rates[2]);

/* Streaming multiprocessors of the current device (the unit count of every
 * roofline above).  Errors: PE_ERR_ARG for NULL, PE_ERR_CUDA without a device. */
pe_status poly_eval_num_sms(uint32_t *sms);

#ifdef __cplusplus
}
#endif
#endif /* POLY_EVAL_H */
