/*
 * h2eig.h -- C ABI of the GB300 library for the k-th eigenvalue of a symmetric
 * kernel matrix compressed as an H^2-matrix, by slicing the spectrum with the
 * generalized H^2-LDL^T factorization of Apriansyah & Yokota, "Computing the
 * k-th Eigenvalue of Symmetric H^2-Matrices" (arXiv 2311.08618).
 *
 * Problem statement (Sec. 1, Sec. 2): A is n x n real symmetric with entries
 * A_ij = f(|x_i - x_j|) for points x_i; nu(A - mu I) = #{lambda(A) < mu} is
 * the number of negative pivots of an LDL^T of the shifted matrix (Sylvester's
 * law of inertia, Eq. 2); Algorithm 1 bisects on nu to find lambda_k.
 *
 * Conventions shared by every entry point:
 *  - Return H2_OK (0) on success, a negative H2_ERR_* code otherwise; the
 *    message of the last failure on the calling thread is h2_last_error().
 *  - No exception crosses this boundary.  Inputs are copied; caller-owned
 *    outputs are written only on success.
 *  - Host pointers are plain CPU memory; "device" pointers are CUDA global
 *    memory on the handle's device.  The library owns all memory it allocates
 *    and frees it in h2_destroy.
 *  - A handle is used by one host thread at a time (one handle per stream).
 *    Several handles may share one stream.  Running several handles' batches
 *    concurrently on separate streams stalled the device in testing (every
 *    started kernel completed while a queued one never started); prefer one
 *    stream for handles that are used together.
 *  - Every computation runs in the library's CUDA kernels; there is no CPU
 *    fallback.  Without a usable CUDA device, h2_build fails with H2_ERR_CUDA.
 */
#ifndef H2EIG_H
#define H2EIG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define H2_OK               0
#define H2_ERR_INVALID_ARG (-1)  /* a null pointer, n < 1, k out of 1..n, ... */
#define H2_ERR_OOM         (-2)  /* device allocation failed                  */
#define H2_ERR_NUMERICAL   (-3)  /* NaN/Inf met in the factorization           */
#define H2_ERR_TIMEOUT     (-4)  /* a bounded device wait ran out              */
#define H2_ERR_INTERVAL    (-5)  /* nu(a) != 0 or nu(b) != n at the start      */
#define H2_ERR_CUDA        (-6)  /* a CUDA runtime call failed                 */

/* ---- kernels f(r) (Sec. 5.1 and the synthetic workloads) ----------------- */
typedef enum {
    H2_K_LAPLACE_EPS    = 0,  /* 1/(r + p0)              (Sec. 5.1, p0 = 1e-3) */
    H2_K_YUKAWA_EPS     = 1,  /* exp(-r)/(r + p0)                              */
    H2_K_GAUSS_PLUS_INV = 2,  /* exp(-r^2/2) + p0/(r + p1)                     */
    H2_K_TRIDIAG_TEST   = 3,  /* 2 at r = 0, -1 at r = 1, else 0 (1D integers) */
    H2_K_MIN_TEST       = 4   /* min(x_i, x_j) of the first coordinates        */
} h2_kernel_kind;

typedef struct {
    int kind;        /* an h2_kernel_kind */
    double p[4];     /* its parameters, unused entries ignored */
} h2_kernel;

/* ---- options ------------------------------------------------------------ */
#define H2_ADM_BOX    0  /* max(diam c, diam d) <= eta * dist(box c, box d) */
#define H2_ADM_CENTER 1  /* (diam c + diam d)/2 <= eta * |center c - center d| */
#define H2_ADM_WEAK   2  /* every pair of distinct clusters (HSS, Sec. 3.3): only
                            diagonal blocks stay dense, no fill-ins, one colour per
                            level; eta is ignored */

#define H2_PREC_FP64  0  /* every step in FP64 */
#define H2_PREC_MIXED 1  /* Schur-update, triangular-solve and rotation
                            products in FP32 (FP32 accumulation); storage,
                            Bunch-Kaufman pivoting, pivot counts and interval
                            updates in FP64; counts certified, uncertified
                            shifts re-run in FP64 (see h2_inertia,
                            h2_kth_eig) */
#define H2_PREC_FP64_TC 2 /* as H2_PREC_FP64, but the Schur-update products
                            W_a Y_b^T and the rotation products (block x V)
                            run on the tensor cores: 8 exact 7-bit
                            integer digits per FP64 entry (row-scaled), BF16
                            digit products summed exactly, one FP64 rounding
                            per entry; the error stays below 2^-53 of the
                            result plus 1.24e-16 K of the row-scale products
                            (the powers of two above each row's entries) */

typedef struct {
    int precision;       /* H2_PREC_FP64 (default), H2_PREC_MIXED or
                            H2_PREC_FP64_TC */
    int admissibility;   /* H2_ADM_BOX (default), H2_ADM_CENTER or H2_ADM_WEAK */
    double eps_h2;       /* truncation tolerance relative to ||A||_inf (Sec. 3.1,
                            eps_H2; default 1e-10 = 1e-2 * 1e-8, Sec. 5) */
    int fill_cap;        /* max skeleton columns per cluster after fill-in
                            recompression (Sec. 3.4); 0 = 2 * rank */
    int sketch_cols;     /* columns of the random sketch of A_{l;c,+}; 0 = rank + 16 */
    uint64_t seed;       /* SplitMix64 state for the sketch matrix */
    int max_lanes;       /* shifts factorized concurrently, <= 65535; 0 = 64
                            (without hbm_budget) */
    double pivot_guard;  /* mixed precision: a shift whose min |pivot| is below
                            pivot_guard * ||A||_inf is re-run in FP64 (on top
                            of the certificate of h2_inertia); 0 = 1e-3.  At
                            a shift where the reduced blocks are nearly
                            singular, the FP32 error can exceed Delta; the
                            mixed pivots there were measured below
                            4e-4 ||A||_inf */
    void* stream;        /* cudaStream_t for all work of the handle; NULL = a
                            stream created by the library */
    int graphs;          /* 1 (default): each batch replays a CUDA graph
                            captured at build; 0: the batch's kernels are
                            launched one by one (the plain launch path) */
    int recomp_cluster_cols; /* fill recompression of a level whose Z (the
                            redundant rows of all fill blocks of a row, Sec.
                            3.4) may reach this many columns runs on a cluster
                            of 8 CTAs; 0 = 4096, < 0 = never */
    int autotune;        /* 1: at build, time the Bunch-Kaufman kernels (one
                            warp, one 128-thread or one 256-thread CTA per
                            block) and both recompression kernels (one CTA,
                            8-CTA cluster) on full batches of shifts over the
                            Gershgorin interval and keep the fastest per level
                            (overrides recomp_cluster_cols); 0 (default):
                            fixed rules */
    size_t hbm_budget;   /* bytes of device memory the per-batch factorization
                            workspace may take (admission by HBM footprint):
                            0 (default) = no budget, max_lanes lanes; > 0 =
                            the most lanes whose workspace fits, at most
                            max_lanes (max_lanes = 0: no other bound); h2_build
                            fails with H2_ERR_OOM when one lane does not fit.
                            h2_info reports the lanes and bytes chosen */
    int tc_schur;        /* H2_PREC_FP64_TC, levels whose blocks have at most 64
                            rows: 1 = the Schur digit products on the
                            5th-generation tensor cores (tcgen05.mma, tensor-
                            memory accumulators; one CTA per 128-row panel of an
                            elimination's stacked targets), 0 (default) =
                            warp-level mma.sync tiles of 32 x 32.  Both give the
                            same values */
    int lookahead;       /* 1: within a level, once colour c's Schur updates
                            of the blocks in rows and columns of colour c + 1's
                            clusters are done, colour c + 1's recompression,
                            rotation, LDL^T and solves run on a second stream
                            beside colour c's remaining updates (graph-replayed
                            batches of the handle's own shifts; each block
                            takes its updates in the same order, so the results
                            are the same bit for bit; twice the factor-step
                            scratch); 0 (default): one stream, colour after
                            colour, which measured faster (the concurrent
                            Schur blocks slow the solves on the critical path) */
    int shifts_per_interval; /* h2_kth_eig rounds: at most this many shifts per
                            bracket still wider than tol (default 16), so
                            that few brackets do not take every lane: at
                            n = 1024 one k converges faster with 16 shifts
                            per round (17-section) than with 64; 0 = every
                            round uses all max_lanes lanes */
} h2_options;

/* Fills *opt with the defaults above.  Never fails. */
void h2_default_options(h2_options* opt);

/* ---- handle lifecycle ---------------------------------------------------- */
typedef struct h2_matrix* h2_handle;

/*
 * h2_build -- construct the H^2 matrix of A_ij = f(|x_i - x_j|) (Sec. 3.1,
 * Eqs. shared-bases, transfer-matrices, dense_skeleton, lr_skeleton) and keep
 * it resident and factor-ready on the current CUDA device.
 *   points : host, n x d row-major FP64, copied.
 *   n >= 1, 1 <= d <= 3, leaf >= 2 (maximum points per leaf cluster),
 *   rank   : cap on the skeleton rank of each shared basis (>= 0),
 *   eta > 0: strong-admissibility parameter.
 *   opt    : NULL for defaults.
 *   *out   : receives the handle on success, untouched on failure.
 * Errors: H2_ERR_INVALID_ARG, H2_ERR_OOM, H2_ERR_CUDA.
 */
int h2_build(const double* points, int64_t n, int d, h2_kernel kernel, int leaf,
             int rank, double eta, const h2_options* opt, h2_handle* out);

/* Frees every resource of h.  NULL is a no-op. */
void h2_destroy(h2_handle h);

/* Message of the last failure of an h2_* call on this thread ("" if none). */
const char* h2_last_error(void);

/* ---- inertia (Sec. 4, Eq. 2 with Eq. h2-generalized-ldl) ------------------ */
/*
 * h2_inertia -- counts[i] = nu(A~ - shifts[i] I) = #{j : D_jj < 0} of the
 * generalized H^2-LDL^T of the shifted matrix (strict: a zero pivot is not
 * negative).  min_abs_pivot[i] (nullable) = the smallest |eigenvalue| of a
 * 1x1 or 2x2 block of D, a guard for shifts close to an eigenvalue.
 *   shifts        : host, ns FP64.
 *   counts        : host, caller-owned, ns int64.
 *   min_abs_pivot : host, caller-owned, ns FP64, or NULL.
 * Shifts are processed in batches of max_lanes.  Blocks until done.
 * H2_PREC_MIXED: counts are certified (Parlett's criterion, Sec. 4.1).  The
 * FP32 products make each mixed factorization exact for a perturbed matrix
 * A~ + E; with Delta = 64 * 2^-24 * ||A||_inf > 2 ||E||, mixed counts at
 * mu - Delta and mu + Delta that agree equal nu(mu).  Each shift is therefore
 * factorized in mixed precision at mu - Delta and mu + Delta (two lanes); a
 * shift whose two counts differ, or whose smaller min |pivot| is below
 * pivot_guard * ||A||_inf, is factorized again in FP64 at mu.  All of it runs
 * on the device.  min_abs_pivot of a certified shift is the smaller of its two
 * mixed values.  h2_info counts the shifts checked and re-run.
 */
int h2_inertia(h2_handle h, const double* shifts, int64_t ns, int64_t* counts,
               double* min_abs_pivot);

/*
 * h2_inertia_device -- as h2_inertia with DEVICE pointers; enqueued on the
 * handle's stream and returns without waiting (ns <= max_lanes).  In
 * H2_PREC_MIXED the certified counts of h2_inertia, with the pair batches
 * (max_lanes / 2 shifts each) and the FP64 re-run batch all enqueued on the
 * stream (a one-lane handle runs every shift in FP64).
 */
int h2_inertia_device(h2_handle h, const double* d_shifts, int64_t ns, int64_t* d_counts,
                      double* d_min_abs_pivot);

/*
 * h2_autotune_choice -- the kernel choices of one level (0 = root .. L =
 * leaves): out[0] = threads per Bunch-Kaufman block factorization (32: one
 * warp per block, for blocks up to 64; 128 or 256: one CTA), out[1] = 1 if the fill
 * recompression runs on an 8-CTA cluster, else 0.  Reports the fixed rules
 * when the handle was built without autotune.
 *   out: host, 2 ints.  Errors: H2_ERR_INVALID_ARG.
 */
int h2_autotune_choice(h2_handle h, int level, int* out);

/*
 * h2_plan_summary -- the cluster tree and block structure that h2_build would
 * use for these points (binary tree, top-down block tree under the given
 * admissibility, fill-in closure, distance-2 colouring); host only, no device
 * is touched.  For tests and inspection.
 *   points    : host, n x d row-major FP64.
 *   perm      : host, n int64 (tree position -> input index), or NULL.
 *   levels    : receives L + 1 (levels 0 = root .. L = leaves).
 *   per_level : host, 5 * 64 int64, or NULL; for level l: [5l] clusters,
 *               [5l+1] near pairs, [5l+2] fill pairs, [5l+3] far pairs
 *               (ordered pairs, the diagonal included in near), [5l+4] colours.
 *   colours   : host, one int per cluster of every level (level-major, root
 *               first), or NULL.  The caller sizes it from a first call.
 * Errors: H2_ERR_INVALID_ARG (as h2_build; more than 64 levels).
 */
int h2_plan_summary(const double* points, int64_t n, int d, int leaf, double eta, int rule,
                    int64_t* perm, int* levels, int64_t* per_level, int* colours);

/* ---- batches over several matrices (one launch per level and colour) ---- */
typedef struct h2_group_set* h2_group;

/*
 * h2_group_create -- prepares one inertia batch over several resident
 * matrices.  Every kernel of the generalized LDL^T (Sec. 3.2-3.4) runs as one
 * launch per tree level, counted from the leaves, and per colour, covering the
 * work of all handles.  Each block finds its matrix in a per-launch table.
 * The batch is one CUDA graph.  The handles keep their own workspaces, so the
 * counts equal those of each handle's own batch.
 *   hs  : host, nh handles with equal max_lanes and precision, built on one
 *         stream (the group's); they must outlive the group and must not run
 *         their own batches while the group's is in flight.
 *   *out: receives the group on success, untouched on failure.
 * Errors: H2_ERR_INVALID_ARG (nh < 1, a null handle, mixed lanes or
 * precision), H2_ERR_OOM, H2_ERR_CUDA.
 */
int h2_group_create(const h2_handle* hs, int nh, h2_group* out);

/*
 * h2_group_inertia_device -- the counts (and min |pivot|) of every handle's
 * shifts, in one batch.  Enqueued on the group's stream; returns without
 * waiting.
 *   d_shifts        : device, nh * max_lanes FP64; handle i's shifts start at
 *                     i * max_lanes.
 *   ns              : host, nh ints in 0..max_lanes, the shifts of each handle.
 *   d_counts        : device, nh * max_lanes int64, same layout (caller-owned).
 *   d_min_abs_pivot : device, same layout FP64, or NULL.
 * H2_PREC_MIXED handles return certified counts as h2_inertia_device does:
 * group batches of (mu - Delta, mu + Delta) pairs, then one FP64 group batch
 * of every handle's uncertified shifts.  Errors: H2_ERR_INVALID_ARG,
 * H2_ERR_CUDA.
 */
int h2_group_inertia_device(h2_group g, const double* d_shifts, const int* ns, int64_t* d_counts,
                            double* d_min_abs_pivot);

/* Launches (grouped kernels plus the per-handle bookkeeping kernels) of one
 * group batch; < 0 for a NULL group. */
int h2_group_launches(h2_group g);

/* Frees the group (not its handles).  NULL is a no-op. */
void h2_group_destroy(h2_group g);

/* ---- k-th eigenvalues (Algorithm 1 with the inertia reuse of Sec. 4.2) ---- */
/*
 * h2_kth_eig -- out[i] = lambda~_{k[i]} of A~, the midpoint of a final
 * interval of width < tol found by bisection/multisection from the Gershgorin
 * interval (|lambda_k - lambda~_k| < tol/2, Eq. error-bound).  Every evaluated
 * (mu, nu) narrows every k (Sec. 4.2); each round spreads up to max_lanes
 * shifts, at most shifts_per_interval per interval, over the distinct active
 * intervals, the first max_lanes of them in k order (any number of k, in any
 * order, repeats allowed: up to all n eigenvalues in one call).  The
 * intervals stay on the device.
 * H2_PREC_MIXED: mixed rounds (one mixed factorization per shift, no per-shift
 * certificate) run while the brackets are wider than Delta = 64 * 2^-24 *
 * ||A||_inf: a wrong mixed count at mu means an eigenvalue within ||E|| of
 * mu, which as a rule moves a bracket end by less than Delta.  Every bracket
 * is then widened by Delta and checked in FP64 (nu(lo) < k <= nu(hi), else it
 * restarts from the Gershgorin interval), so a larger error costs a restart,
 * not a wrong result; FP64 rounds finish to tol.
 *   k         : host, nk int64, 1-based, each in 1..n.
 *   tol > 0   : absolute interval width.
 *   out       : host, caller-owned, nk FP64.
 *   err_bound : host, caller-owned, nk FP64 (half the final width), or NULL.
 * Errors: H2_ERR_INVALID_ARG, H2_ERR_INTERVAL, H2_ERR_NUMERICAL, H2_ERR_CUDA.
 */
int h2_kth_eig(h2_handle h, const int64_t* k, int64_t nk, double tol, double* out,
               double* err_bound);

/*
 * h2_kth_eig_in -- as h2_kth_eig, starting every bracket from the caller's
 * interval [lo, hi] instead of the Gershgorin interval: the work unit of the
 * parallel bisections of Sec. 4.2 (an interval known to hold a range of
 * eigenvalue indices, e.g. from earlier inertia counts or a master's free
 * list).  nu(lo) and nu(hi) are evaluated in FP64 first; every k must satisfy
 * nu(lo) < k <= nu(hi), else H2_ERR_INTERVAL (the message gives both counts).
 * Errors: as h2_kth_eig; H2_ERR_INVALID_ARG also for lo >= hi.
 */
int h2_kth_eig_in(h2_handle h, const int64_t* k, int64_t nk, double lo, double hi, double tol,
                  double* out, double* err_bound);

/*
 * h2_status -- waits for the handle's stream, then returns and clears the
 * device error record accumulated since the last h2_status or host-array call
 * (the asynchronous h2_inertia_device reports only here):
 *   info[0] = flags: 1 = NaN met in pivoting or recompression; 2 = a kernel
 *             found a size outside its buffers and skipped its work;
 *   info[1] = first reporting kernel (1 recompression, 2 rotation, 3 LDL^T,
 *             4 triangular solves, 5 Schur update, 6 merge);
 *   info[2..5] = its values, info[6..7] = its block indices.
 * info: host, caller-owned, 8 int64.  Returns H2_ERR_NUMERICAL when flags != 0.
 */
int h2_status(h2_handle h, int64_t* info);

/*
 * h2_heartbeat -- diagnostic, active only when the environment variable
 * H2_HEARTBEAT=1 is set before the first h2_build: copies 64 counters that
 * every factorization kernel updates in zero-copy host memory -- for kernel
 * kind j (0 init, 1 recompression, 2 rotation, 3 LDL^T, 4 triangular solves,
 * 5 Schur, 6 merge, 8 dims, 9 merge dims, 10 finish, 11 lane count):
 * out[4j] CTAs started, out[4j+1] threads finished, out[4j+2..4j+3] block
 * indices of the last CTA started.  Makes no CUDA call, so it can be read
 * while the device is busy.  Zeros when not enabled.  out: host, 64 uint32.
 */
void h2_heartbeat(uint32_t* out);

/* ---- introspection -------------------------------------------------------- */
typedef struct {
    int64_t n;
    int levels;              /* L + 1 (root level 0 .. leaf level L) */
    int leaves;
    int max_rank;            /* largest build rank of any shared basis */
    int64_t near_pairs;      /* ordered leaf pairs stored dense */
    int64_t fill_pairs;      /* ordered leaf pairs receiving fill-ins */
    double norm_inf;         /* ||A||_inf (max absolute row sum) */
    double gershgorin_lo;    /* min_i (A_ii - R_i) */
    double gershgorin_hi;    /* max_i (A_ii + R_i) */
    double trunc_tol;        /* eps_h2 * ||A||_inf */
    int64_t workspace_bytes; /* per-batch factorization workspace */
    int lanes;               /* shifts per batch */
    int kernels_per_batch;   /* kernel launches of one batch (CUDA graph nodes) */
    int last_rounds;         /* bisection rounds of the last h2_kth_eig */
    int64_t last_shifts;     /* shifts evaluated by the last h2_kth_eig */
    int last_mixed_rounds;   /* of those rounds, the mixed-precision ones */
    int64_t guard_reruns;    /* mixed precision: shifts the guard of h2_inertia,
                                h2_inertia_device and group batches re-ran in
                                FP64, total since the build (waits for the
                                handle's stream) */
    int64_t bracket_resets;  /* mixed brackets that failed their FP64 check (total) */
    int cap_bound;           /* clusters (all levels) whose pivoted QR stopped at
                                the rank cap with the sketch remainder still above
                                trunc_tol: the cap, not eps_h2, set their rank */
    double max_residual;     /* largest Frobenius norm of a sketch remainder left
                                out by the truncation (<= trunc_tol where the
                                tolerance, not the cap, stopped the QR) */
    int64_t guard_checked;   /* mixed precision: shifts the guard checked, total
                                since the build (guard_reruns / guard_checked =
                                re-run rate) */
} h2_stats;

int h2_info(h2_handle h, h2_stats* out);

/*
 * h2_profile_batch -- measurement aid.  Runs one batch of ns <= max_lanes
 * device-resident shifts like h2_inertia_device but without the CUDA graph,
 * recording CUDA events around every kernel launch on the handle's stream, and
 * blocks until done.  Per kernel kind j (H2_KIND_*): ms[j] = summed device time
 * of its launches, launches[j] = their number, flops[j] = algorithmic FP64
 * flops and bytes[j] = algorithmic bytes moved (operands read once, results
 * written once; see the design notes for the per-unit formulas).
 * All four arrays: host, caller-owned, H2_NKINDS entries.  d_counts: device, ns.
 */
#define H2_KIND_INIT   0   /* leaf blocks of A~ - sigma I                   */
#define H2_KIND_RECOMP 1   /* fill-in recompression basis (pivoted QR)      */
#define H2_KIND_ROTATE 2   /* rotation of a row's blocks, fill truncation   */
#define H2_KIND_LDL    3   /* Bunch-Kaufman LDL^T of S^RR, pivot count      */
#define H2_KIND_TRSM   4   /* S^{xR} P L^-T and D^-1 for each coupled block */
#define H2_KIND_SCHUR  5   /* Schur-complement updates                       */
#define H2_KIND_MERGE  6   /* merge into the parent level + transfer bases  */
#define H2_KIND_OTHER  7   /* dims, counts                                   */
#define H2_NKINDS      8
int h2_profile_batch(h2_handle h, const double* d_shifts, int64_t ns, int64_t* d_counts,
                     double* ms, int64_t* launches, double* flops, double* bytes);

/*
 * h2_dense_inertia_noalloc -- counts[i] = #{negative pivots} of a
 * Bunch-Kaufman LDL^T of A - shifts[i] I for a small DENSE symmetric matrix A
 * (the same kernel routine the H^2 factorization uses for its diagonal
 * blocks), and min_abs_pivot[i] as in h2_inertia, WITHOUT allocating any
 * memory.  The paper has no counterpart to this entry point.  It is for
 * callers that cannot call cudaMalloc: code that runs under a fixed device
 * memory budget reserved up front (an allocator owned by another framework
 * or a pre-sized pool), and code that must not add the device-wide
 * synchronization an allocation can cause (for example inside a
 * latency-critical serving loop).
 *   d_A             : device, n x n row-major FP64, leading dimension lda >= n;
 *                     only read; the full matrix is read and must be symmetric.
 *   d_shifts        : device, ns FP64.
 *   d_counts        : device, caller-owned, ns int64.
 *   d_min_abs_pivot : device, caller-owned, ns FP64, or NULL.
 *   stream          : cudaStream_t to enqueue on, NULL for the default stream.
 * Working memory is one static device array of H2_NOALLOC_MAX_DOUBLES doubles
 * (8 MiB) inside the library, which every GPU that loads the library holds
 * until the process exits.  A call uses ns * n * n doubles of it and returns
 * H2_ERR_INVALID_ARG, touching nothing, when that exceeds the maximum or when
 * n < 1, n > 1024, ns < 1, ns > 1024 or lda < n.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current, and later calls reuse it; make that first call before any stream
 * capture.  cudaDeviceReset on a device unloads the library's device code and
 * leaves that stored address stale: do not call this entry point on a device
 * after resetting it in the same process.  Every call shares the array: calls
 * that overlap on the GPU (on different streams or from different threads)
 * race and give wrong results.  Each call overwrites every scratch element it
 * reads, so nothing needs clearing between calls.
 * Asynchronous: returns once the kernel is enqueued.
 */
#define H2_NOALLOC_MAX_DOUBLES 1048576
int h2_dense_inertia_noalloc(const double* d_A, int n, int lda, const double* d_shifts, int ns,
                             int64_t* d_counts, double* d_min_abs_pivot, void* stream);

/*
 * h2_export -- copies one level of the resident H^2 representation (Sec. 3.1,
 * Eqs. shared-bases, transfer-matrices, lr_skeleton, dense_skeleton) to host
 * memory, for tests and inspection.  Every point index is in tree order
 * (h2_tree_perm).  Set buf->level (0 = root .. L = leaves) and the array
 * pointers; NULL arrays are skipped, so a first call with all of them NULL
 * returns the sizes.  Out:
 *   nc, dq     : clusters; leading dimension of each basis/transfer matrix;
 *   nfar, rbmax: stored far pairs (c > d); leading dimension of a coupling;
 *   nnear, dm  : stored leaf near pairs (c >= d, leaf level only, else 0);
 *                leading dimension of a near block.
 * Arrays (host, caller-owned):
 *   offsets  [nc + 1] int64: cluster c holds tree positions offsets[c]..;
 *   ranks    [nc] int: build rank r_c (skeleton size);
 *   residuals[nc] double: Frobenius norm of the sketch remainder that the
 *             truncation of c's basis left out;
 *   colours  [nc] int: distance-2 colour (elimination order, colour-major);
 *   Q        [nc][dq][dq] double, row-major: at the leaves the orthogonal
 *             [U^S U^R] of each cluster (m_c x m_c, the first r_c columns
 *             U^S); above, the transfer matrix of each cluster, rows = the
 *             children's skeleton coordinates (r_c1 + r_c2), first r_c
 *             columns the parent skeleton;
 *   far_pairs[2 nfar] int (c, d) and C [nfar][rbmax][rbmax] double: the
 *             coupling S_cd^SS = E_c^T A_cd E_d (r_c x r_d), E the expanded
 *             skeleton bases; S_dc^SS is its transpose;
 *   near_pairs[2 nnear] int (c, d) and B [nnear][dm][dm] double: the
 *             transformed near block [U^S U^R]_c^T A_cd [U^S U^R]_d.
 * Errors: H2_ERR_INVALID_ARG (level outside 0..L, null handle or buf),
 * H2_ERR_CUDA.
 */
typedef struct {
    int level;
    int nc, dq, nfar, rbmax, nnear, dm;
    int64_t* offsets;
    int* ranks;
    double* residuals;
    int* colours;
    double* Q;
    int* far_pairs;
    double* C;
    int* near_pairs;
    double* B;
} h2_export_buf;
int h2_export(h2_handle h, h2_export_buf* buf);

/*
 * h2_compression_error -- the compression error of the resident H^2 matrix,
 * measured on the device: *err2 = ||A - A~||_2 and *norm2 = ||A||_2, each by
 * `iters` steps of power iteration from one seeded start vector.  A~ x is the
 * nested H^2 product (skeleton coordinates up through the transfer matrices,
 * couplings, back down, plus the dense near blocks; Sec. 3.1), A x evaluates
 * the kernel entries on the fly (O(n^2) per step).  The accuracy requirement
 * of the compression is err2 / norm2 <= 1e-8.  Power iteration approaches both norms from below.
 * Blocks until done.  Errors: H2_ERR_INVALID_ARG (iters < 1, null pointers),
 * H2_ERR_OOM, H2_ERR_CUDA.
 */
int h2_compression_error(h2_handle h, int iters, double* err2, double* norm2);

/* tree order: perm[i] = index (0-based, in the input) of the i-th point in
 * tree order.  perm: host, caller-owned, n int64. */
int h2_tree_perm(h2_handle h, int64_t* perm);

/* build ranks of the shared bases of level `level` (0 = root .. L = leaves);
 * ranks: host, caller-owned, 2^level ints. */
int h2_level_ranks(h2_handle h, int level, int* ranks);

#ifdef __cplusplus
}
#endif

#endif /* H2EIG_H */
