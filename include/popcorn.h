/*
 * popcorn.h -- C ABI of a GB300 (sm_103a) Kernel K-means engine.
 *
 * The method is the matrix formulation of Kernel K-means of "Popcorn:
 * Accelerating Kernel K-means on GPUs through Sparse Linear Algebra"
 * (arXiv 2501.05587):
 *
 *   K = kappa(P P^T)                     (Sec. 3.2, Alg. 2 line 1)
 *   D = -2 K V^T + P~ + C~               (Eq. 11, Alg. 2 lines 7-10)
 *   cl(i) = argmin_j D_ij                (Alg. 2 lines 11-13)
 *
 * where V (k x n) holds 1/|L_j| at (j, i) for every point i of cluster j
 * (Eq. 8), P~ broadcasts diag(K) (Sec. 3.3) and C~ broadcasts the centroid
 * norms ||c_j||^2 = diag(V K V^T) (Eq. 13), obtained from the entries
 * (K V^T)_{i, cl(i)} (Eq. 14, "cnorms_gemv").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are row-major FP32.  P is n x d with leading dimension ldp >= d
 *   (elements).  K is n x n with leading dimension ldk >= n.
 * - Labels are 0-based int32 in [0, k).  (The paper draws labels in 1..k.)
 * - "stream" is a cudaStream_t (a CUstream); NULL means the legacy default
 *   stream.  Every call is stream-ordered on that stream.
 * - Pointers documented as "device" must be device-accessible memory of the
 *   current CUDA device.  Pointers documented as "host or device" are
 *   classified with cudaPointerGetAttributes; host memory is copied in and out
 *   by the library inside the call.
 * - The caller owns every pointer it passes.  Calls allocate their temporary
 *   workspace from a library-private, stream-ordered memory pool of the
 *   current device (it keeps freed blocks for reuse) and release it before
 *   returning.
 * - Calls return a popcorn_status and never abort the process.  On an error
 *   the outputs are unspecified, nothing is leaked, and
 *   popcorn_last_error_message() describes the error of the calling thread.
 * - k <= 256 (labels are kept as bytes on the device); n < 2^31.
 */
#ifndef POPCORN_H
#define POPCORN_H

#include <stdint.h>

#if defined(__GNUC__)
#define POPCORN_API __attribute__((visibility("default")))
#else
#define POPCORN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* popcorn_stream_t;  /* == cudaStream_t */

typedef enum {
    POPCORN_OK = 0,
    POPCORN_ERR_INVALID = 1,      /* an argument is out of range or inconsistent            */
    POPCORN_ERR_NOMEM = 2,        /* device workspace could not be allocated                */
    POPCORN_ERR_CUDA = 3,         /* a CUDA runtime call or a kernel launch failed          */
    POPCORN_ERR_TIMEOUT = 4,      /* a bounded device-side wait ran out; context still usable */
    POPCORN_ERR_UNSUPPORTED = 5   /* valid request this build does not implement            */
} popcorn_status;

/* Kernel functions of Sec. 3.2 (and the linear kernel K = P P^T). */
typedef enum {
    POPCORN_LINEAR = 0,      /* kappa(x, y) = x . y                              */
    POPCORN_POLYNOMIAL = 1,  /* kappa(x, y) = (gamma x . y + coef0)^degree       */
    POPCORN_GAUSSIAN = 2     /* kappa(x, y) = exp(-gamma ||x - y||^2 / sigma^2)  */
} popcorn_kernel_kind;

typedef struct {
    int32_t kind;    /* popcorn_kernel_kind                                  */
    int32_t degree;  /* polynomial degree r >= 1 (integer)                  */
    double gamma;    /* gamma > 0 (polynomial and Gaussian; 1 if unsure)    */
    double coef0;    /* c (polynomial)                                      */
    double sigma;    /* sigma > 0 (Gaussian)                                */
} popcorn_kernel;

/* Arithmetic used to form B = P P^T for the kernel matrix. */
typedef enum {
    POPCORN_FP32 = 0,    /* FP32 CUDA-core arithmetic; Gaussian distances from coordinate differences */
    POPCORN_BF16 = 1,    /* tcgen05 tensor cores, BF16 operands, FP32 accumulate                       */
    POPCORN_BF16X3 = 2,  /* tcgen05, split-BF16 (hi*hi + hi*lo + lo*hi), FP32 accumulate              */
    POPCORN_FP8 = 3      /* tcgen05, FP8 E4M3 operands with per-row scales s_i = max|p_i| / 448, FP32
                            accumulate; the recompute path (store_k = 0) only                          */
} popcorn_precision;

/* Element type of a stored K (the paper stores FP32). */
typedef enum {
    POPCORN_K_FP32 = 0,
    POPCORN_K_FP16 = 1,   /* half the bytes per pass; values must fit FP16 (e.g. Gaussian K <= 1) */
    POPCORN_K_BF16 = 2    /* half the bytes per pass; FP32 range, 8 significant bits             */
} popcorn_k_storage;

typedef struct {
    int32_t precision;          /* popcorn_precision for the K build                         */
    int32_t store_k;            /* 1: materialize K once (the paper's design)                */
    int32_t check_convergence;  /* 1: stop when a pass changes no label (or on tol); 0: run
                                   exactly max_iter passes (the paper's fixed-iteration mode) */
    int32_t timing;             /* 1: record CUDA-event times per phase and per kernel of every
                                   pass into popcorn_fit_info; 2: per phase only (K build,
                                   passes).  Without per-kernel events (0 or 2), a stored-K fit
                                   in fixed-iteration mode (check_convergence = 0) runs all its
                                   passes and the final objective pass as one CUDA graph,
                                   captured on a private stream and launched on `stream`
                                   (plain launches when `stream` is itself being captured)   */
    int32_t k_storage;          /* popcorn_k_storage of the stored K; 0 = FP32.  FP16 / BF16
                                   from any build, rounded once.  A pass reads it on the tensor
                                   cores: the symmetric pass's tensor-core form (k <= 32), or,
                                   read as the full square (k > 32 or k_pass = 2), 32 KB half
                                   tiles of the square with each 128-row block's row sums as
                                   MMAs against one-hot label operands (any k; for the FP32
                                   build from n = 8192, below which a CUDA-core pass reads a
                                   row-major half K)                                         */
    int32_t autotune;           /* 1: pick the schedule by timing candidates on this workload
                                   (first call per workload signature; later calls reuse the
                                   cached choice, see popcorn_autotune_entries); 0: fixed
                                   heuristics.  Used by popcorn_fit_batched (K-stream unit
                                   length, warps per block, blocks per SM) and by the
                                   recompute path of popcorn_fit (row blocks per tile, units
                                   per SM).  Results differ only by summation order.        */
    int32_t k_pass;             /* how a pass reads a stored K.  0 = automatic (the
                                   default): the symmetric read below for n >= 8192 (where K
                                   outgrows L2 and reading half of it pays; measured faster
                                   on GB300 for every k up to 32), and at every n for an
                                   FP16 / BF16 K from a BF16 / BF16X3 build; else the full
                                   square.
                                   1 = symmetric (k <= 32; larger k falls back to the full
                                   square): only the 128 x 128 blocks on and above the
                                   diagonal (K is symmetric, and is then stored as that packed
                                   triangle; an FP16 / BF16 K is written as half tiles by a
                                   BF16 / BF16X3 build, or rounded from the FP32 build's
                                   triangle by one more launch); a block's row sums serve its
                                   rows and its column sums its columns' rows.  Blocks are
                                   taken in super-tiles of a x a (sym_tile below), largest
                                   first; an FP32 K's pass sorts each block's labels once
                                   (CUDA cores), an FP16 / BF16 K's pass takes each block's
                                   sums as MMAs against one-hot label operands (tensor cores);
                                   each super-tile writes one slot per row it touches, and
                                   the slots are folded, so a pass reads half of K plus about
                                   8 k n ceil(n / 128a) bytes of slots.  2 = the full square,
                                   row by row (the paper's read of K; an FP16 / BF16 K on the
                                   tensor cores as described under k_storage).  The recompute
                                   path has its own scheme.  Results differ only by summation
                                   order                                                     */
    int32_t sym_tile;           /* super-tile edge a of the symmetric pass, in 128-blocks,
                                   0..8: 0 = automatic (4 for k <= 16 and 3 for k <= 32,
                                   narrowed until there are at least 8 super-tiles per SM);
                                   1..8 to force one (6 or 8 for k <= 12 gives each warp two
                                   block rows, FP32 K only; an edge the register file does not
                                   allow falls back to the full square).  k <= 8 with an edge
                                   of 1 and an FP32 K runs the branch form (single blocks, a
                                   uniform branch a label)                                    */
    int64_t reserved[4];        /* must be zero                                              */
} popcorn_options;

/* Optional per-call report of popcorn_fit (all fields written by the call,
   except the two caller-provided history arrays). */
typedef struct {
    double kbuild_ms;          /* K build (norms + kernel matrix), when timing = 1          */
    double loop_ms;            /* all assignment passes, when timing = 1                    */
    double reduce_ms;          /* sum over passes of the K-streaming reduction kernel       */
    double assign_ms;          /* sum over passes of the distance/argmin kernel             */
    double eval_ms;            /* final objective evaluation pass, if one was needed        */
    int32_t reduce_launches;   /* launches of the K-streaming reduction kernel              */
    int32_t assign_launches;   /* launches of the distance/argmin kernel                   */
    int32_t kernel_launches;   /* all kernels this call launched                            */
    int32_t converged;         /* 1 if a pass changed no label                              */
    int64_t h2d_bytes;         /* host->device bytes the call copied                        */
    int64_t d2h_bytes;         /* device->host bytes the call copied                        */
    double* J_history;         /* caller-provided host array of >= max_iter doubles, or NULL:
                                  J_t = J(labels before pass t)                             */
    int32_t* changed_history;  /* caller-provided host array of >= max_iter ints, or NULL:
                                  labels changed by pass t                                  */
    int32_t tune_cache_hit;    /* autotune = 1: the schedule came from the cache            */
    int32_t tune_candidates;   /* autotune = 1: schedules this call timed (0 on a cache hit)  */
    double tune_ms;            /* host wall time this call spent timing candidates           */
    int32_t schedule[4];       /* the schedule used (tuned or heuristic):
                                  batched: {columns per K-stream unit, warps per block,
                                            blocks per SM, 0};
                                  recompute: {row blocks per tile, column segments,
                                              units per SM target, 0};
                                  symmetric pass: {super-tile edge, block ring depth,
                                                   slots, sums per row: 4 or 8 registers
                                                   in the branch form, 12, 16 or 32 in
                                                   the sorted form, 16 or 32 TMEM
                                                   columns (the MMA's N) in the
                                                   tensor-core form};
                                  full square of a half K on the tensor cores: {0, ring
                                                   depth, 0, TMEM columns (k rounded up
                                                   to 16)};
                                  zeros otherwise                                           */
    double fold_ms;            /* symmetric pass: the slot fold kernel, summed over passes
                                  (part of reduce_ms), when timing = 1                      */
    int32_t k_pass_used;       /* stored K: 1 = symmetric pass, 2 = full square, 3 = the whole
                                  fit in one cooperative launch (automatic choice for an FP32
                                  K that sits in L2: n <= 6144, k <= 32; it reads the full
                                  square); 0 recompute                                     */
    int32_t sym_form;          /* k_pass_used = 1: the form of the symmetric pass: 1 branch
                                  (FP32 K, single blocks), 2 sorted (FP32 K, label-sorted
                                  lists, CUDA cores), 3 tensor-core (FP16 / BF16 K: MMAs of
                                  the packed tiles against one-hot label operands); else 0  */
    float* E_out;              /* caller-provided DEVICE array of n x k floats (row-major,
                                  ld = k), or NULL.  Stored-K fits with max_iter >= 1: E =
                                  K V^T of the labels the last assignment pass started
                                  from (the E that pass took its argmin from; with
                                  max_iter = 1 those are init_labels).  Ignored by the
                                  recompute path and by popcorn_fit_batched               */
} popcorn_fit_info;

/* Human-readable name of a status code (static storage). */
POPCORN_API const char* popcorn_status_string(popcorn_status status);

/* Message describing the last error returned on the calling thread (static
   thread-local storage; empty after a successful call). */
POPCORN_API const char* popcorn_last_error_message(void);

/* Version of this library as MAJOR*10000 + MINOR*100 + PATCH. */
POPCORN_API int32_t popcorn_version(void);
/* Allocations the library has made in this process: blocks of its device workspace pool and
 * pinned host staging buffers (a diagnostic; popcorn_assign_step_noalloc never adds to it). */
POPCORN_API int64_t popcorn_allocation_count(void);

/*
 * popcorn_kernel_matrix -- K = kappa(P P^T) and diag(K).
 *
 * Sec. 3.2 (polynomial and Gaussian kernels from B = P P^T, Eq. 12 for the
 * Gaussian) and Alg. 2 lines 1-2 (K once, P~ from diag(K)).  The tile schedule
 * is POPCORN_SCHEDULE_AUTO (see popcorn_kernel_matrix_ex).
 *
 *   P      device, n x d FP32, leading dimension ldp >= d.
 *   K      device, n x n FP32 output, leading dimension ldk >= n; ldk must be
 *          a multiple of 4 and K 16-byte aligned.  The full square is written
 *          (both triangles), symmetric.
 *   kdiag  device, n FP32 output: kdiag[i] = K[i][i] (== 1 for Gaussian).
 *   precision  POPCORN_FP32, POPCORN_BF16 or POPCORN_BF16X3.
 *
 * Errors: POPCORN_ERR_INVALID for n < 1, d < 1, ldp < d, ldk < n, ldk % 4,
 * misaligned K, degree < 1 (polynomial), sigma <= 0 or gamma <= 0 (Gaussian);
 * POPCORN_ERR_UNSUPPORTED for POPCORN_FP8.
 */
POPCORN_API popcorn_status popcorn_kernel_matrix(const float* P, int64_t n, int32_t d, int64_t ldp,
                                     popcorn_kernel kern, int32_t precision,
                                     float* K, int64_t ldk, float* kdiag,
                                     popcorn_stream_t stream);

/* Tile schedule of the K build: which 128 x 128 tiles of B = P P^T are formed.  The
   paper builds B with a GEMM or a SYRK and switches on the shape (Sec. 4.2, n/d
   threshold; Sec. 5.2 measures both). */
typedef enum {
    POPCORN_SCHEDULE_AUTO = 0,       /* the cached tuned choice for this workload signature,
                                        else SYMMETRIC                                        */
    POPCORN_SCHEDULE_SYMMETRIC = 1,  /* the tiles on and above the diagonal, each stored with
                                        its transpose (the SYRK form: n (n + 1) / 2 products) */
    POPCORN_SCHEDULE_FULL = 2,       /* every tile of the square, each stored once (the GEMM
                                        form: n^2 products)                                 */
    POPCORN_SCHEDULE_TUNE = 3        /* time SYMMETRIC and FULL on this call's inputs once per
                                        workload signature (precision, bucketed n and d,
                                        kernel kind, SM count), cache the faster, use it     */
} popcorn_kbuild_schedule;

/*
 * popcorn_kernel_matrix_ex -- popcorn_kernel_matrix with a chosen tile schedule.
 *
 * Sec. 3.2 and Alg. 2 lines 1-2, with the GEMM-or-SYRK choice of Sec. 4.2 made by
 * `schedule` (popcorn_kbuild_schedule) instead of the paper's fixed n/d threshold.
 * Arguments and errors as popcorn_kernel_matrix, plus POPCORN_ERR_INVALID for an
 * unknown schedule.  Under FULL each (i, j) and (j, i) are formed separately: the FP32
 * build gives the same value for both (the same products in the same order); BF16X3
 * adds its three partial products in another order for the transposed tile, so the two
 * may differ in the last bits.  TUNE runs the build several times on the call's stream.
 */
POPCORN_API popcorn_status popcorn_kernel_matrix_ex(const float* P, int64_t n, int32_t d, int64_t ldp,
                                                    popcorn_kernel kern, int32_t precision, int32_t schedule,
                                                    float* K, int64_t ldk, float* kdiag,
                                                    popcorn_stream_t stream);

/*
 * popcorn_assign_step -- one pass of the loop body of Alg. 2 on a given K.
 *
 * From labels cl (Eq. 8 defines V from them): E = K V^T (Alg. 2 line 7,
 * the paper's SpMM), ||c_j||^2 = sum over i in L_j of E_{i,j} / |L_j|
 * (line 8-9, Eq. 14, the paper's SpMV), D = E-term + P~ + C~ (line 10) and
 * new labels = row argmin of D (lines 11-13), ties to the lowest index, an
 * empty cluster never chosen.
 *
 *   K, ldk     device, n x n FP32 (ldk % 4 == 0, 16-byte aligned).
 *   kdiag      device, n FP32: diag(K).
 *   labels     device, n int32 in [0, k): the current assignment.
 *   new_labels device, n int32 output (may alias labels).
 *   counts     device, k int32 output or NULL: |L_j| of the NEW labels.
 *   E          device, n x k FP32 output (row-major, ld = k) or NULL:
 *              E_ij = (K V^T)_ij for the CURRENT labels (0 for empty j).
 *   cnorm      device, k FP64 output or NULL: ||c_j||^2 (0 for empty j).
 *   objective  host, 1 double output or NULL: J(labels) = sum_i D_{i,cl(i)}.
 *   changed    host, 1 int32 output or NULL: number of labels that changed.
 * Host outputs are written after the call synchronizes the stream.
 *
 * Errors: POPCORN_ERR_INVALID for n < 2, k < 1, k > n, k > 256, bad ldk or
 * alignment, or a label outside [0, k) (detected on the device).
 */
POPCORN_API popcorn_status popcorn_assign_step(const float* K, int64_t ldk, const float* kdiag, int64_t n,
                                   int32_t k, const int32_t* labels, int32_t* new_labels,
                                   int32_t* counts, float* E, double* cnorm,
                                   double* objective, int32_t* changed,
                                   popcorn_stream_t stream);

/*
 * popcorn_fit -- Kernel K-means (Alg. 2) from points and initial labels.
 *
 * Builds K once (Alg. 2 lines 1-2), then runs assignment passes (lines 6-15).
 * Pass t computes D from labels cl_t, J_t = J(cl_t) and cl_{t+1} = argmin.
 * Stopping (Alg. 1/2 "while iter < maxiter and centroids are changing"):
 * always after max_iter passes; with opt->check_convergence also after a pass
 * that changes no label, or after a pass t >= 1 with J_{t-1} - J_t <=
 * tol * |J_t| when tol > 0.
 *
 *   P            host or device, n x d FP32, leading dimension ldp >= d.
 *   k            number of clusters, 1 <= k < n, k <= 256.
 *   init_labels  host or device, n int32 in [0, k).
 *   max_iter     >= 0.  0 returns init_labels and their objective.
 *   tol          >= 0, relative objective-decrease threshold (0 = off).
 *   opt          options, or NULL for {FP32, store_k = 1, check_convergence = 1}.
 *   labels_out   host or device, n int32 output (may alias init_labels).
 *   objective_out    host, 1 double: J(labels_out) = sum_i ||phi(p_i) - c_cl(i)||^2.
 *   iterations_out   host, 1 int32: passes performed.
 *   info         host, optional report (NULL allowed).
 *
 * Errors: as popcorn_kernel_matrix, plus POPCORN_ERR_INVALID for k outside
 * [1, n) or > 256, max_iter < 0, tol < 0, labels out of range, nonzero
 * reserved fields; POPCORN_ERR_UNSUPPORTED for store_k = 1 with POPCORN_FP8
 * (FP8 runs on the recompute path only), for store_k = 0 with POPCORN_FP32 or
 * POPCORN_BF16X3 (the recompute path runs in POPCORN_BF16 or POPCORN_FP8), and
 * for a recompute request with d or k beyond its limits (d <= 256 for BF16,
 * d <= 512 for FP8), and for an FP16 / BF16 K from a BF16 / BF16X3 build read
 * as the full square inside a caller's stream capture; POPCORN_ERR_NOMEM when K (or the workspace) does not fit
 * in device memory; POPCORN_ERR_TIMEOUT when a bounded wait inside a
 * tensor-core or symmetric-pass kernel ran out (the context stays usable).
 */
POPCORN_API popcorn_status popcorn_fit(const float* P, int64_t n, int32_t d, int64_t ldp, int32_t k,
                           popcorn_kernel kern, const int32_t* init_labels, int32_t max_iter,
                           double tol, const popcorn_options* opt, int32_t* labels_out,
                           double* objective_out, int32_t* iterations_out,
                           popcorn_fit_info* info, popcorn_stream_t stream);

/* One clustering problem of a batch (all pointers device memory). */
typedef struct {
    const float* P;             /* n x d FP32, leading dimension ldp >= d                  */
    int64_t n;                  /* points, 2 <= n < 2^31                                   */
    int32_t d;                  /* features >= 1                                           */
    int64_t ldp;
    int32_t k;                  /* clusters, 1 <= k < n, k <= 256                          */
    popcorn_kernel kern;        /* each instance has its own kernel function               */
    const int32_t* init_labels; /* n labels in [0, k)                                      */
    int32_t* labels_out;        /* n labels (may alias init_labels)                        */
} popcorn_instance;

/*
 * popcorn_kmeanspp -- K-means++ seeding in the kernel's feature space: k initial centers
 * and the initial labels popcorn_fit can start from.
 *
 * Sec. 2.1 names K-means++ as the initialization that samples each next centroid from a
 * weighted distribution favouring points far from those already chosen.  The weight here
 * is the squared feature-space distance to the nearest chosen point,
 * D(i) = min_c (K_ii - 2 K_ic + K_cc), with kappa evaluated in FP64 from the points (K is
 * not formed).  The caller supplies the random numbers: u[0] picks the first point,
 * floor(u[0] n); for t >= 1, point t is the first i in index order at which the running sum
 * of D exceeds u[t] sum_i D(i) (floor(u[t] n) when that sum is 0, i.e. every point
 * coincides with a chosen one).  labels_out[i] is the index t of i's nearest chosen point
 * (the lowest t on ties).  All sums are taken in a fixed order: repeated calls give the
 * same result.
 *
 *   P           host or device, n x d FP32, leading dimension ldp >= d.
 *   u           host or device, k doubles in [0, 1).
 *   labels_out  host or device, n int32 output (values in [0, k)).
 *   centers_out host or device, k int32 output (the chosen points in order), or NULL.
 *   stream      work is ordered on it; the call returns after the results are written.
 *
 * Errors: POPCORN_ERR_INVALID for null P / u / labels_out, n < 1, d < 1, ldp < d, k outside
 * [1, min(n, 256)], a host draw outside [0, 1), or an invalid kernel; POPCORN_ERR_UNSUPPORTED
 * when the per-SM state (about 20 (n / SMs) + 8 d bytes) exceeds shared memory;
 * POPCORN_ERR_TIMEOUT if a bounded wait between the SMs ran out.
 */
POPCORN_API popcorn_status popcorn_kmeanspp(const float* P, int64_t n, int32_t d, int64_t ldp, int32_t k,
                                            popcorn_kernel kern, const double* u, int32_t* labels_out,
                                            int32_t* centers_out, popcorn_stream_t stream);

/*
 * popcorn_fit_batched -- many independent Kernel K-means problems at once.
 *
 * Each instance runs Alg. 2 exactly as popcorn_fit would, with the shared
 * max_iter, tol and options (store_k must be 1).  The whole batch -- the K
 * builds of all instances, max_iter assignment passes over every instance
 * that has not stopped, the final objective pass -- is captured once into a
 * CUDA graph and launched on `stream`; an instance that converges stops
 * doing work on the device while the others go on.  Instances of uneven n,
 * d, k and kernel share every launch: work is flattened over (instance,
 * tile / row segment / row block).  options.k_storage FP16 / BF16 stores every
 * instance's square as 32 KB half tiles (written by the FP32 build, or rounded
 * from a BF16 / BF16X3 build's FP32 square) and each pass reads them on the
 * tensor cores: per 128-row block, MMAs of its tiles against one-hot label
 * operands, the row sums in TMEM.  k_pass and sym_tile do not apply here (each
 * square is read whole).
 *
 *   instances        host array of `count` descriptors.
 *   objectives_out   host, count doubles: J(labels_out) per instance.
 *   iterations_out   host, count ints: passes per instance.
 *   info             optional; loop_ms (timing = 1) is the graph's time.
 * Errors: as popcorn_fit for each instance (the message names the index).
 */
POPCORN_API popcorn_status popcorn_fit_batched(int32_t count, const popcorn_instance* instances, int32_t max_iter,
                                               double tol, const popcorn_options* opt, double* objectives_out,
                                               int32_t* iterations_out, popcorn_fit_info* info,
                                               popcorn_stream_t stream);

/*
 * popcorn_assign_step_noalloc -- popcorn_assign_step without any allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory, for example a host framework that owns all
 * device memory through its own allocator, or a long-running loop that
 * forbids allocation once it has started.  It computes exactly what
 * popcorn_assign_step computes (same kernels, same launch plan), with the
 * same arguments, layouts and ownership, but it calls no cudaMalloc,
 * cudaFree, pool or pinned-host allocation: its temporary buffers live in one
 * statically allocated device array of POPCORN_NOALLOC_SCRATCH_BYTES bytes.
 *
 *   - Every GPU that loads this library holds that array until the process
 *     exits.
 *   - The first call on a device does a one-time set-up for that device (it
 *     looks up the array's device address and sets kernel attributes); make
 *     that first call before any stream capture.
 *   - A step needs about 4 * k * max(n, ~80,000) + 5 n bytes (grows with the
 *     row segmentation of the K stream).  A request that does not fit returns
 *     POPCORN_ERR_INVALID with the needed and available sizes in
 *     popcorn_last_error_message(); nothing is launched.
 *   - All calls share the array and it keeps the last call's contents (the
 *     call itself clears what must start at zero).  Calls that overlap on
 *     the GPU -- on two streams, or from two host threads -- race on it and
 *     give wrong results: serialize them.
 *
 * Errors: as popcorn_assign_step, plus the size limit above.
 */
/*
 * Autotune cache (options.autotune = 1).
 *
 * The paper has no counterpart: its kernels have fixed launch shapes.  Tuned
 * schedules are kept per workload signature (bucketed sizes, precision, SM
 * count) for the life of the process; if the environment variable
 * POPCORN_TUNE_CACHE names a writable file, entries are appended to it and
 * read back by later processes.  popcorn_autotune_entries returns how many
 * signatures are cached; popcorn_autotune_clear forgets them (the file is not
 * touched).  Both are thread-safe and never fail.
 */
POPCORN_API int32_t popcorn_autotune_entries(void);
POPCORN_API void popcorn_autotune_clear(void);

#define POPCORN_NOALLOC_SCRATCH_BYTES (32ll * 1024 * 1024)

POPCORN_API popcorn_status popcorn_assign_step_noalloc(const float* K, int64_t ldk, const float* kdiag,
                                                       int64_t n, int32_t k, const int32_t* labels,
                                                       int32_t* new_labels, int32_t* counts, float* E,
                                                       double* cnorm, double* objective, int32_t* changed,
                                                       popcorn_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* POPCORN_H */
