/*
 * dcd_gb300.h -- C ABI of the GB300 (sm_103a) s-step dual coordinate descent
 * library: s-step DCD for the kernel SVM duals and s-step block DCD for kernel
 * ridge regression, after "Scalable Dual Coordinate Descent for Kernel
 * Methods" (arXiv 2406.18001).
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers owned by the caller unless the
 *    opts flag DCD_FLAG_HOST_IO says the solve's arrays live in host memory.
 *    The library never frees caller memory.
 *  - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL is
 *    the legacy default stream).  Each call returns only after its work on
 *    that stream has finished, so outputs are ready when it returns.
 *  - Errors come back as a dcd_status, never as an abort or a device trap.
 *    Device-side failures (an index out of range, a bounded wait that ran
 *    out) are recorded in a device error word and turned into a status.
 *  - The library allocates its scratch memory with cudaMallocAsync on
 *    `stream` and frees it before returning.
 *  - All indices are 0-based.  Dense matrices are row-major with leading
 *    dimension ld >= n (elements).  CSR uses int64 row_ptr[m+1] and int32
 *    col_idx[nnz] with values in `dtype`.
 */
#ifndef DCD_GB300_H
#define DCD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DCD_OK = 0,
    DCD_EINVAL = 1,       /* an argument failed validation */
    DCD_ENOMEM = 2,       /* device allocation failed */
    DCD_ECUDA = 3,        /* a CUDA runtime call failed */
    DCD_ETIMEOUT = 4,     /* a bounded device wait ran out (kernel returned early) */
    DCD_ENOTCONV = 5,     /* iteration budget used before reaching opts.tol; alpha is valid */
    DCD_EINTERNAL = 6,    /* a device-side consistency check failed */
    DCD_ENOTSPD = 7,      /* a b x b block system G was not positive definite */
    DCD_EUNSUPPORTED = 8  /* valid request this build does not implement */
} dcd_status;

typedef enum { DCD_DENSE = 0, DCD_CSR = 1 } dcd_format;
typedef enum { DCD_F64 = 0, DCD_F32 = 1, DCD_BF16 = 2, DCD_FP8E4M3 = 3 } dcd_dtype;

/* The data matrix A (m x n), paper Section 3: rows a_i are samples. */
typedef struct {
    int32_t fmt;              /* dcd_format */
    int32_t dtype;            /* dcd_dtype of values */
    int64_t m, n;             /* rows (samples) and columns (features) */
    int64_t ld;               /* dense: leading dimension in elements, >= n */
    const void *values;       /* dense: m*ld elements; CSR: nnz elements */
    const int64_t *row_ptr;   /* CSR only: m+1 offsets, row_ptr[0] = 0, non-decreasing */
    const int32_t *col_idx;   /* CSR only: nnz column indices in [0, n), distinct within a row */
    const float *row_scale;   /* FP8 only: a_i = row_scale[i] * q_i (m finite scales >= 0,
                                 host memory under DCD_FLAG_HOST_IO); else ignored */
} dcd_matrix;
/*
 * FP8 storage (dtype DCD_FP8E4M3, dense only): values holds one OCP e4m3 code
 * per element (sign, 4 exponent bits with bias 7, 3 mantissa bits, largest
 * finite 448, codes 0x7f/0xff NaN) and row i stands for row_scale[i] * q_i.
 * A NaN code or a negative or non-finite scale gives DCD_EINVAL.  Under
 * DCD_PREC_FP8 the codes feed the tensor cores as they are; every other
 * precision dequantises first (exactly for DCD_PREC_FP64).
 */
/*
 * CSR matrices take F32 or F64 values (BF16 / FP8 give DCD_EUNSUPPORTED).
 * Their kernel block is an SpMM on the CUDA cores, streamed once per outer
 * step: FP64 under DCD_PREC_FP64, FP32 under every tensor-core precision
 * (the block is bound by HBM, not arithmetic).  Offsets that decrease or
 * exceed nnz, and columns outside [0, n), give DCD_EINVAL (checked on the
 * device before the solve starts).
 */

/* Kernel functions of Table 1 (Section 3.1). */
typedef enum { DCD_LINEAR = 0, DCD_POLY = 1, DCD_RBF = 2 } dcd_kernel_kind;
typedef struct {
    int32_t kind;    /* dcd_kernel_kind */
    int32_t degree;  /* POLY: (coef0 + a.b)^degree, degree >= 2 */
    double gamma;    /* RBF: exp(-gamma * ||a - b||^2), gamma > 0 (the paper's sigma) */
    double coef0;    /* POLY: coef0 >= 0 */
} dcd_kernel;

/* Arithmetic used for the m x (s*b) kernel block.  The s-step recurrence,
 * the b x b solves and the alpha / gradient accumulation are FP64 in every
 * mode. */
typedef enum {
    DCD_PREC_FP64 = 0,   /* FP64 CUDA-core block, direct RBF distances */
    DCD_PREC_TF32 = 1,   /* tcgen05 kind::tf32 block, FP32 accumulation */
    DCD_PREC_BF16 = 2,   /* tcgen05 kind::f16 (bf16) block, FP32 accumulation */
    DCD_PREC_FP8 = 3,    /* tcgen05 kind::f8f6f4 block on e4m3 codes with per-row scales (the
                            FP8 storage below), FP32 accumulation; the epilogue scales each
                            dot by s_i s_j.  A non-FP8 dense A is quantised first as
                            dcd_quantize_e4m3 does.  Dense A only (CSR: DCD_EUNSUPPORTED) */
    DCD_PREC_BF16X3 = 4, /* split bf16: a = hi + lo, three tcgen05 kind::f16 MMAs per
                            k-step (hi.hi + hi.lo + lo.hi), FP32 accumulation */
    DCD_PREC_TF32X3 = 5, /* split tf32 (both halves on the tf32 grid, ~22 significant bits),
                            three kind::tf32 MMAs per k-step, FP32 accumulation */
    DCD_PREC_FP16 = 7,   /* fp16: each row scaled by a power of two so that its largest magnitude lies
                            in [2^14, 2^15), rounded to fp16 (11 significant bits, against bf16's 8);
                            one tcgen05 kind::f16 MMA per k-step, FP32 accumulation; the epilogue
                            scales each dot back by s_i s_j (exact: powers of two) */
    DCD_PREC_REFRESH = 6 /* the arithmetic of the gradient recomputed under DCD_FLAG_REFRESH (every
                            tensor-core mode): each row scaled by a power of two and cut into four
                            bf16 planes of integers in [-64, 64] (27 bits of the row's largest
                            entry); the 10 plane products of order <= 3 are summed in FP32 tensor
                            memory, where their sums are exact integers for n <= 1024 (beyond:
                            split tf32 products); the RBF exponent and kernel value in
                            double-single arithmetic (exp2 by reduction to the nearest integer and
                            a degree-7 Taylor polynomial), and the contraction with the FP64
                            coefficients in double-single.  dcd_kernel_block_apply only
                            (elsewhere DCD_EUNSUPPORTED) */
} dcd_precision;

/* opts.flags */
#define DCD_FLAG_GRAD_VALID 0x1   /* `grad` holds the gradient of `alpha` on entry */
#define DCD_FLAG_HOST_IO 0x2      /* A.values/row_ptr/col_idx, y, alpha, grad are host memory */
#define DCD_FLAG_PHASE_TIMERS 0x4 /* fill the per-phase times of dcd_stats (adds one sync per step) */
#define DCD_FLAG_NO_GRAPH 0x8     /* launch every kernel directly instead of replaying CUDA graphs */
#define DCD_FLAG_LITERAL 0x20     /* run every outer step in the order Algorithms 2 and 4 print: the m x sb
                                     block U_k / Q_k is stored in device memory, U_j^T alpha_sk is formed
                                     from it and the Gram is its rows at the sample (G_k = V_k^T U_k); no
                                     gradient is cached between steps (grad, when given, is recomputed at
                                     the end).  The verification and byte-comparison form of the fused
                                     step: it moves the m x sb block through memory twice.  Dense data
                                     matrices only; requires tol = 0 (else DCD_EINVAL) */
#define DCD_FLAG_CSR_FULL_PASS 0x40 /* CSR data matrix: stream every nonzero in each step's kernel block (the
                                       paper's SpMM) even where the apply through the transposed copy would
                                       read less; both give the same bits (for comparison and testing) */
#define DCD_FLAG_NO_DEFER 0x80  /* steps with the look-ahead (a stream of the caller's, graphs allowed, no
                                   phase timers) of tensor-core K-RR, and of K-SVM with s <= 128: run each
                                   step's recurrence after the previous step's block and update, which it
                                   then overlaps no longer.  By default the recurrence
                                   of step k+1 runs beside the block of step k, on the gradient (K-SVM: and
                                   alpha) before that block plus the block's part at the rows step k+1
                                   samples (an s b x s b product) and the update's: the same sums up to
                                   their association, so the bits differ from the in-order steps by
                                   rounding only.  With this flag the steps give the bits of the one-stream
                                   steps */
#define DCD_FLAG_REFRESH 0x10     /* with tol > 0: when the metric of the cached gradient first meets tol,
                                     recompute the gradient from alpha by full kernel passes (tensor-core
                                     modes: DCD_PREC_REFRESH; FP64 mode: FP64) and accept convergence only
                                     if the recomputed metric meets tol too; the check at the end of the
                                     budget always recomputes */

typedef struct {
    int32_t s;            /* inner steps per outer step, s >= 1 (Algorithms 2 and 4) */
    int32_t b;            /* block size, 1 <= b <= min(m, 128); DCD requires b = 1 */
    int64_t max_iters;    /* H: coordinate updates (DCD) or block updates (BDCD), >= 0 */
    uint64_t seed;        /* index-stream seed */
    uint64_t start_iter;  /* stream position of the first inner iteration (resume) */
    double tol;           /* stop once the relative duality gap (K-SVM) or relative
                             residual ||g||/||y|| (K-RR) is <= tol; 0 runs all H */
    int32_t check_every;  /* outer steps between convergence checks (0: only at the end) */
    int32_t prec;         /* dcd_precision */
    int32_t flags;        /* DCD_FLAG_* */
    int32_t reserved;
} dcd_opts;

typedef struct {
    int64_t iters_done;       /* inner iterations performed */
    int64_t outer_steps;      /* outer s-steps performed */
    int32_t converged;        /* 1 if the tolerance was met */
    int32_t gpu_launches_per_step; /* kernels one outer step launches */
    double final_metric;      /* relative gap (K-SVM) or relative residual (K-RR); NaN after a
                                 dcd_plan_run that neither reached a check point nor the budget end */
    double primal, dual;      /* K-SVM: P and D at the final alpha (from the cached gradient) */
    double ms_total;          /* wall time of the call, device-timed */
    double ms_setup, ms_sample, ms_gram, ms_recur, ms_block, ms_update, ms_check;
    int64_t refreshes;        /* gradient recomputations (DCD_FLAG_REFRESH) */
    double ms_refresh;        /* their device time */
    int64_t s_used;           /* inner steps per outer step of this solve (batched: the autotuner's) */
} dcd_stats;

/*
 * s-step DCD for the kernel SVM dual (Algorithm 2; s = 1 is Algorithm 1).
 *   min_a 1/2 a^T Q a - 1^T a [+ ||a||^2/(4C) for loss 2],  Q = diag(y) K diag(y),
 *   0 <= a_i <= C (loss 1, hinge) or a_i >= 0 (loss 2, squared hinge).
 * y: m labels, each +1 or -1.  alpha: m values, alpha_0 in, alpha_H out.
 * grad: NULL, or m values of g = Q a - 1 + omega a (omega = 1/(2C) for loss 2,
 * else 0): input when DCD_FLAG_GRAD_VALID, always written on return (with
 * device io the solver keeps its cached gradient in this array).
 * Iteration t of the index stream uses coordinate floor(u_t * m / 2^64) with
 * u_t the SplitMix64 draw (seed, stream 0, counter t).
 * Returns DCD_EINVAL for b != 1, C <= 0, labels not +-1, bad kernel
 * parameters or shapes.  st may be NULL.
 */
dcd_status dcd_svm_solve(const dcd_matrix *A, const double *y, const dcd_kernel *k, int32_t loss,
                         double C, const dcd_opts *o, double *alpha, double *grad, dcd_stats *st,
                         void *stream);

/*
 * s-step block DCD for kernel ridge regression (Algorithm 4; s = 1 is
 * Algorithm 3), eq. (krr-problem):
 *   min_a 1/2 a^T (K/lambda + m I) a - y^T a.
 * Block t of the index stream is a b-subset of [0, m) drawn by Floyd's
 * algorithm from SplitMix64 stream t+1.  grad: NULL or m values of
 * g = (K/lambda + m I) a - y, as for dcd_svm_solve.  lambda > 0.
 */
dcd_status bdcd_krr_solve(const dcd_matrix *A, const double *y, const dcd_kernel *k, double lambda,
                          const dcd_opts *o, double *alpha, double *grad, dcd_stats *st, void *stream);

/*
 * Persistent solves ("plans").  A plan validates the arguments, allocates the
 * workspace, packs A and initialises the cached gradient once; dcd_plan_run
 * then continues the same iteration for up to max_outer_steps outer steps
 * (all remaining when < 0) and can be called repeatedly -- running a budget
 * of H in pieces gives bit-identical iterates to one call.  alpha is updated
 * in place (device io) or copied back to the caller's host array after every
 * dcd_plan_run (DCD_FLAG_HOST_IO); grad, when non-NULL, likewise receives the
 * cached gradient.  A, y, alpha and grad must stay valid until
 * dcd_plan_destroy, which frees the workspace (stream-ordered) and
 * synchronises the stream.  st receives cumulative statistics.
 * dcd_plan_run returns DCD_ENOTCONV only once the budget H is exhausted with
 * opts.tol > 0 not reached.  The solve entry points above are create + run
 * all + destroy.
 */
typedef struct dcd_plan dcd_plan;
dcd_status dcd_svm_plan_create(const dcd_matrix *A, const double *y, const dcd_kernel *k, int32_t loss, double C,
                               const dcd_opts *o, double *alpha, double *grad, void *stream, dcd_plan **plan);
dcd_status bdcd_krr_plan_create(const dcd_matrix *A, const double *y, const dcd_kernel *k, double lambda,
                                const dcd_opts *o, double *alpha, double *grad, void *stream, dcd_plan **plan);
dcd_status dcd_plan_run(dcd_plan *plan, int64_t max_outer_steps, dcd_stats *st);
dcd_status dcd_plan_destroy(dcd_plan *plan);

/*
 * Asynchronous continuation: enqueues up to outer_steps (>= 0) further outer
 * steps of the plan on its stream and returns without synchronising the
 * host.  No convergence check runs, alpha / grad are not published and no
 * per-phase times are recorded; the next dcd_plan_run (which may be asked for
 * 0 steps) reports any device-side error, publishes and fills the
 * statistics.  *enqueued (may be NULL) receives the number of steps
 * enqueued, fewer than asked once the budget H is exhausted.  Full outer
 * steps are replayed from a CUDA graph unless DCD_FLAG_NO_GRAPH is set or
 * the plan's stream is the legacy default stream.  Returns DCD_EINVAL for a
 * NULL plan or outer_steps < 0, DCD_ECUDA if a launch fails.
 */
dcd_status dcd_plan_enqueue(dcd_plan *plan, int64_t outer_steps, int64_t *enqueued);

/*
 * Batched K-RR (many independent s-step BDCD solves, e.g. a sweep over sigma
 * and lambda or cross-validation folds).  Every problem is a full solve of
 * its own (its own A, y, kernel, lambda, b, s, budget, seed; the results
 * equal those of bdcd_krr_solve with the same arguments); the batch runs
 * them together: one plan per problem spread over `streams` worker streams,
 * `rounds_per_graph` outer steps of every active problem captured into one
 * CUDA graph (fork/join over the streams) and replayed, the graph rebuilt
 * only when the set of active problems or their step lengths change.
 * Convergence (tol > 0) is checked every check_every rounds for all active
 * problems with one synchronisation; converged problems leave the graph.
 * A problem with s <= 0 takes the s the autotuner measures fastest for its
 * (m, b) (dcd_krr_autotune_s; one measurement per bucket of m within a
 * factor of 2 and b).  st[i] (may be NULL) receives problem i's statistics.
 * Returns the first failing problem's status.
 */
typedef struct {
    dcd_matrix A;             /* dense or CSR, device arrays */
    const double *y;          /* m targets (device) */
    dcd_kernel k;
    double lambda;            /* > 0 */
    int32_t b;                /* block size */
    int32_t s;                /* inner steps per outer step; <= 0: autotuned */
    int64_t max_iters;        /* H block updates */
    uint64_t seed;
    double *alpha;            /* m (device): alpha_0 in, result out */
    double *grad;             /* NULL or m (device): gradient out */
} dcd_krr_problem;

typedef struct {
    int32_t prec;             /* dcd_precision of every solve */
    int32_t streams;          /* worker streams (0: 16) */
    int32_t rounds_per_graph; /* outer steps per problem in one graph replay (0: 8) */
    int32_t check_every;      /* graph replays between convergence checks (0: only at the end) */
    double tol;               /* as dcd_opts.tol */
    int32_t flags;            /* DCD_FLAG_REFRESH, DCD_FLAG_NO_GRAPH */
    int32_t reserved;
} dcd_batch_opts;

dcd_status bdcd_krr_solve_batched(const dcd_krr_problem *probs, int32_t count, const dcd_batch_opts *o,
                                  dcd_stats *st, void *stream);

/*
 * The autotuner: times a few outer steps of each candidate s in {1, 2, 4,
 * ..., 128} with s*b <= 8192 on this problem (alpha = 0, a scratch copy) and
 * returns the fastest per block update in *s_out (ties to the smaller s).
 */
dcd_status dcd_krr_autotune_s(const dcd_matrix *A, const double *y, const dcd_kernel *k, double lambda, int32_t b,
                              int32_t prec, int32_t *s_out, void *stream);

/* Human-readable name of a status code (static string). */
const char *dcd_status_string(int32_t status);

/*
 * Component entry points (one hot-path step each; used for testing and
 * measurement).
 *
 * dcd_sample_indices -- step "sample" of Algorithms 2 and 4.
 *   method 0 (DCD): out[j] = coordinate of iteration first+j, j < count.
 *   method 1 (BDCD): out[j*b + q], q < b, = block first+j, j < count.
 *   out: device int32, count (method 0) or count*b (method 1) entries.
 */
dcd_status dcd_sample_indices(int32_t method, uint64_t seed, int64_t m, int32_t b, uint64_t first,
                              int64_t count, int32_t *out, void *stream);

/*
 * dcd_kernel_block -- the sampled kernel block U_k / Q_k of Algorithms 2 and
 * 4: out[r*ldo + c] = K(a_rows[r], a_cols[c]) for r < nrows, c < ncols.
 *   rows: device int32 indices, or NULL for rows 0..nrows-1.
 *   cols: device int32 indices.  out: device float (prec != FP64) or double
 *   (prec == FP64), ldo >= ncols.  Dense A only.
 */
dcd_status dcd_kernel_block(const dcd_matrix *A, const dcd_kernel *k, int32_t prec, const int32_t *rows,
                            int64_t nrows, const int32_t *cols, int64_t ncols, void *out, int64_t ldo,
                            void *stream);

/*
 * dcd_kernel_block_apply -- the fused "kernel block times coefficients"
 * update that closes every outer step (the gradient form of the alpha update
 * in Algorithms 2 and 4), without storing the block:
 *   g[i] += rowscale[i] * sum_{c < ncols} K(a_i, a_cols[c]) * w[c],  0 <= i < m.
 *   cols: device int32 (ncols entries); w: device double; rowscale: device
 *   double or NULL (= 1); g: device double, m entries, updated in place.
 */
dcd_status dcd_kernel_block_apply(const dcd_matrix *A, const dcd_kernel *k, int32_t prec,
                                  const int32_t *cols, int64_t ncols, const double *w,
                                  const double *rowscale, double *g, void *stream);

/*
 * dcd_kernel_block_static -- dcd_kernel_block (same arguments, layout, output
 * and error codes) without any device memory allocation.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate
 * device memory at the moment they need a kernel block: a framework that has
 * reserved the device memory for its own caching pool (an extra cudaMalloc
 * can fail there, or force the pool to give back cached blocks), or a
 * deployment whose policy forbids dynamic device allocation after start-up
 * (cudaMalloc / cudaFree may also synchronise the device).
 *
 * Its scratch is one library-owned device array of DCD_STATIC_SCRATCH_BYTES
 * per GPU, held from the first call on that GPU (below) until the process
 * exits.  A call needs 256 bytes plus
 *   tensor-core precisions: (nrows + ncols) * R + 4 * nrows + 4 * roundup(ncols, 256)
 *     with R = 2 * n_pad (bf16), 4 * n_pad (tf32 or bf16x3), n_pad = n rounded up
 *     to 64 (bf16, bf16x3) or 32 (tf32), plus alignment padding;
 *   FP64 with a non-FP64 A: 8 * m * n;  FP64 with an FP64 A: nothing more.
 * A request needing more than DCD_STATIC_SCRATCH_BYTES returns DCD_EINVAL
 * before any device work is enqueued.
 *
 * The first call made on a device (with that device current) looks up the
 * array's device address once; the CUDA runtime may load the array's module
 * and commit its memory only then (lazy module loading).  A caller that must
 * not allocate later therefore makes one call at start-up -- an empty request
 * (nrows or ncols 0) does it -- before its own pool reserves the device
 * memory and before any stream capture begins.  The address is kept for the
 * device's primary context (the one the CUDA runtime and PyTorch use): it is
 * not valid under another driver context or after cudaDeviceReset.  Every
 * call reuses the same array and clears the parts that must start at zero;
 * calls whose device work overlaps (different streams, or different host
 * threads) race on the array and corrupt each other's output.
 *
 * Arguments are checked as dcd_kernel_block checks them.  Two valid requests
 * that dcd_kernel_block serves give DCD_EUNSUPPORTED here: a CSR data matrix
 * (its column map is sized per call) and FP8 (DCD_PREC_FP8, or FP8 storage).
 * DCD_PREC_FP16 (per-row scales beside the packed rows) gives DCD_EUNSUPPORTED
 * too.
 */
#define DCD_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
dcd_status dcd_kernel_block_static(const dcd_matrix *A, const dcd_kernel *k, int32_t prec, const int32_t *rows,
                                   int64_t nrows, const int32_t *cols, int64_t ncols, void *out, int64_t ldo,
                                   void *stream);

/*
 * dcd_quantize_e4m3 -- per-row FP8 storage of a dense matrix (the FP8 form
 * of the data matrix; the paper computes in FP64 and has no counterpart):
 *   row i is first rounded to FP32; row_scale[i] = fl32(max_k |a_ik| / 448);
 *   q[i*ldq + k] = e4m3 code of fl32(a_ik / row_scale[i]) (IEEE FP32
 *   division, round to nearest even, saturating at +-448; a value that rounds
 *   to zero keeps its sign); a row of zeros gets row_scale 0 and zero codes.
 *   Columns n..ldq-1 of q are set to 0.
 *   A: dense F64/F32/BF16 on the device.  q: device, m*ldq bytes, ldq >= n.
 *   row_scale: device, m floats.  Both are caller-owned.
 * A non-finite value gives DCD_EINVAL (q and row_scale are then unspecified).
 */
dcd_status dcd_quantize_e4m3(const dcd_matrix *A, uint8_t *q, int64_t ldq, float *row_scale, void *stream);

/*
 * Row-sharded outer step (components).  Rows are split over ranks: a rank
 * holds rows [row0, row0 + m_local) of A, y, alpha and g (global indices;
 * m = the total row count).  One outer step of Algorithms 2 / 4 then takes
 * one exchange, of s*b*(n + 4) words per rank, where the paper's 1D-column
 * layout reduces an m x s*b block (Section 4, Theorem 2):
 *   1. every rank draws the same S (dcd_sample_indices);
 *   2. dcd_shard_contribute, then an all-gather of the buffers (caller's
 *      transport), then dcd_shard_assemble: A_S, g_S, alpha_S, y_S on every
 *      rank;
 *   3. the sampled Gram of A_S (dcd_kernel_block on the matrix A_S with
 *      rows = cols = first_pos from dcd_shard_assemble) and the recurrence (dcd_bdcd_recurrence /
 *      dcd_dcd_recurrence), redundantly on every rank, as the paper's ranks
 *      repeat the recurrence;
 *   4. dcd_kernel_block_apply_points on the rank's own rows against A_S,
 *      then dcd_shard_update.
 * Buffers are device memory owned by the caller; every call synchronises the
 * stream before it returns.
 *
 * dcd_shard_contribute -- buf (cnt x (n + 4) doubles): for position j whose
 *   row S[j] lies in this rank's range, [1, g[r], alpha[r], y[r], a_r (n
 *   values in FP64, exact from F32 / BF16)] with r = S[j] - row0; zeros for
 *   every other position.  A: the rank's rows (dense F64 / F32 / BF16;
 *   FP8 gives DCD_EUNSUPPORTED).  y may be NULL (0 written).  An S entry
 *   outside [0, m) gives DCD_EINVAL.  cnt <= 8192.
 *
 * dcd_shard_assemble -- bufs: nranks contribution buffers one after another
 *   (the all-gather's output).  For every position, exactly one buffer must
 *   hold the row (else DCD_EINVAL); A_S (cnt x n, row-major FP64), g_S,
 *   alpha_S and y_S (y_S may be NULL) receive it.  first_pos (optional,
 *   needs S): first_pos[j] = the first position q with S[q] == S[j]; as the
 *   rows and cols of dcd_kernel_block on the matrix A_S it gives the sampled
 *   Gram with the ids of the single-GPU step (a repeated row is its own
 *   sample).
 *
 * dcd_bdcd_recurrence -- the K-RR recurrence of Algorithm 4 on gathered
 *   values (eq. bdcd-sstep): Kss the sampled kernel block K(A_S, A_S)
 *   (FP64 when kss_f64, else FP32; leading dimension ldk >= nblk*b), S the
 *   sampled row ids (repeats across the nblk blocks of b are allowed and
 *   handled), g_S[p] = g[S[p]].  The Gram is Kss / lambda + mdiag * [S_p ==
 *   S_q] (mdiag = m).  Output: delta[p] (the change of alpha at position p)
 *   and, when w is non-NULL, w[p] = delta[p] / lambda (the coefficients of
 *   the kernel-block update).  FP64 arithmetic throughout; an FP64 Kss gets
 *   the adaptive refinement of the FP64 solve, an FP32 one a refined FP32
 *   factorisation.  A non-positive-definite diagonal block gives DCD_ENOTSPD.
 *
 * dcd_dcd_recurrence -- the K-SVM recurrence of Algorithm 2 on gathered
 *   values: Kss the sampled kernel block (raw kernel values), S the sampled
 *   row ids (repeats allowed), y_S / alpha_S / g_S the values at them, loss 1
 *   (hinge: omega = 0, nu = C) or 2 (squared hinge: omega = 1/(2C), nu =
 *   infinity).  Output: theta[p] and, when w is non-NULL, w[p] = y_S[p] *
 *   theta[p].  cnt <= 8192.
 *
 * dcd_kernel_block_apply_points -- dcd_kernel_block_apply with the column
 *   points given as the rows of a matrix P (dense, P->n == A->n) instead of
 *   indices into A:
 *     g[i] += rowscale[i] * sum_{c < P->m} K(a_i, p_c) * w[c],  i < A->m.
 *   In the tensor-core precisions the squared distance of a row to itself is
 *   taken as exactly 0 (as in the single-GPU step); "itself" compares ids:
 *   row_id0 + i for row i of A, col_ids[c] for row c of P (col_ids NULL: no
 *   row matches).  FP8 storage or precision gives DCD_EUNSUPPORTED.
 *
 * dcd_shard_update -- the alpha / g update (a6) restricted to this rank's
 *   rows: for each distinct S entry in [row0, row0 + m_local), the delta of
 *   all its positions summed in position order, alpha[r] += sum, g[r] +=
 *   diag * sum (diag: m for K-RR, omega for K-SVM).  Other entries are
 *   skipped.
 */
dcd_status dcd_shard_contribute(const dcd_matrix *A, int64_t row0, int64_t m, const int32_t *S, int64_t cnt,
                                const double *g, const double *alpha, const double *y, double *buf, void *stream);
dcd_status dcd_shard_assemble(const double *bufs, int32_t nranks, const int32_t *S, int64_t cnt, int64_t n,
                              double *A_S, double *g_S, double *alpha_S, double *y_S, int32_t *first_pos,
                              void *stream);
dcd_status dcd_bdcd_recurrence(const void *Kss, int32_t kss_f64, int64_t ldk, const int32_t *S, int64_t nblk,
                               int32_t b, double lambda, double mdiag, const double *g_S, double *delta, double *w,
                               void *stream);
dcd_status dcd_dcd_recurrence(const void *Kss, int32_t kss_f64, int64_t ldk, const int32_t *S, int64_t cnt,
                              const double *y_S, const double *alpha_S, const double *g_S, int32_t loss, double C,
                              double *theta, double *w, void *stream);
dcd_status dcd_kernel_block_apply_points(const dcd_matrix *A, int64_t row_id0, const dcd_matrix *P,
                                         const int32_t *col_ids, const dcd_kernel *k, int32_t prec, const double *w,
                                         const double *rowscale, double *g, void *stream);
dcd_status dcd_shard_update(const int32_t *S, const double *delta, int64_t cnt, double diag, int64_t row0,
                            int64_t m_local, double *alpha, double *g, void *stream);

/*
 * Failure-path hooks (the paper has no counterpart; for testing how failures
 * are reported without faulting, trapping or hanging a GPU).
 *
 * dcd_selftest_bounded_wait -- runs the library's bounded device wait for
 *   real: one thread waits on an mbarrier whose arrival count is never
 *   reached, giving up after about limit_ns nanoseconds (1e3 <= limit_ns <=
 *   1e9, else DCD_EINVAL); the kernel then records the timeout and returns.
 *   Returns DCD_ETIMEOUT (the expected result), DCD_ENOMEM / DCD_ECUDA on a
 *   runtime failure.  The stream is usable afterwards.
 *
 * dcd_inject_alloc_failures -- the next `count` (>= 0) device allocations the
 *   library makes fail as if the device had no memory left, so the call that
 *   makes them returns DCD_ENOMEM; 0 clears the injection.
 */
dcd_status dcd_selftest_bounded_wait(int64_t limit_ns, void *stream);
dcd_status dcd_inject_alloc_failures(int32_t count);

#ifdef __cplusplus
}
#endif
#endif /* DCD_GB300_H */
