// dcd_internal.cuh -- device helpers and host launch declarations shared by
// the translation units of libdcd_gb300.so.  Nothing here is visible through
// the C ABI (include/dcd_gb300.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/dcd_gb300.h"

namespace dcd {

// ---------------------------------------------------------------- errors --
// Device error word codes (first writer wins).
enum DevErr : int {
    DEV_OK = 0,
    DEV_TIMEOUT = 1,     // an mbarrier / flag wait ran past its bound
    DEV_BAD_INDEX = 2,   // a sampled or CSR index fell outside [0, m) / [0, n)
    DEV_NOT_SPD = 3,     // a block system had a non-positive pivot
    DEV_INTERNAL = 4,
    DEV_BAD_VALUE = 5,   // a non-finite data value, FP8 code or row scale
};

__device__ __forceinline__ void set_error(int *err, int code)
{
    if (err) atomicCAS(err, 0, code);
}

// ------------------------------------------------------------ SplitMix64 --
// Steele, Lea & Flood (OOPSLA 2014): the state advances by the golden-ratio
// increment and each output is the 64-bit finaliser of the new state.
// draw(seed, stream, c) is output c+1 of the sequence whose starting state is
// output 2*stream+1 of the sequence seeded with `seed`; stream 0 feeds DCD and
// stream t+1 feeds BDCD block t.
__host__ __device__ __forceinline__ uint64_t sm64_finalise(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t sm64_output(uint64_t state, uint64_t k)
{
    return sm64_finalise(state + k * 0x9E3779B97F4A7C15ULL);
}

__host__ __device__ __forceinline__ uint64_t sm64_draw(uint64_t seed, uint64_t stream, uint64_t ctr)
{
    return sm64_output(sm64_output(seed, 2 * stream + 1), ctr + 1);
}

// floor(u * range / 2^64)
__device__ __forceinline__ uint64_t below(uint64_t u, uint64_t range) { return __umul64hi(u, range); }

// ------------------------------------------------------ kernel functions --
struct KernelParams {
    int kind;       // DCD_LINEAR / DCD_POLY / DCD_RBF
    int degree;
    double gamma;
    double coef0;
};

// Table 1 applied to a dot product (linear, poly) or to a squared distance
// (RBF), in FP64.
__device__ __forceinline__ double kfun_f64(const KernelParams &kp, double v)
{
    if (kp.kind == DCD_RBF) return exp(-kp.gamma * v);
    if (kp.kind == DCD_LINEAR) return v;
    double t = kp.coef0 + v, r = t;
    for (int e = 1; e < kp.degree; ++e) r *= t;
    return r;
}

// ------------------------------------------------- argument validation --
// The checks every entry point applies to a data matrix and a kernel
// (solver.cu): DCD_OK, DCD_EINVAL, or DCD_EUNSUPPORTED for a valid request
// the build does not implement (CSR with BF16 / FP8 values).
dcd_status validate_kernel(const dcd_kernel *k);
dcd_status validate_dense(const dcd_matrix *A);

// Every device allocation of the library (selftest.cu): cudaMallocAsync, or a
// failure injected by dcd_inject_alloc_failures.
cudaError_t malloc_async(void **p, size_t bytes, cudaStream_t st);

// --------------------------------------------------------- host launches --
// All launchers enqueue on `st` and return cudaGetLastError().
// ctr_next (optional, not ctr_dev): receives the stream position after this
// sample, *ctr_dev + first_host + count.
cudaError_t launch_sample(int method, uint64_t seed, const uint64_t *ctr_dev, uint64_t first_host,
                          int64_t m, int b, int64_t count, int32_t *out, int *err, cudaStream_t st,
                          uint64_t *ctr_next = nullptr);

// FP64 CUDA-core kernel block over a dense matrix of doubles.
//   apply (out == nullptr): g[i] += rs[i] * sum_c K(a_i, a_cols[c]) * w[c] for i < nrows
//   store (g == nullptr):   out[r*ldo + c] = K(a_rows[r], a_cols[c])
// Column points: rows cols[c] (cols == nullptr: row c) of B (B == nullptr: of A).
cudaError_t launch_block_simt_f64(const double *A, int64_t lda, int64_t m, int64_t n, const KernelParams &kp,
                                  const int32_t *rows, int64_t nrows, const int32_t *cols, int64_t ncols,
                                  const double *w, const double *rs, double *g, double *out, int64_t ldo,
                                  int *err, cudaStream_t st, const double *B = nullptr, int64_t ldb = 0,
                                  int64_t mb = 0);

// tcgen05 kernel block over the packed, padded operand copy (bf16 or fp32
// rows of n_pad elements, zero padded).
// Packed operand modes (also the pack kernel's dst_kind):
//   0 bf16 rows of n_pad; 1 fp32 rows of n_pad rounded to tf32;
//   3 split bf16 rows of 2*n_pad = [hi | lo].   (dst_kind 2 = fp64, FP64 path)
// Packed operand kinds.  Split kinds keep a = hi + lo as two planes per row
// ([hi | lo], n_pad elements each): bf16x3 with hi = bf16(a), lo = bf16(a -
// hi) (~16 significant bits), tf32x3 with both planes on the tf32 grid (~22
// bits).
// fp8: e4m3 codes (one byte per feature) of the per-row-scaled storage
// a_i ~ scale_i * q_i; the scales travel beside the packed rows.
// sliced: every row scaled by a power of two sc_i = 2^e_i with max |a_ik| < sc_i and cut into 4
// planes of integers in [-64, 64] (exact in bf16), a_ik ~ sc_i (s0 2^-6 + s1 2^-13 + s2 2^-20 +
// s3 2^-27); the per-row scales travel beside the rows like FP8 scales.  The products of two
// such rows are exact integers, and their FP32-accumulated sums stay exact for n_pad <= 1024.
// fp16: the matrix scaled by one power of two sc with max |a_ik| / sc in [2^14, 2^15) and
// rounded to fp16 (11 significant bits), a_ik ~ sc q_ik; sc travels as a per-row scale array
// holding the same value for every row (the block's epilogue reads one row's and one column's).
enum PackKind : int {
    PACK_BF16 = 0, PACK_TF32 = 1, PACK_F64 = 2, PACK_BF16X3 = 3, PACK_TF32X3 = 4, PACK_FP8 = 5, PACK_SLICED = 6,
    PACK_FP16 = 7
};
constexpr int64_t SLICED_N_MAX = 1024;  // exact slice-product sums up to this many features
struct TcOperand {
    const void *rows;     // packed matrix, row-major
    int64_t nrows;
    int64_t n_pad;        // features per half, multiple of the k-block
    int kind;             // PACK_BF16, PACK_TF32, PACK_BF16X3, PACK_TF32X3, PACK_FP8, PACK_SLICED or PACK_FP16
    const float *scale = nullptr;  // PACK_FP8, PACK_SLICED, PACK_FP16: per-row scales (padded with zeros)
    // the data-matrix row each packed row holds (nrows entries; nullptr: row r holds row r).
    // The RBF kernel of a row with itself is 1: where the ids of a block's row and column
    // are equal the epilogues take d^2 = 0 instead of the expansion, whose cancellation
    // there leaves the FP32-accumulated dot's error (a bias of up to ~1e-5 in K_ii)
    const int32_t *ids = nullptr;
};
// elements per 128-byte k-block of a packed row (the padding unit of n_pad)
__host__ __device__ inline int k_block_elems(int kind)
{
    return (kind == PACK_TF32 || kind == PACK_TF32X3) ? 32 : kind == PACK_FP8 ? 128 : 64;
}

__host__ __device__ inline int64_t packed_row_bytes(int kind, int64_t n_pad)
{
    return (kind == PACK_TF32X3 || kind == PACK_SLICED) ? 8 * n_pad
           : (kind == PACK_TF32 || kind == PACK_BF16X3) ? 4 * n_pad
           : kind == PACK_FP8                           ? n_pad
                                                        : 2 * n_pad;
}
bool tc_available();
// lower (store form only): write only the N-chunks that reach the diagonal
// (column chunk start <= last row of the tile); the rest of out is left as is
//
// pdl (apply form): launch as a programmatic dependent of the kernel before
// it on st; the products start at once, the epilogue waits for that kernel
// to finish before it reads col_w or g (the kernel before must not write
// anything else this launch reads).  max_pairs > 0 caps the CTA pairs of
// the apply form (to leave SMs to a kernel running beside it), or the CTAs
// of the store form (which then takes N-chunks of up to 256 columns).
//
// Apply form: the CTA pairs split the (row tile, N-chunk) units into equal
// contiguous ranges when a TcSplit scratch is given (a row tile may then be
// shared by two pairs; the one finishing last adds the per-chunk sums of
// both), else each pair takes whole row tiles round-robin.  Both orders
// give the same bits: every row sum is formed from per-chunk partial sums
// added in chunk order.
struct TcSplit {
    double *part = nullptr;    // tc_split_part_elems(pairs, chunks) doubles
    unsigned *cnt = nullptr;   // 2 * pairs counters, zero before the first launch (left at zero)
    int pairs = 0;             // capacity: CTA pairs
    int chunks = 0;            // capacity: N-chunks of 256 columns
    // the last late_pairs pairs of the grid take late_units units fewer than the
    // others (pairs that start late, on SMs a kernel before this one still holds)
    int late_pairs = 0;
    int late_units = 0;
};
inline int64_t tc_split_part_elems(int pairs, int chunks) { return (int64_t)pairs * chunks * 2 * 256; }
// N-chunks of a block of ncols columns (capacity: chunks of 128 columns, the narrowest the apply uses)
inline int tc_split_chunks(int64_t ncols) { return ncols <= 128 ? 1 : (int)((ncols + 127) / 128); }
// The accurate apply epilogue (PACK_SLICED or PACK_TF32X3 operands): the RBF
// exponent and kernel value in double-single arithmetic and the contraction
// with FP64 coefficients w64 (col_w is then unused); row_hl / col_hl are the
// low parts of the RBF terms from launch_row_terms(..., h_lo) (RBF only).
// Columns past ncols read as zero coefficients.  On sliced operands the dot
// products come from the slices' exact integer sums (4 group accumulators).
struct TcAccurate {
    const double *w64 = nullptr;
    const float *row_hl = nullptr;
    const float *col_hl = nullptr;
};
cudaError_t launch_block_tc(const TcOperand &Aop, const TcOperand &Bop, const KernelParams &kp,
                            const float *row_h, const float *col_h, const float *col_w, const double *rs,
                            double *g, float *out, int64_t ldo, int64_t nrows_out, int64_t ncols,
                            int *err, cudaStream_t st, bool lower = false, const TcSplit *split = nullptr,
                            bool pdl = false, int max_pairs = 0, const TcAccurate *acc = nullptr,
                            bool pdl_wait = true, int prio = 0);
// (pdl: launched as the programmatic dependent of the kernel before it in the stream, whose
// results the epilogue waits for unless pdl_wait is false: a block that reads nothing the
// kernel before it writes, started once that kernel has started.  prio: the launch's scheduling
// priority (0: the stream's), so that its CTAs take SMs before those of kernels beside it)

// setup / per-step helpers (sample_update.cu)
// src_scale: the per-row scales of an FP8 source (dtype DCD_FP8E4M3), else unused
cudaError_t launch_pack_rows(const void *src, int dtype, int64_t ld, int64_t m, int64_t n, const int32_t *rows,
                             void *dst, int dst_kind, int64_t n_pad, int64_t count, int *err, cudaStream_t st,
                             const float *src_scale = nullptr);
// Per-row e4m3 codes and scales of rows `rows` (or the first count) of a
// dense source: quantised from F64/F32/BF16, copied from an FP8 source.
// dst rows have ldq bytes (zero past n); a non-finite row sets DEV_BAD_VALUE.
cudaError_t launch_quantize_rows(const void *src, int dtype, int64_t ld, int64_t m, int64_t n, const int32_t *rows,
                                 const float *src_scale, uint8_t *dst, int64_t ldq, float *dst_scale, int64_t count,
                                 int *err, cudaStream_t st);
cudaError_t launch_label_check(const double *y, int64_t m, int *bad, cudaStream_t st);
cudaError_t launch_f64_to_f32(const double *src, int64_t count, float *dst, cudaStream_t st);
// h_lo (PACK_TF32X3, PACK_SLICED): the term as a pair of floats h + h_lo (FP64 sums), for the accurate
// epilogue; PACK_SLICED takes its per-row scales in `scale`
cudaError_t launch_row_terms(const void *packed, int kind, int64_t n_pad, int64_t m, const KernelParams &kp,
                             float *h, cudaStream_t st, const float *scale = nullptr, float *h_lo = nullptr);
// with the rows, optionally the per-row values f0 (and f1) of the same
// indices: d0[j] = f0[idx[j]] (0 for an index outside [0, m))
cudaError_t launch_gather_rows(const void *src, int64_t row_bytes, const int32_t *idx, int64_t count, int64_t m,
                               void *dst, int *err, cudaStream_t st, const float *f0 = nullptr, float *d0 = nullptr,
                               const float *f1 = nullptr, float *d1 = nullptr, const float *f2 = nullptr,
                               float *d2 = nullptr);
// The largest magnitude over rows `rows` (or the first count) of a dense
// source, folded by atomicMax into *bits (FP32 bits; zero it first).
cudaError_t launch_absmax_rows(const void *src, int dtype, int64_t ld, int64_t m, int64_t n, const int32_t *rows,
                               int64_t count, unsigned *bits, int *err, cudaStream_t st,
                               const float *src_scale = nullptr);
// fp16 rows (PACK_FP16) of rows `rows` (or the first count) of a dense
// source, all scaled by the power of two that *gbits (launch_absmax_rows over
// every row that shares the scale) fixes, written to sc[r] for each row; an
// FP8 source is dequantised first.  dst rows are n_pad fp16 values (zero padded).
cudaError_t launch_pack_fp16(const void *src, int dtype, int64_t ld, int64_t m, int64_t n, const int32_t *rows,
                             void *dst, int64_t n_pad, int64_t count, float *sc, const unsigned *gbits, int *err,
                             cudaStream_t st, const float *src_scale = nullptr);
// Sliced rows (PACK_SLICED) of rows `rows` (or the first count) of a dense
// source, with their power-of-two scales in sc (count floats); an FP8
// source is dequantised first.  dst rows are 4 planes of n_pad bf16.
cudaError_t launch_pack_sliced(const void *src, int dtype, int64_t ld, int64_t m, int64_t n, const int32_t *rows,
                               void *dst, int64_t n_pad, int64_t count, float *sc, int *err, cudaStream_t st,
                               const float *src_scale = nullptr);
cudaError_t launch_fill_f64(double *p, double v, int64_t count, cudaStream_t st);
// out[i] = start + i, i < count (shard.cu)
cudaError_t launch_iota(int32_t *out, int64_t count, int64_t start, cudaStream_t st);
cudaError_t launch_init_grad(int problem, const double *y, const double *alpha, double diag, int64_t m, double *g,
                             cudaStream_t st);
// the deferred gradient (solver.cu): acc[p] += add[p] (add may be NULL) + diag * (the sum of dprev
// over the previous step's positions q holding row S[p], in position order) where any does -- the
// update's part of the gradient at the next step's rows.  cprev <= 8192.
// the deferred K-SVM step (sample_update.cu): alpha and g at S (before they change), and the
// pending parts of the next step's alpha and g from this step's Kx = K(A_S, A_Sc) (row-major,
// leading dimension ldx), theta and w = y theta
cudaError_t launch_dcd_snapshot(const int32_t *S, int64_t cnt, int64_t m, const double *alpha, const double *g,
                                double *alpha_out, double *g_out, cudaStream_t st);
cudaError_t launch_dcd_pending(const int32_t *S, int64_t cnt, const double *y, const void *Kx, bool kx_f64,
                               int64_t ldx, const int32_t *Sc, const double *theta, const double *w, int64_t cc,
                               double diag, double *alpha_add, double *g_add, cudaStream_t st);
cudaError_t launch_defer_repeat(const int32_t *S, int64_t cnt, const int32_t *Sprev, const double *dprev,
                                int64_t cprev, double diag, const double *add, double *acc, cudaStream_t st);
// (pdl: launched as the programmatic dependent of the kernel before it, whose results it does not
// read; it signals its own dependent at once)
cudaError_t launch_update(const int32_t *S, const double *delta, int64_t cnt, double diag, double *alpha,
                          double *g, uint64_t *ctr, uint64_t ctr_advance, int64_t m, int *err, cudaStream_t st,
                          bool pdl = false, int prio = 0);
// The literal-order step's middle (Algorithms 2 and 4 as printed): from the stored
// block Q (m x ncols, FP64 or FP32, leading dimension ldq) and alpha, the gradient
// values of the step's coordinates written at their positions in g (K-SVM:
// y_i (U^T alpha)_p - 1 + diag alpha_i; K-RR: (U^T alpha)_p / lambda + diag alpha_i - y_i),
// and the Gram Kss = rows S of Q.  partials: max_blocks * ncols doubles.
cudaError_t launch_literal_terms(const void *Q, int q_f64, int64_t ldq, int64_t m, int64_t ncols, const int32_t *S,
                                 int problem, const double *y, const double *alpha, double inv_lambda, double diag,
                                 double *partials, int64_t max_blocks, double *g, void *Kss, int64_t ldk,
                                 cudaStream_t st);
cudaError_t launch_check(int problem, const double *g, const double *alpha, const double *y, int64_t m,
                         double C, int loss, double *partials, double *result, cudaStream_t st);
cudaError_t launch_nnz_count(const double *alpha, int64_t m, int *count, cudaStream_t st);
cudaError_t launch_coef(const double *y, const double *alpha, const int32_t *cols, int64_t count, double scale,
                        double *w, cudaStream_t st);

// CSR kernel block (block_csr.cu).  Values in FP32 (vals32) or FP64 (vals64,
// which takes precedence); squared row norms filled by launch_csr_prep.
struct CsrOperand {
    const int64_t *row_ptr = nullptr;
    const int32_t *col_idx = nullptr;
    const float *vals32 = nullptr;
    const double *vals64 = nullptr;
    int64_t m = 0, n = 0, nnz = 0;
    float *norm32 = nullptr;
    double *norm64 = nullptr;
    bool vec = false;  // col_idx and the values are 16-byte aligned (set by the launcher)
};
// Column map of the sampled rows: bitmap over [0, n), popcount prefix per
// 32-column word, per-slot entry offsets and (j, value) entries; capacity
// `cap` >= the sampled rows' nonzeros; counts zero between uses.
// With the apply through a transposed copy, the same kernel also writes per
// sampled position j and nonzero q < pmax of its row the column's CSC range
// (pstart, plen; plen = 0 past the row's end) and the value (pval).
struct CsrColMap {
    uint32_t *bits = nullptr;
    int32_t *wprefix = nullptr, *slot_off = nullptr, *counts = nullptr, *ent_j = nullptr;
    double *ent_v = nullptr;
    int nw = 0;
    int64_t cap = 0;
    const int64_t *csc_col_ptr = nullptr;
    int64_t *pstart = nullptr;
    int32_t *plen = nullptr;
    double *pval = nullptr;
    int pmax = 0;
};
size_t csr_colmap_bytes(int64_t n, int64_t cap);
CsrColMap csr_colmap_carve(void *base, int64_t n, int64_t cap);
cudaError_t launch_csr_prep(const CsrOperand &A, int *bad, int *maxlen, cudaStream_t st);
cudaError_t launch_csr_colmap(const CsrOperand &A, const int32_t *S, int64_t cnt, const CsrColMap &M, int *err,
                              cudaStream_t st);
// Transposed copy of a CSR operand: per column its entries' rows, CSR element
// indices and values (in the block's precision); and the per-step scratch of
// the apply through it: per 32-row tile a counter (zero between uses) and a
// bucket of incidence keys and products.
struct CscOperand {
    const int64_t *col_ptr = nullptr;
    const int32_t *row = nullptr;
    const int64_t *elem = nullptr;
    const void *val = nullptr;
    int64_t n = 0;
};
struct CscStep {
    int32_t *tile_cnt = nullptr;
    int64_t *key = nullptr;
    void *prod = nullptr;
};
size_t csc_bytes(int64_t n, int64_t nnz, bool fp64);
// builds the copy in `base` (csc_bytes); *maxcol_dev receives the longest column
cudaError_t launch_csc_build(const CsrOperand &A, bool fp64, void *base, CscOperand *C, int *maxcol_dev,
                             cudaStream_t st);
// cnt: sampled positions per step, maxrow: the longest row (the pair table of the column map)
size_t csc_step_bytes(int64_t m, int64_t cnt, int maxrow, bool fp64);
// base zeroed by the caller; the pair-table fields of *M are set
CscStep csc_step_carve(void *base, int64_t m, int64_t cnt, int maxrow, const CscOperand &C, CsrColMap *M);
// the apply form of launch_csr_block over all m rows through the transposed
// copy (bit-identical to the full pass); M is the step's column map (used by
// tiles whose bucket overflowed); maxrow = the longest row
// (first_scattered: the first chunk's incidences are already in the buckets,
// from launch_csr_csc_scatter_first after this step's column map)
cudaError_t launch_csr_apply_csc(const CsrOperand &A, const CsrColMap &M, const CscOperand &C, const CscStep &W,
                                 bool fp64, int maxrow, const KernelParams &kp, const int32_t *S, int64_t ncols,
                                 const float *w32, const double *w64, const double *rs, double *g, cudaStream_t st,
                                 bool first_scattered = false);
// the scatter of the first chunk only (it needs the step's sample and column map, not its coefficients)
cudaError_t launch_csr_csc_scatter_first(const CsrColMap &M, const CscOperand &C, const CscStep &W, bool fp64,
                                         int maxrow, int64_t ncols, cudaStream_t st);
// apply (out == nullptr): g[i] += rs[i] * sum_j K(a_i, a_{S_j}) w_j for i < nrows (rows == nullptr);
// store: out[r*ldo + j] = K(a_{rows[r]}, a_{S_j}) (rows == nullptr: row r).  FP64 (w64, out
// double) or FP32 (w32, out float).
cudaError_t launch_csr_block(const CsrOperand &A, const CsrColMap &M, bool fp64, const KernelParams &kp,
                             const int32_t *rows, int64_t nrows, const int32_t *S, int64_t ncols, const float *w32,
                             const double *w64, const double *rs, double *g, void *out, int64_t ldo, cudaStream_t st);

// recurrence (recur.cu)
// alpha and g at a DCD step's coordinates given as a snapshot plus the parts not yet in it (the
// deferred K-SVM step; position order of the step)
struct DcdPending {
    const double *alpha_snap = nullptr, *alpha_add = nullptr, *g_snap = nullptr, *g_add = nullptr;
};
// (pend: the chain reads alpha and g from it; only for cnt <= 128, else cudaErrorInvalidValue)
cudaError_t launch_recur_dcd(const void *Kss, int kss_f64, int64_t ldk, const int32_t *S, int64_t cnt,
                             const double *y, const double *alpha, const double *g, double omega, double nu,
                             double *delta, double *w64, float *w32, int *err, cudaStream_t st,
                             const DcdPending *pend = nullptr);
size_t recur_bdcd_scratch_bytes(int64_t nblk, int b);
// true when launch_recur_bdcd with these arguments reads only the lower
// triangle (with the diagonal blocks) of an FP32 Gram
bool recur_bdcd_lower_gram(int64_t nblk, int b, int refinements, int64_t ldk);
// The alpha / cached-gradient update (a6) done by the recurrence itself when
// it can: alpha_S += Delta, g_S += mdiag * Delta (repeats summed in position
// order) and the stream counter advanced.  `done` reports whether it ran.
struct FusedUpdate {
    double *alpha = nullptr;
    uint64_t *ctr = nullptr;
    uint64_t ctr_advance = 0;
    bool done = false;
};
// cluster recurrence (recur_cluster.cu): cluster size, or 0 when it does not apply;
// scratch of recur_cluster_scratch_bytes (super-block inverses, repeat masks and links)
int recur_cluster_size(int nblk, int b, int rounds);
size_t recur_cluster_scratch_bytes(int64_t nblk, int b);
// rhs: the right-hand sides by position (default -g[S]), for a diagonal panel of a longer chain
cudaError_t launch_recur_cluster(const float *Kss, int64_t ldk, const int32_t *S, int nblk, int b, int P,
                                 double lambda, double mdiag, double *g, int rounds, void *scratch, double *delta,
                                 double *w64, float *w32, const FusedUpdate *upd, int *err, cudaStream_t st,
                                 const double *rhs = nullptr);
int recur_cluster_panel_blocks(int b, int rounds);
// the prep and chain halves of launch_recur_cluster (a step's prep may run
// ahead, on another stream, of the previous step's chain)
cudaError_t launch_recur_cluster_prep(const float *Kss, int64_t ldk, const int32_t *S, int nblk, int b, double lambda,
                                      double mdiag, void *scratch, int *err, cudaStream_t st);
cudaError_t launch_recur_cluster_chain(const float *Kss, int64_t ldk, const int32_t *S, int nblk, int b, int P,
                                       double lambda, double mdiag, double *g, int rounds, void *scratch,
                                       double *delta, double *w64, float *w32, const FusedUpdate *upd, int *err,
                                       cudaStream_t st, const double *rhs = nullptr, int trig_sup = -1,
                                       bool rhs_add_g = false, int prio = 0);
// (trig_sup: the super-block of 32 rows after whose first-round result a
// kernel launched as this one's programmatic dependent may start; -1: at once.
// rhs_add_g: the right-hand side is -(g[S] + rhs), rhs holding a part of the
// gradient not yet added to g)
// 2-D tensor map over a row-major fp32 matrix (rows x cols, leading dimension
// ld elements, ld * 4 a multiple of 16), box of box_rows x box_cols, no
// swizzle, out-of-range elements read as zero (block_tc.cu)
bool make_map_f32_2d(CUtensorMap *map, const float *base, int64_t cols, int64_t rows, int64_t ld, int box_cols,
                     int box_rows);
// refinements < 0 selects the plain FP64 forward substitution.  With upd
// non-NULL the recurrence may also apply a6 (then g must be writable and
// upd->done is set); otherwise the caller runs launch_update.
cudaError_t launch_recur_bdcd(const void *Kss, int kss_f64, int64_t ldk, const int32_t *S, int64_t nblk, int b,
                              double lambda, double mdiag, const double *g, int refinements, void *scratch,
                              double *delta, double *w64, float *w32, FusedUpdate *upd, int *err, cudaStream_t st);

}  // namespace dcd
