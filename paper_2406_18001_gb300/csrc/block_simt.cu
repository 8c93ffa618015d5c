// block_simt.cu -- FP64 CUDA-core evaluation of the sampled kernel block
// (U_k = K(A, A_k) of Algorithm 2, Q_k of Algorithm 4) for the FP64 form.
//
// Two epilogues share one tile loop:
//   apply: g[i] += rs[i] * sum_c K(a_i, b_cols[c]) w[c]   (block never stored)
//   store: out[r, c] = K(a_rows[r], b_cols[c])            (the Gram of a3)
// The column points b are rows of A itself (the sampled rows) or of a second
// matrix B (rows gathered from other ranks in the row-sharded step);
// cols == nullptr takes B's rows 0..ncols-1.
// RBF distances are summed from coordinate differences (Table 1's definition)
// rather than expanded, so the FP64 form carries no cancellation error.
// The k-order of every dot product is fixed (0..n-1 in steps of BK), so the
// store and apply epilogues see bit-identical kernel values.
#include "dcd_internal.cuh"

namespace dcd {

namespace {

constexpr int TX = 16, TY = 16;   // 256 threads
constexpr int RM = 4;             // rows per thread
constexpr int BM = TY * RM;       // 64 rows per tile
constexpr int BK = 16;

template <int RN, bool STORE, bool RBF>
__global__ void __launch_bounds__(256) block_simt_f64_kernel(const double *__restrict__ A, int64_t lda, int64_t m,
                                                            int64_t n, KernelParams kp, const int32_t *rows,
                                                            int64_t nrows, const double *__restrict__ Bm,
                                                            int64_t ldb, int64_t mb, const int32_t *cols,
                                                            int64_t ncols, const double *__restrict__ w,
                                                            const double *__restrict__ rs, double *g, double *out,
                                                            int64_t ldo, int *err)
{
    constexpr int BN = TX * RN;
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    __shared__ double rowacc[BM];
    __shared__ int64_t rowoff[BM];
    __shared__ int64_t coloff[BN];

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int64_t ntiles = (nrows + BM - 1) / BM;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = tile * BM;
        if (threadIdx.x < BM) {
            int64_t r = r0 + threadIdx.x, off = -1;
            if (r < nrows) {
                int64_t ri = rows ? (int64_t)rows[r] : r;
                if (ri >= 0 && ri < m) off = ri * lda;
                else set_error(err, DEV_BAD_INDEX);
            }
            rowoff[threadIdx.x] = off;
            rowacc[threadIdx.x] = 0.0;
        }
        for (int64_t c0 = 0; c0 < ncols; c0 += BN) {
            __syncthreads();
            if (threadIdx.x < BN) {
                int64_t c = c0 + threadIdx.x, off = -1;
                if (c < ncols) {
                    int64_t ci = cols ? (int64_t)cols[c] : c;
                    if (ci >= 0 && ci < mb) off = ci * ldb;
                    else set_error(err, DEV_BAD_INDEX);
                }
                coloff[threadIdx.x] = off;
            }
            double acc[RM][RN];
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < RN; ++j) acc[i][j] = 0.0;
            for (int64_t k0 = 0; k0 < n; k0 += BK) {
                __syncthreads();
                for (int e = threadIdx.x; e < BM * BK; e += 256) {
                    int rr = e / BK, kk = e % BK;
                    int64_t off = rowoff[rr], k = k0 + kk;
                    As[kk][rr] = (off >= 0 && k < n) ? A[off + k] : 0.0;
                }
                for (int e = threadIdx.x; e < BN * BK; e += 256) {
                    int cc = e / BK, kk = e % BK;
                    int64_t off = coloff[cc], k = k0 + kk;
                    Bs[kk][cc] = (off >= 0 && k < n) ? Bm[off + k] : 0.0;
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    double a[RM], b[RN];
#pragma unroll
                    for (int i = 0; i < RM; ++i) a[i] = As[kk][ty + TY * i];
#pragma unroll
                    for (int j = 0; j < RN; ++j) b[j] = Bs[kk][tx + TX * j];
#pragma unroll
                    for (int i = 0; i < RM; ++i)
#pragma unroll
                        for (int j = 0; j < RN; ++j) {
                            if (RBF) {
                                double d = a[i] - b[j];
                                acc[i][j] = fma(d, d, acc[i][j]);
                            } else {
                                acc[i][j] = fma(a[i], b[j], acc[i][j]);
                            }
                        }
                }
            }
            if (STORE) {
#pragma unroll
                for (int i = 0; i < RM; ++i) {
                    int64_t r = r0 + ty + TY * i;
#pragma unroll
                    for (int j = 0; j < RN; ++j) {
                        int64_t c = c0 + tx + TX * j;
                        if (r < nrows && c < ncols) out[r * ldo + c] = kfun_f64(kp, acc[i][j]);
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < RM; ++i) {
                    double part = 0.0;
#pragma unroll
                    for (int j = 0; j < RN; ++j) {
                        int64_t c = c0 + tx + TX * j;
                        if (c < ncols) part = fma(kfun_f64(kp, acc[i][j]), w[c], part);
                    }
                    // fixed-order reduction over the 16 lanes that share these rows
#pragma unroll
                    for (int o = TX / 2; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                    if (tx == 0) rowacc[ty + TY * i] += part;
                }
            }
        }
        __syncthreads();
        if (!STORE && threadIdx.x < BM) {
            int64_t r = r0 + threadIdx.x;
            if (r < nrows) g[r] += (rs ? rs[r] : 1.0) * rowacc[threadIdx.x];
        }
    }
}

template <bool STORE, bool RBF>
cudaError_t launch_rn(int rn, int64_t grid, const double *A, int64_t lda, int64_t m, int64_t n, const KernelParams &kp,
                      const int32_t *rows, int64_t nrows, const double *Bm, int64_t ldb, int64_t mb,
                      const int32_t *cols, int64_t ncols, const double *w, const double *rs, double *g, double *out,
                      int64_t ldo, int *err, cudaStream_t st)
{
    switch (rn) {
    case 1:
        block_simt_f64_kernel<1, STORE, RBF><<<(unsigned)grid, 256, 0, st>>>(A, lda, m, n, kp, rows, nrows, Bm, ldb, mb,
                                                                           cols, ncols, w, rs, g, out, ldo, err);
        break;
    case 2:
        block_simt_f64_kernel<2, STORE, RBF><<<(unsigned)grid, 256, 0, st>>>(A, lda, m, n, kp, rows, nrows, Bm, ldb, mb,
                                                                           cols, ncols, w, rs, g, out, ldo, err);
        break;
    default:
        block_simt_f64_kernel<4, STORE, RBF><<<(unsigned)grid, 256, 0, st>>>(A, lda, m, n, kp, rows, nrows, Bm, ldb, mb,
                                                                           cols, ncols, w, rs, g, out, ldo, err);
        break;
    }
    return cudaGetLastError();
}

// Small blocks (few rows, at most 32 columns): one thread per (row, column)
// entry, so that the FP64 work (GB300 issues ~1.6 FP64 lane operations per
// clock per SM) spreads over every SM instead of filling a few 64 x 16 tiles.
// Each entry's dot product (or squared distance) runs over k = 0..n-1 with the
// operations of block_simt_f64_kernel, so both kernels produce the same bits.
// A one-warp CTA holds 32 / CW rows x CW columns (CW a power of two >= the
// columns).  Their vectors go through shared memory SMALL_KC dimensions at a
// time by asynchronous copies, all of a chunk in flight at once (coalesced, a
// lane per dimension): the dependent FMA chain then reads shared memory
// instead of waiting on an L2 round trip every few steps.  The apply sums a row's CW
// terms by a fixed butterfly and lane 0 of the row's group adds rs * sum to g.
constexpr int SMALL_KC = 64;

// an 8-byte asynchronous copy from global to shared memory (completed by cp.async.wait_all)
__device__ __forceinline__ void cp_async_8(double *dst, const double *src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(src) : "memory");
}

template <bool STORE, bool RBF>
__global__ void __launch_bounds__(32) block_small_f64_kernel(const double *__restrict__ A, int64_t lda, int64_t m,
                                                             int64_t n, KernelParams kp, const int32_t *rows,
                                                             int64_t nrows, const double *__restrict__ Bm,
                                                             int64_t ldb, int64_t mb, const int32_t *cols,
                                                             int64_t ncols, int cw, const double *__restrict__ w,
                                                             const double *__restrict__ rs, double *g, double *out,
                                                             int64_t ldo, int *err)
{
    // vectors 0..R-1: the CTA's rows; R..R+ncols-1: the columns (R + cw <= 33)
    __shared__ double sv[33][SMALL_KC + 1];
    __shared__ const double *src[33];
    const int lane = threadIdx.x;
    const int R = 32 / cw;
    const int64_t r0 = (int64_t)blockIdx.x * R;
    const int nc = (int)(ncols < cw ? ncols : cw);
    const int nv = R + nc;
    for (int v = lane; v < nv; v += 32) {  // nv reaches 33 (one column, or one row)
        const double *p = nullptr;
        if (v < R) {
            const int64_t r = r0 + v;
            if (r < nrows) {
                const int64_t ri = rows ? (int64_t)rows[r] : r;
                if (ri >= 0 && ri < m)
                    p = A + ri * lda;
                else
                    set_error(err, DEV_BAD_INDEX);
            }
        } else {
            const int64_t ci = cols ? (int64_t)cols[v - R] : (int64_t)(v - R);
            if (ci >= 0 && ci < mb)
                p = Bm + ci * ldb;
            else
                set_error(err, DEV_BAD_INDEX);
        }
        src[v] = p;
    }
    __syncwarp();
    const int c = lane % cw, rl = lane / cw;
    const int64_t r = r0 + rl;
    const bool ok = r < nrows && c < nc && src[rl] != nullptr && src[R + c] != nullptr;
    double acc = 0.0;
    for (int64_t k0 = 0; k0 < n; k0 += SMALL_KC) {
        const int kc = (int)(n - k0 < SMALL_KC ? n - k0 : SMALL_KC);
        // stage the chunk: two dimensions per lane per vector, every copy in flight at once (only
        // the valid vectors' first kc entries are read below)
        for (int v = 0; v < nv; ++v) {
            const double *p = src[v];
            if (!p) continue;
            if (lane < kc) cp_async_8(&sv[v][lane], p + k0 + lane);
            if (lane + 32 < kc) cp_async_8(&sv[v][lane + 32], p + k0 + lane + 32);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncwarp();
        if (ok) {
            const double *a = sv[rl], *b = sv[R + c];
#pragma unroll 8
            for (int k = 0; k < kc; ++k) {
                if (RBF) {
                    const double d = a[k] - b[k];
                    acc = fma(d, d, acc);
                } else {
                    acc = fma(a[k], b[k], acc);
                }
            }
        }
        __syncwarp();
    }
    const double kv = ok ? kfun_f64(kp, acc) : 0.0;
    if (STORE) {
        if (ok) out[r * ldo + c] = kv;
        return;
    }
    double part = ok ? kv * w[c] : 0.0;
    for (int o = 1; o < cw; o <<= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (c == 0 && r < nrows) g[r] += (rs ? rs[r] : 1.0) * part;
}

}  // namespace

cudaError_t launch_block_simt_f64(const double *A, int64_t lda, int64_t m, int64_t n, const KernelParams &kp,
                                  const int32_t *rows, int64_t nrows, const int32_t *cols, int64_t ncols,
                                  const double *w, const double *rs, double *g, double *out, int64_t ldo, int *err,
                                  cudaStream_t st, const double *Bm, int64_t ldb, int64_t mb)
{
    if (nrows <= 0 || ncols <= 0) return cudaSuccess;
    if (!Bm) {  // the column points are rows of A
        Bm = A;
        ldb = lda;
        mb = m;
    }
    const int rn = ncols <= 16 ? 1 : (ncols <= 32 ? 2 : 4);
    int64_t tiles = (nrows + BM - 1) / BM;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ncols <= 32 && tiles < 2 * (int64_t)sms) {  // too few tiles to occupy the GPU: an entry per thread
        int cw = 1;
        while (cw < ncols) cw <<= 1;
        // one warp per CTA: a few thousand entries then spread over every SM (the FP64 pipe, not
        // the warp count, bounds each SM)
        const int64_t threads = nrows * cw;
        const unsigned blocks = (unsigned)((threads + 31) / 32);
        const bool store = (out != nullptr), rbf = (kp.kind == DCD_RBF);
        if (store && rbf)
            block_small_f64_kernel<true, true><<<blocks, 32, 0, st>>>(A, lda, m, n, kp, rows, nrows, Bm, ldb, mb,
                                                                      cols, ncols, cw, w, rs, g, out, ldo, err);
        else if (store)
            block_small_f64_kernel<true, false><<<blocks, 32, 0, st>>>(A, lda, m, n, kp, rows, nrows, Bm, ldb, mb,
                                                                       cols, ncols, cw, w, rs, g, out, ldo, err);
        else if (rbf)
            block_small_f64_kernel<false, true><<<blocks, 32, 0, st>>>(A, lda, m, n, kp, rows, nrows, Bm, ldb, mb,
                                                                       cols, ncols, cw, w, rs, g, out, ldo, err);
        else
            block_small_f64_kernel<false, false><<<blocks, 32, 0, st>>>(A, lda, m, n, kp, rows, nrows, Bm, ldb, mb,
                                                                        cols, ncols, cw, w, rs, g, out, ldo, err);
        return cudaGetLastError();
    }
    int64_t grid = tiles < (int64_t)sms * 8 ? tiles : (int64_t)sms * 8;
    const bool store = (out != nullptr);
    const bool rbf = (kp.kind == DCD_RBF);
    if (store)
        return rbf ? launch_rn<true, true>(rn, grid, A, lda, m, n, kp, rows, nrows, Bm, ldb, mb, cols, ncols, w, rs, g, out, ldo, err, st)
                   : launch_rn<true, false>(rn, grid, A, lda, m, n, kp, rows, nrows, Bm, ldb, mb, cols, ncols, w, rs, g, out, ldo, err, st);
    return rbf ? launch_rn<false, true>(rn, grid, A, lda, m, n, kp, rows, nrows, Bm, ldb, mb, cols, ncols, w, rs, g, out, ldo, err, st)
               : launch_rn<false, false>(rn, grid, A, lda, m, n, kp, rows, nrows, Bm, ldb, mb, cols, ncols, w, rs, g, out, ldo, err, st);
}

}  // namespace dcd
