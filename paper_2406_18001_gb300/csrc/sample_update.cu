// sample_update.cu -- the small kernels of one outer s-step: index sampling
// (Algorithms 2 and 4, "choose i uniformly at random"), operand packing and
// norms, the scatter update of alpha and the cached gradient, and the
// convergence reductions (Section 5.1's duality gap and residual).
#include "dcd_internal.cuh"

#include <cuda_fp16.h>

namespace dcd {

// ----------------------------------------------------------- sampling -----
// DCD: one thread per iteration.  out[j] = floor(u * m / 2^64), u the
// SplitMix64 draw (seed, stream 0, counter first + j).
__global__ void sample_dcd_kernel(uint64_t seed, const uint64_t *ctr_dev, uint64_t first_host, int64_t m,
                                  int64_t count, int32_t *out, uint64_t *ctr_next)
{
    uint64_t first = (ctr_dev ? *ctr_dev : 0) + first_host;
    if (ctr_next && blockIdx.x == 0 && threadIdx.x == 0) *ctr_next = first + (uint64_t)count;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count; j += (int64_t)gridDim.x * blockDim.x)
        out[j] = (int32_t)below(sm64_draw(seed, 0, first + (uint64_t)j), (uint64_t)m);
}

// BDCD: one warp per block.  Floyd's algorithm (Bentley & Floyd 1987): for
// q = 0..b-1, J = m-b+q, r uniform in [0, J] from draw (seed, t+1, q); take r
// unless it was already taken, else take J.  The warp tests membership of r
// against the q indices taken so far in parallel.
__global__ void sample_bdcd_kernel(uint64_t seed, const uint64_t *ctr_dev, uint64_t first_host, int64_t m,
                                   int b, int64_t nblocks, int32_t *out, uint64_t *ctr_next)
{
    extern __shared__ int32_t sblk[];  // b indices per warp
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (warp >= nblocks) return;
    const uint64_t t0 = (ctr_dev ? *ctr_dev : 0) + first_host;
    if (ctr_next && warp == 0 && lane == 0) *ctr_next = t0 + (uint64_t)nblocks;
    const uint64_t t = t0 + (uint64_t)warp;
    int32_t *blk = sblk + (threadIdx.x >> 5) * b;
    for (int q = 0; q < b; ++q) {
        const int64_t J = m - b + q;
        const int64_t r = (int64_t)below(sm64_draw(seed, t + 1, (uint64_t)q), (uint64_t)(J + 1));
        bool hit = false;
        for (int p = lane; p < q; p += 32) hit |= (blk[p] == (int32_t)r);
        const unsigned any = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) blk[q] = (int32_t)(any ? J : r);
        __syncwarp();
    }
    for (int q = lane; q < b; q += 32) out[warp * b + q] = blk[q];
}

cudaError_t launch_sample(int method, uint64_t seed, const uint64_t *ctr_dev, uint64_t first_host, int64_t m,
                          int b, int64_t count, int32_t *out, int *err, cudaStream_t st, uint64_t *ctr_next)
{
    (void)err;
    if (count <= 0) return cudaSuccess;
    if (method == 0) {
        int threads = 128;
        int64_t blocks = (count + threads - 1) / threads;
        if (blocks > 4096) blocks = 4096;
        sample_dcd_kernel<<<(unsigned)blocks, threads, 0, st>>>(seed, ctr_dev, first_host, m, count, out, ctr_next);
    } else {
        int threads = 128;  // 4 warps = 4 blocks per CTA
        int64_t blocks = (count * 32 + threads - 1) / threads;
        sample_bdcd_kernel<<<(unsigned)blocks, threads, sizeof(int32_t) * 4 * b, st>>>(seed, ctr_dev, first_host, m,
                                                                                       b, count, out, ctr_next);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------ packing -----
// Value of an e4m3 code (OCP FP8: sign, 4 exponent bits with bias 7, 3
// mantissa bits; exponent field 0 holds the subnormals f * 2^-9; 0x7f / 0xff
// are NaN).  Exact in FP32: the float's bits are assembled directly.
__device__ __forceinline__ float e4m3_value(uint32_t c)
{
    const uint32_t e = (c >> 3) & 15u, f = c & 7u;
    float v;
    if ((c & 0x7Fu) == 0x7Fu) v = __int_as_float(0x7fc00000);
    else if (e) v = __uint_as_float(((e + 120u) << 23) | (f << 20));  // (1 + f/8) * 2^(e-7)
    else v = (float)f * 0.001953125f;                                 // f * 2^-9
    return (c & 0x80u) ? -v : v;
}

// Nearest e4m3 code of x (ties to even), saturating at +-448.
__device__ __forceinline__ uint32_t e4m3_code(float x)
{
    uint16_t pair;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(pair) : "f"(0.f), "f"(x));  // x -> low byte
    return pair & 0xFFu;
}

// Element `off` of a dense source as FP32; an FP8 source is scale * value(q)
// rounded once.
__device__ __forceinline__ float load_as_f32(const void *src, int dtype, int64_t off, float scale = 0.f)
{
    switch (dtype) {
    case DCD_F64: return (float)((const double *)src)[off];
    case DCD_F32: return ((const float *)src)[off];
    case DCD_BF16: return __bfloat162float(((const __nv_bfloat16 *)src)[off]);
    case DCD_FP8E4M3: return (float)((double)scale * (double)e4m3_value(((const uint8_t *)src)[off]));
    default: return 0.f;
    }
}

// dst row r (n_pad elements, zero padded) = src row rows[r] (or r),
// converted to bf16 (round to nearest even, dst_kind 0), fp32 (1, the tf32
// path reads fp32 storage) or fp64 (2).  An FP8 source is dequantised with
// its row scales (exactly, for fp64).
// Row indices outside [0, m) produce a zero row and set DEV_BAD_INDEX.
__global__ void pack_rows_kernel(const void *src, int dtype, int64_t ld, int64_t m, int64_t n, const int32_t *rows,
                                 void *dst, int dst_kind, int64_t n_pad, int64_t count, int *err,
                                 const float *src_scale)
{
    const int64_t total = count * n_pad;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / n_pad, c = e - r * n_pad;
        const int64_t sr = rows ? (int64_t)rows[r] : r;
        const bool inb = sr >= 0 && sr < m;
        if (!inb && c == 0) set_error(err, DEV_BAD_INDEX);
        const float rsc = (dtype == DCD_FP8E4M3 && inb) ? src_scale[sr] : 0.f;
        if (dst_kind == 2) {
            double v = 0.0;
            if (c < n && inb)
                v = (dtype == DCD_F64)       ? ((const double *)src)[sr * ld + c]
                    : (dtype == DCD_FP8E4M3) ? (double)rsc * (double)e4m3_value(((const uint8_t *)src)[sr * ld + c])
                                             : (double)load_as_f32(src, dtype, sr * ld + c);
            ((double *)dst)[e] = v;
            continue;
        }
        float v = (c < n && inb) ? load_as_f32(src, dtype, sr * ld + c, rsc) : 0.f;
        if (dst_kind == PACK_BF16X3) {
            // hi = bf16(v), lo = bf16(v - hi); v - hi is exact in fp32
            __nv_bfloat16 hi = __float2bfloat16_rn(v);
            __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
            __nv_bfloat16 *d = (__nv_bfloat16 *)dst + r * 2 * n_pad;
            d[c] = hi;
            d[n_pad + c] = lo;
        } else if (dst_kind == PACK_TF32X3) {
            // hi = tf32(v), lo = tf32(v - hi) (v - hi exact in fp32), both on the tf32 grid
            uint32_t th, tl;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(th) : "f"(v));
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(tl) : "f"(v - __uint_as_float(th)));
            float *d = (float *)dst + r * 2 * n_pad;
            d[c] = __uint_as_float(th);
            d[n_pad + c] = __uint_as_float(tl);
        } else if (dst_kind == 1) {
            // round to the tf32 grid (10-bit mantissa, nearest, ties away) so the
            // tensor core sees exactly the stored value and the row norms match
            uint32_t t;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
            ((float *)dst)[e] = __uint_as_float(t);
        } else {
            ((__nv_bfloat16 *)dst)[e] = __float2bfloat16_rn(v);
        }
    }
}

cudaError_t launch_pack_rows(const void *src, int dtype, int64_t ld, int64_t m, int64_t n, const int32_t *rows,
                             void *dst, int dst_kind, int64_t n_pad, int64_t count, int *err, cudaStream_t st,
                             const float *src_scale)
{
    if (dst_kind == PACK_FP8 || (dtype == DCD_FP8E4M3 && !src_scale)) return cudaErrorInvalidValue;
    if (count <= 0) return cudaSuccess;
    int64_t total = count * n_pad;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    pack_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, dtype, ld, m, n, rows, dst, dst_kind, n_pad, count, err,
                                                        src_scale);
    return cudaGetLastError();
}

// Per-row FP8 storage (one warp per row): the row is rounded to FP32,
// scale = fl32(max|a| / 448), code = e4m3(fl32(a / scale)) with IEEE FP32
// division; a row of zeros gets scale 0 and zero codes.  An FP8 source is
// copied with its scale.  Columns n..ldq-1 of the destination are zero.
// One warp per row: the row's largest magnitude fixes sc = 2^e with
// max |a| in [2^(e-1), 2^e) (1 for a zero row); u = a / sc in (-1, 1) is cut
// by round-to-nearest into s0 = rint(64 u) and, from the remainder r in
// [-1/2, 1/2], s_p = rint(128 r) for p = 1..3 -- integers in [-64, 64], exact
// in bf16, with u = s0 2^-6 + s1 2^-13 + s2 2^-20 + s3 2^-27 to within 2^-28.
// Every step is exact in FP64 (power-of-two scalings and differences of
// numbers within a factor two).  Columns n..n_pad-1 are zero.
__global__ void pack_sliced_kernel(const void *src, int dtype, int64_t ld, int64_t m, int64_t n, const int32_t *rows,
                                   __nv_bfloat16 *dst, int64_t n_pad, int64_t count, float *sc, int *err,
                                   const float *src_scale)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= count) return;
    const int64_t sr = rows ? (int64_t)rows[r] : r;
    const bool inb = sr >= 0 && sr < m;
    if (!inb && lane == 0) set_error(err, DEV_BAD_INDEX);
    const float rsc = (dtype == DCD_FP8E4M3 && inb) ? src_scale[sr] : 0.f;
    auto val = [&](int64_t c) -> double {
        if (c >= n || !inb) return 0.0;
        if (dtype == DCD_F64) return ((const double *)src)[sr * ld + c];
        if (dtype == DCD_FP8E4M3) return (double)rsc * (double)e4m3_value(((const uint8_t *)src)[sr * ld + c]);
        return (double)load_as_f32(src, dtype, sr * ld + c);
    };
    double mx = 0.0;
    for (int64_t c = lane; c < n; c += 32) mx = fmax(mx, fabs(val(c)));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0 && isfinite(mx)) frexp(mx, &e);
    else if (!(mx == 0.0) && lane == 0) set_error(err, DEV_BAD_VALUE);
    if (lane == 0) sc[r] = (float)ldexp(1.0, e);
    __nv_bfloat16 *d = dst + r * 4 * n_pad;
    for (int64_t c = lane; c < n_pad; c += 32) {
        double v = ldexp(val(c), 6 - e);
        const double s0 = rint(v);
        v = (v - s0) * 128.0;
        const double s1 = rint(v);
        v = (v - s1) * 128.0;
        const double s2 = rint(v);
        v = (v - s2) * 128.0;
        const double s3 = rint(v);
        d[c] = __double2bfloat16(s0);
        d[n_pad + c] = __double2bfloat16(s1);
        d[2 * n_pad + c] = __double2bfloat16(s2);
        d[3 * n_pad + c] = __double2bfloat16(s3);
    }
}

// The largest magnitude over rows `rows` (or the first count) of a dense
// source, folded into *bits (the FP32 bit pattern, which orders like the value
// for non-negative floats) by atomicMax; a non-finite value sets
// DEV_BAD_VALUE.  One warp per row.
__global__ void absmax_rows_kernel(const void *src, int dtype, int64_t ld, int64_t m, int64_t n, const int32_t *rows,
                                   int64_t count, unsigned *bits, int *err, const float *src_scale)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= count) return;
    const int64_t sr = rows ? (int64_t)rows[r] : r;
    if (sr < 0 || sr >= m) return;  // the pack reports bad indices
    const float rsc = dtype == DCD_FP8E4M3 ? src_scale[sr] : 0.f;
    float mx = 0.f;
    bool bad = false;
    for (int64_t c = lane; c < n; c += 32) {
        const float v = load_as_f32(src, dtype, sr * ld + c, rsc);
        bad |= !isfinite(v);
        mx = fmaxf(mx, fabsf(v));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (__any_sync(0xffffffffu, bad)) {
        if (lane == 0) set_error(err, DEV_BAD_VALUE);
        return;
    }
    if (lane == 0) atomicMax(bits, __float_as_uint(mx));
}

// One warp per row.  The scale is one power of two for every row, sc = 2^(e -
// 15) with the largest magnitude over the matrix in [2^(e-1), 2^e) (from
// *gbits), so that |a| / sc < 2^15 (fp16's largest finite value is 65504);
// q = fp16(a / sc) rounds to nearest even (the division by a power of two is
// exact).  fp16's exponent range keeps every value down to 2^-29 of the
// largest at full precision.  A zero matrix gets sc = 2^-15.  sc[r] = sc for
// every row; columns n..n_pad-1 are zero.
__global__ void pack_fp16_kernel(const void *src, int dtype, int64_t ld, int64_t m, int64_t n, const int32_t *rows,
                                 __half *dst, int64_t n_pad, int64_t count, float *sc, const unsigned *gbits,
                                 int *err, const float *src_scale)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= count) return;
    const int64_t sr = rows ? (int64_t)rows[r] : r;
    const bool inb = sr >= 0 && sr < m;
    if (!inb && lane == 0) set_error(err, DEV_BAD_INDEX);
    const float rsc = (dtype == DCD_FP8E4M3 && inb) ? src_scale[sr] : 0.f;
    const float mx = __uint_as_float(*gbits);
    int e = 0;
    if (mx > 0.f && isfinite(mx)) frexpf(mx, &e);
    e = max(e, -110);  // the scale 2^(e - 15) stays a normal FP32 number
    if (lane == 0) sc[r] = ldexpf(1.f, e - 15);
    __half *d = dst + r * n_pad;
    for (int64_t c = lane; c < n_pad; c += 32)
        d[c] = __float2half_rn((c < n && inb) ? ldexpf(load_as_f32(src, dtype, sr * ld + c, rsc), 15 - e) : 0.f);
}

cudaError_t launch_absmax_rows(const void *src, int dtype, int64_t ld, int64_t m, int64_t n, const int32_t *rows,
                               int64_t count, unsigned *bits, int *err, cudaStream_t st, const float *src_scale)
{
    if (count <= 0) return cudaSuccess;
    if (dtype == DCD_FP8E4M3 && !src_scale) return cudaErrorInvalidValue;
    const int64_t blocks = (count * 32 + 255) / 256;
    absmax_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, dtype, ld, m, n, rows, count, bits, err, src_scale);
    return cudaGetLastError();
}

cudaError_t launch_pack_fp16(const void *src, int dtype, int64_t ld, int64_t m, int64_t n, const int32_t *rows,
                             void *dst, int64_t n_pad, int64_t count, float *sc, const unsigned *gbits, int *err,
                             cudaStream_t st, const float *src_scale)
{
    if (count <= 0) return cudaSuccess;
    if (!sc || !gbits || n_pad < n || n_pad % 64 || (dtype == DCD_FP8E4M3 && !src_scale))
        return cudaErrorInvalidValue;
    const int64_t blocks = (count * 32 + 255) / 256;
    pack_fp16_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, dtype, ld, m, n, rows, (__half *)dst, n_pad, count, sc,
                                                       gbits, err, src_scale);
    return cudaGetLastError();
}

cudaError_t launch_pack_sliced(const void *src, int dtype, int64_t ld, int64_t m, int64_t n, const int32_t *rows,
                               void *dst, int64_t n_pad, int64_t count, float *sc, int *err, cudaStream_t st,
                               const float *src_scale)
{
    if (count <= 0) return cudaSuccess;
    if (!sc || n_pad < n || n_pad % 64 || (dtype == DCD_FP8E4M3 && !src_scale)) return cudaErrorInvalidValue;
    const int64_t blocks = (count * 32 + 255) / 256;
    pack_sliced_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, dtype, ld, m, n, rows, (__nv_bfloat16 *)dst, n_pad,
                                                         count, sc, err, src_scale);
    return cudaGetLastError();
}

// ------------------------------------------------ literal-order step --
// The paper's printed order (Algorithms 2 and 4) keeps the m x sb block U_k /
// Q_k in memory and forms U_j^T alpha_sk from it.  literal_partial_kernel:
// block b sums rows [b R, (b+1) R) of (y_i) Q[i][c] alpha_i for every column
// c (consecutive threads read consecutive columns of a row), in row order.
template <typename QT>
__global__ void literal_partial_kernel(const QT *Q, int64_t ldq, int64_t m, int64_t ncols, const double *alpha,
                                       const double *y, int64_t rows_per_block, double *partials)
{
    const int64_t r0 = blockIdx.x * rows_per_block, r1 = min(m, r0 + rows_per_block);
    for (int64_t c = threadIdx.x; c < ncols; c += blockDim.x) {
        double acc = 0.0;
        for (int64_t i = r0; i < r1; ++i) {
            const double a = y ? y[i] * alpha[i] : alpha[i];
            acc = fma((double)Q[i * ldq + c], a, acc);
        }
        partials[blockIdx.x * ncols + c] = acc;
    }
}

// u_p = sum of the partials in block order, then the gradient value of the
// step's coordinate i = S[p] written at position i of a full-length array g
// (repeats write the same value):
//   K-SVM: g_i = y_i u_p - 1 + omega alpha_i        (u = U_k^T alpha)
//   K-RR:  g_i = u_p / lambda + m alpha_i - y_i
__global__ void literal_grad_kernel(const double *partials, int64_t nblk, int64_t ncols, const int32_t *S,
                                    int problem, const double *y, const double *alpha, double inv_lambda,
                                    double diag, double *g)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= ncols) return;
    double u = 0.0;
    for (int64_t b = 0; b < nblk; ++b) u += partials[b * ncols + p];
    const int32_t i = S[p];
    g[i] = problem == 0 ? fma(y[i], u, -1.0) + diag * alpha[i] : u * inv_lambda + diag * alpha[i] - y[i];
}

// G_k = V_k^T U_k: row r of the Gram is row S[r] of the stored block
template <typename QT>
__global__ void literal_gram_kernel(const QT *Q, int64_t ldq, const int32_t *S, int64_t ncols, QT *Kss,
                                    int64_t ldk)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= ncols * ncols) return;
    const int64_t r = e / ncols, c = e - r * ncols;
    Kss[r * ldk + c] = Q[(int64_t)S[r] * ldq + c];
}

cudaError_t launch_literal_terms(const void *Q, int q_f64, int64_t ldq, int64_t m, int64_t ncols, const int32_t *S,
                                 int problem, const double *y, const double *alpha, double inv_lambda, double diag,
                                 double *partials, int64_t max_blocks, double *g, void *Kss, int64_t ldk,
                                 cudaStream_t st)
{
    if (ncols <= 0) return cudaSuccess;
    int64_t nblk = max_blocks < 1 ? 1 : max_blocks;
    const int64_t rpb = (m + nblk - 1) / nblk;
    nblk = (m + rpb - 1) / rpb;
    const int thr = ncols >= 256 ? 256 : (int)((ncols + 31) / 32 * 32);
    const double *ys = problem == 0 ? y : nullptr;
    if (q_f64)
        literal_partial_kernel<double><<<(unsigned)nblk, thr, 0, st>>>((const double *)Q, ldq, m, ncols, alpha, ys,
                                                                     rpb, partials);
    else
        literal_partial_kernel<float><<<(unsigned)nblk, thr, 0, st>>>((const float *)Q, ldq, m, ncols, alpha, ys, rpb,
                                                                    partials);
    literal_grad_kernel<<<(unsigned)((ncols + 255) / 256), 256, 0, st>>>(partials, nblk, ncols, S, problem, y, alpha,
                                                                       inv_lambda, diag, g);
    const unsigned gb = (unsigned)((ncols * ncols + 255) / 256);
    if (q_f64)
        literal_gram_kernel<double><<<gb, 256, 0, st>>>((const double *)Q, ldq, S, ncols, (double *)Kss, ldk);
    else
        literal_gram_kernel<float><<<gb, 256, 0, st>>>((const float *)Q, ldq, S, ncols, (float *)Kss, ldk);
    return cudaGetLastError();
}

__global__ void quantize_rows_kernel(const void *src, int dtype, int64_t ld, int64_t m, int64_t n,
                                     const int32_t *rows, const float *src_scale, uint8_t *dst, int64_t ldq,
                                     float *dst_scale, int64_t count, int *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= count) return;
    const int64_t sr = rows ? (int64_t)rows[r] : r;
    uint8_t *d = dst + r * ldq;
    if (sr < 0 || sr >= m) {
        if (lane == 0) {
            set_error(err, DEV_BAD_INDEX);
            dst_scale[r] = 0.f;
        }
        for (int64_t c = lane; c < ldq; c += 32) d[c] = 0;
        return;
    }
    bool bad = false;
    float scale;
    if (dtype == DCD_FP8E4M3) {
        const uint8_t *s = (const uint8_t *)src + sr * ld;
        for (int64_t c = lane; c < ldq; c += 32) {
            const uint8_t v = c < n ? s[c] : 0;
            bad |= (v & 0x7F) == 0x7F;
            d[c] = v;
        }
        scale = src_scale[sr];
        bad |= !(scale >= 0.f && scale <= 3.4028234e38f);
    } else {
        float amax = 0.f;
        for (int64_t c = lane; c < n; c += 32) {
            const float v = load_as_f32(src, dtype, sr * ld + c);
            bad |= !(fabsf(v) <= 3.4028234e38f);
            amax = fmaxf(amax, fabsf(v));
        }
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        scale = __fdiv_rn(amax, 448.f);
        for (int64_t c = lane; c < ldq; c += 32) {
            uint32_t code = 0;
            if (c < n && scale > 0.f) code = e4m3_code(__fdiv_rn(load_as_f32(src, dtype, sr * ld + c), scale));
            d[c] = (uint8_t)code;
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) set_error(err, DEV_BAD_VALUE);
    if (lane == 0) dst_scale[r] = scale;
}

cudaError_t launch_quantize_rows(const void *src, int dtype, int64_t ld, int64_t m, int64_t n, const int32_t *rows,
                                 const float *src_scale, uint8_t *dst, int64_t ldq, float *dst_scale, int64_t count,
                                 int *err, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    if (ldq < n || (dtype == DCD_FP8E4M3 && !src_scale)) return cudaErrorInvalidValue;
    const int64_t blocks = (count * 32 + 255) / 256;
    quantize_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, dtype, ld, m, n, rows, src_scale, dst, ldq, dst_scale,
                                                           count, err);
    return cudaGetLastError();
}

// Number of labels that are not exactly +1 or -1.
__global__ void label_check_kernel(const double *y, int64_t m, int *bad)
{
    int local = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        local += !(y[i] == 1.0 || y[i] == -1.0);
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(bad, local);
}

cudaError_t launch_label_check(const double *y, int64_t m, int *bad, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    int64_t blocks = (m + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    label_check_kernel<<<(unsigned)blocks, 256, 0, st>>>(y, m, bad);
    return cudaGetLastError();
}

__global__ void f64_to_f32_kernel(const double *src, int64_t count, float *dst)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count; j += (int64_t)gridDim.x * blockDim.x)
        dst[j] = (float)src[j];
}

cudaError_t launch_f64_to_f32(const double *src, int64_t count, float *dst, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    f64_to_f32_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, count, dst);
    return cudaGetLastError();
}

// h[r] = gamma * log2(e) * ||x_r||^2 of the packed (already rounded) row, for
// the RBF expansion ||a||^2 + ||b||^2 - 2 a.b (Section 5.2); 0 for the other
// kernels.  For split rows the norm is the one the three MMAs reproduce,
// sum(hi^2 + 2 hi lo), so that a row's distance to itself stays ~0; FP8 and
// FP16 rows take the dequantised norm rscale[r]^2 * sum value(q)^2.  One warp
// per row, FP64 partial sums, fixed order.
__global__ void row_terms_kernel(const void *packed, int kind, int64_t n_pad, int64_t m, double scale, float *h,
                                 const float *rscale, float *h_lo)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= m) return;
    if (kind == PACK_SLICED) {
        // the slices' own product sums, truncated as the apply truncates them (groups p + q <= 3),
        // exact in FP64: a.a = sc^2 2^-12 (S0 + 2^-7 S1 + 2^-14 S2 + 2^-21 S3)
        const __nv_bfloat16 *row = (const __nv_bfloat16 *)packed + r * 4 * n_pad;
        double S0 = 0.0, S1 = 0.0, S2 = 0.0, S3 = 0.0;
        for (int64_t c = lane; c < n_pad; c += 32) {
            const double a0 = __bfloat162float(row[c]), a1 = __bfloat162float(row[n_pad + c]);
            const double a2 = __bfloat162float(row[2 * n_pad + c]), a3 = __bfloat162float(row[3 * n_pad + c]);
            S0 += a0 * a0;
            S1 += 2.0 * a0 * a1;
            S2 += 2.0 * a0 * a2 + a1 * a1;
            S3 += 2.0 * (a0 * a3 + a1 * a2);
        }
        for (int o = 16; o > 0; o >>= 1) {
            S0 += __shfl_xor_sync(0xffffffffu, S0, o);
            S1 += __shfl_xor_sync(0xffffffffu, S1, o);
            S2 += __shfl_xor_sync(0xffffffffu, S2, o);
            S3 += __shfl_xor_sync(0xffffffffu, S3, o);
        }
        if (lane == 0) {
            const double sc = rscale[r];
            const double v = scale * (sc * sc) * 0x1p-12 * (S0 + 0x1p-7 * S1 + 0x1p-14 * S2 + 0x1p-21 * S3);
            const float vh = (float)v;
            h[r] = vh;
            if (h_lo) h_lo[r] = (float)(v - (double)vh);
        }
        return;
    }
    if (kind == PACK_FP16) {
        // fp16 values: their squares are exact in FP64 and summed in FP64; times the row scale^2
        const __half *row = (const __half *)packed + r * n_pad;
        double sd = 0.0;
        for (int64_t c = lane; c < n_pad; c += 32) {
            const double v = __half2float(row[c]);
            sd = fma(v, v, sd);
        }
        for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
        if (lane == 0) h[r] = (float)(scale * sd * (double)rscale[r] * (double)rscale[r]);
        return;
    }
    if (kind == PACK_TF32X3) {
        // split tf32: the products the three MMAs form, hi.hi + 2 hi.lo, each exact in FP64 (24-bit
        // factors) and summed in FP64; the term is stored as a pair of floats hi + lo (h_lo given) for
        // the accurate epilogue, or rounded to one float
        const float *row = (const float *)packed + r * 2 * n_pad;
        double sd = 0.0;
        for (int64_t c = lane; c < n_pad; c += 32) {
            const double hi = row[c], lo = row[n_pad + c];
            sd = fma(hi, hi + 2.0 * lo, sd);
        }
        for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
        if (lane == 0) {
            const double v = scale * sd;
            const float vh = (float)v;
            h[r] = vh;
            if (h_lo) h_lo[r] = (float)(v - (double)vh);
        }
        return;
    }
    // per-lane FP32 sums (each lane adds n_pad/32 squares), combined in FP64
    float sf = 0.f;
    for (int64_t c = lane; c < n_pad; c += 32) {
        if (kind == PACK_TF32) {
            const float v = ((const float *)packed)[r * n_pad + c];
            sf = fmaf(v, v, sf);
        } else if (kind == PACK_BF16X3) {
            const __nv_bfloat16 *row = (const __nv_bfloat16 *)packed + r * 2 * n_pad;
            const float hi = __bfloat162float(row[c]), lo = __bfloat162float(row[n_pad + c]);
            sf = fmaf(hi, hi + 2.f * lo, sf);
        } else if (kind == PACK_FP8) {  // sum of value(q)^2; the row scale comes in below
            const float v = e4m3_value(((const uint8_t *)packed)[r * n_pad + c]);
            sf = fmaf(v, v, sf);
        } else {
            const float v = __bfloat162float(((const __nv_bfloat16 *)packed)[r * n_pad + c]);
            sf = fmaf(v, v, sf);
        }
    }
    double s = sf;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (kind == PACK_FP8) s *= (double)rscale[r] * (double)rscale[r];
    if (lane == 0) h[r] = (float)(scale * s);
}

cudaError_t launch_row_terms(const void *packed, int kind, int64_t n_pad, int64_t m, const KernelParams &kp,
                             float *h, cudaStream_t st, const float *rscale, float *h_lo)
{
    if ((kind == PACK_FP8 || kind == PACK_SLICED || kind == PACK_FP16) && !rscale) return cudaErrorInvalidValue;
    if (h_lo && kind != PACK_TF32X3 && kind != PACK_SLICED) return cudaErrorInvalidValue;
    if (m <= 0) return cudaSuccess;
    double scale = (kp.kind == DCD_RBF) ? kp.gamma * 1.4426950408889634 : 0.0;
    int64_t blocks = (m * 32 + 255) / 256;
    row_terms_kernel<<<(unsigned)blocks, 256, 0, st>>>(packed, kind, n_pad, m, scale, h, rscale, h_lo);
    return cudaGetLastError();
}

// dst row j = src row idx[j] (whole packed rows, 16-byte vectors; row_bytes
// is a multiple of 128), and d0[j] = f0[idx[j]], d1[j] = f1[idx[j]] where
// given.  Indices outside [0, m) give a zero row (and zero values) and set
// DEV_BAD_INDEX.
__global__ void gather_rows_kernel(const uint4 *src, int64_t row_vec, const int32_t *idx, int64_t count, int64_t m,
                                   uint4 *dst, int *err, const float *f0, float *d0, const float *f1, float *d1,
                                   const float *f2, float *d2)
{
    const int64_t total = count * row_vec;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / row_vec, c = e - j * row_vec;
        const int64_t r = idx[j];
        const bool bad = r < 0 || r >= m;
        if (bad) {
            if (c == 0) set_error(err, DEV_BAD_INDEX);
            dst[e] = make_uint4(0, 0, 0, 0);
        } else {
            dst[e] = src[r * row_vec + c];
        }
        if (c == 0) {
            if (d0) d0[j] = bad ? 0.f : f0[r];
            if (d1) d1[j] = bad ? 0.f : f1[r];
            if (d2) d2[j] = bad ? 0.f : f2[r];
        }
    }
}

cudaError_t launch_gather_rows(const void *src, int64_t row_bytes, const int32_t *idx, int64_t count, int64_t m,
                               void *dst, int *err, cudaStream_t st, const float *f0, float *d0, const float *f1,
                               float *d1, const float *f2, float *d2)
{
    if (count <= 0) return cudaSuccess;
    if ((d0 && !f0) || (d1 && !f1) || (d2 && !f2)) return cudaErrorInvalidValue;
    const int64_t row_vec = row_bytes / 16;
    int64_t blocks = (count * row_vec + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    gather_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>((const uint4 *)src, row_vec, idx, count, m, (uint4 *)dst,
                                                         err, f0, d0, f1, d1, f2, d2);
    return cudaGetLastError();
}

__global__ void fill_f64_kernel(double *p, double v, int64_t count)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count; j += (int64_t)gridDim.x * blockDim.x)
        p[j] = v;
}

cudaError_t launch_fill_f64(double *p, double v, int64_t count, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    fill_f64_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, v, count);
    return cudaGetLastError();
}

// ------------------------------------------------------ gradient init -----
// The diagonal and constant parts of the cached gradient:
//   K-SVM (problem 0): g = -1 + omega * alpha     (+ Q alpha added by the block kernel)
//   K-RR  (problem 1): g = m * alpha - y          (+ K alpha / lambda added likewise)
__global__ void init_grad_kernel(int problem, const double *y, const double *alpha, double diag, int64_t m, double *g)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        double a = alpha[i];
        g[i] = (problem == 0) ? (-1.0 + diag * a) : (diag * a - y[i]);
    }
}

cudaError_t launch_init_grad(int problem, const double *y, const double *alpha, double diag, int64_t m, double *g,
                             cudaStream_t st)
{
    int64_t blocks = (m + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    init_grad_kernel<<<(unsigned)blocks, 256, 0, st>>>(problem, y, alpha, diag, m, g);
    return cudaGetLastError();
}

// Coefficients of the initial gradient pass for a nonzero alpha_0:
// w[j] = y[c] * alpha[c] (K-SVM, y given) or alpha[c] * scale (K-RR, 1/lambda).
__global__ void coef_kernel(const double *y, const double *alpha, const int32_t *cols, int64_t count, double scale,
                            double *w)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count; j += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = cols[j];
        w[j] = y ? y[c] * alpha[c] : alpha[c] * scale;
    }
}

cudaError_t launch_coef(const double *y, const double *alpha, const int32_t *cols, int64_t count, double scale,
                        double *w, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    coef_kernel<<<(unsigned)blocks, 256, 0, st>>>(y, alpha, cols, count, scale, w);
    return cudaGetLastError();
}

__global__ void nnz_kernel(const double *alpha, int64_t m, int *count)
{
    int local = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        local += (alpha[i] != 0.0);
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

cudaError_t launch_nnz_count(const double *alpha, int64_t m, int *count, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    int64_t blocks = (m + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    nnz_kernel<<<(unsigned)blocks, 256, 0, st>>>(alpha, m, count);
    return cudaGetLastError();
}

// --------------------------------------------------------- alpha update ---
// alpha_{sk+s} = alpha_sk + sum_t V_t delta_t (Algorithms 2 and 4) and the
// diagonal part of the gradient update, g[S_j] += diag * delta_j (omega for
// K-SVM-L2, m for K-RR).  Repeated indices are merged deterministically: a
// position with no earlier occurrence of its index is a run head and adds the
// deltas of its index's occurrences in position order.  One warp per
// position, S staged in shared memory: the warp compares 128 positions per
// step (4 per lane, ballot), so a position costs cnt / 128 steps.
// cnt <= 8192.  Also advances the stream counter.
constexpr int UPD_MAX = 8192;
constexpr int UPD_WARPS = 8;

__global__ void __launch_bounds__(UPD_WARPS * 32)
    update_kernel(const int32_t *S, const double *delta, int cnt, double diag, double *alpha, double *g,
                  uint64_t *ctr, uint64_t ctr_advance, int64_t m, int *err)
{
    __shared__ __align__(16) int32_t sS[UPD_MAX];
    // a kernel launched as this one's programmatic dependent may start; it waits for this grid to
    // finish before it touches alpha or g (a no-op without one)
    if (threadIdx.x == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int c4 = (cnt + 3) & ~3;
    for (int q = threadIdx.x; q < c4; q += blockDim.x) sS[q] = q < cnt ? S[q] : -1;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0 && ctr) *ctr += ctr_advance;
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * UPD_WARPS;
    const int4 *s4 = (const int4 *)sS;
    for (int p = blockIdx.x * UPD_WARPS + (threadIdx.x >> 5); p < cnt; p += nw) {  // warp-uniform
        const int32_t key = sS[p];
        if (key < 0 || key >= m) {
            if (lane == 0) set_error(err, DEV_BAD_INDEX);
            continue;
        }
        // head: no earlier position holds key (128 positions per step, 4 per lane)
        bool head = true;
        for (int q0 = 0; q0 < p && head; q0 += 128) {
            const int q = q0 + 4 * lane;
            bool hit = false;
            if (q < p) {
                const int4 w = s4[q >> 2];
                hit = (w.x == key) || (q + 1 < p && w.y == key) || (q + 2 < p && w.z == key) ||
                      (q + 3 < p && w.w == key);
            }
            head = !__any_sync(0xffffffffu, hit);
        }
        if (!head) continue;
        // occurrences at positions >= p, in position order (every lane the same sum)
        double sum = 0.0;
        for (int q0 = p & ~3; q0 < c4; q0 += 128) {
            const int q = q0 + 4 * lane;
            unsigned mk = 0;
            if (q < c4) {
                const int4 w = s4[q >> 2];
                mk = (w.x == key ? 1u : 0u) | (w.y == key ? 2u : 0u) | (w.z == key ? 4u : 0u) | (w.w == key ? 8u : 0u);
                if (q < p) mk &= ~((1u << (p - q)) - 1u);  // only the group holding p starts below p
            }
            unsigned lanes = __ballot_sync(0xffffffffu, mk != 0);
            while (lanes) {  // rare: lanes in order, each lane's hits in order
                const int l = __ffs(lanes) - 1;
                unsigned ml = __shfl_sync(0xffffffffu, mk, l);
                const int ql = q0 + 4 * l;
                while (ml) {
                    sum += delta[ql + __ffs(ml) - 1];
                    ml &= ml - 1;
                }
                lanes &= lanes - 1;
            }
        }
        if (lane == 0) {
            alpha[key] += sum;
            g[key] += diag * sum;
        }
    }
}

// ------------------------------------------------- deferred gradient --
// The deferred K-SVM step.  snapshot: alpha and g at the next step's coordinates, taken before
// this step's block and update write them.
__global__ void dcd_snapshot_kernel(const int32_t *S, int64_t cnt, int64_t m, const double *alpha, const double *g,
                                    double *alpha_out, double *g_out)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= cnt) return;
    const int64_t i = S[p];
    const bool ok = i >= 0 && i < m;
    alpha_out[p] = ok ? alpha[i] : 0.0;
    g_out[p] = ok ? g[i] : 0.0;
}

cudaError_t launch_dcd_snapshot(const int32_t *S, int64_t cnt, int64_t m, const double *alpha, const double *g,
                                double *alpha_out, double *g_out, cudaStream_t st)
{
    if (cnt <= 0) return cudaSuccess;
    dcd_snapshot_kernel<<<(unsigned)((cnt + 127) / 128), 128, 0, st>>>(S, cnt, m, alpha, g, alpha_out, g_out);
    return cudaGetLastError();
}

// The pending parts of the next step's alpha and g at its coordinates p (rows S[p]) from this
// step (coordinates Sc, steps theta, coefficients w = y theta):
//   g_add[p] = y[S[p]] (sum_j Kx[p][j] w[j]) + diag * (sum of theta over this step's positions
//              holding row S[p], in position order), alpha_add[p] = that sum.
// One warp per p; the lanes' partial sums over j are combined by a fixed butterfly.
template <typename KT>
__global__ void dcd_pending_kernel(const int32_t *S, int cnt, const double *y, const KT *Kx, int64_t ldx,
                                   const int32_t *Sc, const double *theta, const double *w, int cc, double diag,
                                   double *alpha_add, double *g_add)
{
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= cnt) return;  // warp-uniform
    const int32_t key = S[p];
    double dot = 0.0;
    for (int j = lane; j < cc; j += 32) dot = fma((double)Kx[(int64_t)p * ldx + j], w[j], dot);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    double sum = 0.0;
    bool any = false;
    for (int q0 = 0; q0 < cc; q0 += 32) {
        unsigned hit = __ballot_sync(0xffffffffu, q0 + lane < cc && Sc[q0 + lane] == key);
        any = any || hit != 0u;
        while (hit) {  // in position order
            sum += theta[q0 + __ffs(hit) - 1];
            hit &= hit - 1u;
        }
    }
    if (lane == 0) {
        double v = y[key] * dot;
        if (any) v += diag * sum;
        g_add[p] = v;
        alpha_add[p] = any ? sum : 0.0;
    }
}

cudaError_t launch_dcd_pending(const int32_t *S, int64_t cnt, const double *y, const void *Kx, bool kx_f64,
                               int64_t ldx, const int32_t *Sc, const double *theta, const double *w, int64_t cc,
                               double diag, double *alpha_add, double *g_add, cudaStream_t st)
{
    if (cnt <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((cnt + 3) / 4);
    if (kx_f64)
        dcd_pending_kernel<double><<<blocks, 128, 0, st>>>(S, (int)cnt, y, (const double *)Kx, ldx, Sc, theta, w,
                                                           (int)cc, diag, alpha_add, g_add);
    else
        dcd_pending_kernel<float><<<blocks, 128, 0, st>>>(S, (int)cnt, y, (const float *)Kx, ldx, Sc, theta, w,
                                                          (int)cc, diag, alpha_add, g_add);
    return cudaGetLastError();
}

// acc[p] += add[p] (add: optional) + diag * sum of dprev[q] over q with
// Sprev[q] == S[p] (in position order, the update's own sum), where any q
// matches: the update's part of the gradient at a row the next step samples.
// One warp per position p, Sprev staged in shared memory, 32 positions q per
// ballot.
constexpr int REP_WARPS = 8;

__global__ void __launch_bounds__(REP_WARPS * 32)
    defer_repeat_kernel(const int32_t *S, int64_t cnt, const int32_t *Sprev, const double *dprev, int cprev,
                        double diag, const double *add, double *acc)
{
    __shared__ int32_t sp[UPD_MAX];
    for (int q = threadIdx.x; q < cprev; q += blockDim.x) sp[q] = Sprev[q];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * REP_WARPS + (threadIdx.x >> 5);
    if (p >= cnt) return;  // warp-uniform
    const int32_t key = S[p];
    double sum = 0.0;
    bool any = false;
    for (int q0 = 0; q0 < cprev; q0 += 32) {
        const int q = q0 + lane;
        unsigned hit = __ballot_sync(0xffffffffu, q < cprev && sp[q] == key);
        any = any || hit != 0u;
        while (hit) {  // rare: the matches in position order (every lane the same sum)
            sum += dprev[q0 + __ffs(hit) - 1];
            hit &= hit - 1u;
        }
    }
    if (lane == 0) {
        double v = acc[p];
        if (add) v += add[p];
        if (any) v += diag * sum;
        acc[p] = v;
    }
}

cudaError_t launch_defer_repeat(const int32_t *S, int64_t cnt, const int32_t *Sprev, const double *dprev,
                                int64_t cprev, double diag, const double *add, double *acc, cudaStream_t st)
{
    if (cnt <= 0) return cudaSuccess;
    if (cprev > UPD_MAX) return cudaErrorInvalidValue;
    defer_repeat_kernel<<<(unsigned)((cnt + REP_WARPS - 1) / REP_WARPS), REP_WARPS * 32, 0, st>>>(
        S, cnt, Sprev, dprev, (int)cprev, diag, add, acc);
    return cudaGetLastError();
}

cudaError_t launch_update(const int32_t *S, const double *delta, int64_t cnt, double diag, double *alpha, double *g,
                          uint64_t *ctr, uint64_t ctr_advance, int64_t m, int *err, cudaStream_t st, bool pdl,
                          int prio)
{
    if (cnt <= 0) return cudaSuccess;
    if (cnt > UPD_MAX) return cudaErrorInvalidValue;
    int64_t blocks = (cnt + UPD_WARPS - 1) / UPD_WARPS;
    if (blocks > 152) blocks = 152;
    if (!pdl && !prio) {
        update_kernel<<<(unsigned)blocks, UPD_WARPS * 32, 0, st>>>(S, delta, (int)cnt, diag, alpha, g, ctr,
                                                                   ctr_advance, m, err);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks, 1, 1);
    cfg.blockDim = dim3(UPD_WARPS * 32, 1, 1);
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    unsigned na = 0;
    if (pdl) {
        at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[na++].val.programmaticStreamSerializationAllowed = 1;
    }
    if (prio) {
        at[na].id = cudaLaunchAttributePriority;
        at[na++].val.priority = prio;
    }
    cfg.attrs = at;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, update_kernel, S, delta, (int)cnt, diag, alpha, g, ctr, ctr_advance, m, err);
}

// -------------------------------------------------------- convergence ----
// Partial sums over a fixed partition of [0, m), then one block combines the
// partials in index order, so the result is reproducible.
//   K-RR:  r[0] = ||g||^2
//   K-SVM: with (Q a)_i = g_i + 1 - omega a_i:
//          r[0] = a^T Q a, r[1] = sum a, r[2] = ||a||^2, r[3] = sum max(0, 1-(Qa)_i)^p
constexpr int CHECK_BLOCKS = 256;
constexpr int CHECK_THREADS = 256;

__global__ void check_partial_kernel(int problem, const double *g, const double *alpha, int64_t m, double C, int loss,
                                     double *partials)
{
    __shared__ double red[4][CHECK_THREADS];
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    const double omega = (loss == 2) ? 1.0 / (2.0 * C) : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        double gi = g[i];
        if (problem == 1) {
            s0 += gi * gi;
        } else {
            double a = alpha[i];
            double qa = gi + 1.0 - omega * a;
            double xi = fmax(0.0, 1.0 - qa);
            s0 += a * qa;
            s1 += a;
            s2 += a * a;
            s3 += (loss == 1) ? xi : xi * xi;
        }
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    red[2][threadIdx.x] = s2;
    red[3][threadIdx.x] = s3;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) partials[blockIdx.x * 4 + threadIdx.x] = red[threadIdx.x][0];
}

// one warp per quantity: each lane sums a fixed strided subset of the
// partials, then a fixed shuffle tree (FP64 adds have a 64-cycle latency, so
// a serial loop over the partials would dominate the check)
__global__ void check_final_kernel(const double *partials, int nblocks, double *result)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= 4) return;
    double s0 = 0.0, s1 = 0.0;
    int b = lane;
    for (; b + 32 < nblocks; b += 64) {
        s0 += partials[b * 4 + w];
        s1 += partials[(b + 32) * 4 + w];
    }
    if (b < nblocks) s0 += partials[b * 4 + w];
    double s = s0 + s1;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) result[w] = s;
}

cudaError_t launch_check(int problem, const double *g, const double *alpha, const double *y, int64_t m, double C,
                         int loss, double *partials, double *result, cudaStream_t st)
{
    (void)y;
    check_partial_kernel<<<CHECK_BLOCKS, CHECK_THREADS, 0, st>>>(problem, g, alpha, m, C, loss, partials);
    check_final_kernel<<<1, 128, 0, st>>>(partials, CHECK_BLOCKS, result);
    return cudaGetLastError();
}

}  // namespace dcd
