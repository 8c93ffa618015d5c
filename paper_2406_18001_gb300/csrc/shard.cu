// shard.cu -- component entry points of the row-sharded outer step.
//
// With the rows of A (and of y, alpha and the cached gradient g) split over
// ranks, one outer step of Algorithms 2 and 4 needs one exchange: every rank
// draws the same sample S from the counter-based stream; the owner of each
// sampled row contributes that row with g, alpha and y at it; one all-gather
// gives every rank all of them; every rank then forms the sampled Gram and
// runs the recurrence redundantly (the paper's ranks also repeat the s-step
// recurrence, Section 4), applies the kernel block to its own rows
// (dcd_kernel_block_apply_points) and updates its own alpha and g.  The
// exchange moves s*b*(n + 4) words per rank, independent of m, where the
// paper's 1D-column layout reduces an m x s*b block (Section 4, Theorem 2).
//
// The entry points here are the pieces that do not exist in the single-GPU
// plan: the contribution, its assembly after the all-gather, the recurrence
// on gathered values, and the update restricted to a rank's rows.  The
// all-gather itself belongs to the caller (NCCL, or any transport).
#include "dcd_internal.cuh"

#include <cmath>

namespace dcd {
namespace {

constexpr int SH_THREADS = 256;
constexpr int64_t SH_CNT_MAX = 8192;  // sampled positions per outer step

__global__ void iota_kernel(int32_t *out, int64_t count, int64_t start)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) out[i] = (int32_t)(start + i);
}

__device__ __forceinline__ double load_elem(const void *v, int dtype, int64_t off)
{
    if (dtype == DCD_F64) return ((const double *)v)[off];
    if (dtype == DCD_F32) return (double)((const float *)v)[off];
    const uint16_t b = ((const uint16_t *)v)[off];  // bf16: the high half of an fp32
    return (double)__uint_as_float((uint32_t)b << 16);
}

// One CTA per sampled position j: the owner writes [1, g, alpha, y, a_row]
// (the row in FP64, exact from F32 / BF16), every other rank zeros.
__global__ void __launch_bounds__(SH_THREADS)
    contribute_kernel(const void *vals, int dtype, int64_t ld, int64_t mloc, int64_t n, int64_t row0, int64_t m,
                      const int32_t *S, const double *g, const double *alpha, const double *y, double *buf, int *err)
{
    const int64_t j = blockIdx.x;
    const int64_t key = S[j];
    double *dst = buf + j * (n + 4);
    if (key < 0 || key >= m) {
        if (threadIdx.x == 0) set_error(err, DEV_BAD_INDEX);
        for (int64_t c = threadIdx.x; c < n + 4; c += blockDim.x) dst[c] = 0.0;
        return;
    }
    const int64_t r = key - row0;
    const bool own = r >= 0 && r < mloc;
    if (threadIdx.x == 0) {
        dst[0] = own ? 1.0 : 0.0;
        dst[1] = own ? g[r] : 0.0;
        dst[2] = own ? alpha[r] : 0.0;
        dst[3] = own && y ? y[r] : 0.0;
    }
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) dst[4 + c] = own ? load_elem(vals, dtype, r * ld + c) : 0.0;
}

// One CTA per position: the single contribution whose owner flag is set,
// and the first position holding the same row.
__global__ void __launch_bounds__(SH_THREADS)
    assemble_kernel(const double *bufs, int nranks, const int32_t *S, int64_t cnt, int64_t n, double *AS, double *gS,
                    double *aS, double *yS, int32_t *first, int *err)
{
    const int64_t j = blockIdx.x;
    __shared__ int owner;
    if (threadIdx.x == 0 && first) {
        const int32_t key = S[j];
        int64_t q = 0;
        while (S[q] != key) ++q;  // ends at q == j at the latest
        first[j] = (int32_t)q;
    }
    if (threadIdx.x == 0) {
        int who = -1, count = 0;
        for (int p = 0; p < nranks; ++p) {
            const double f = bufs[((int64_t)p * cnt + j) * (n + 4)];
            if (f == 1.0) {
                who = p;
                ++count;
            } else if (f != 0.0) {
                count = 2;  // not a contribution buffer
            }
        }
        if (count != 1) {
            set_error(err, DEV_BAD_INDEX);
            who = -1;
        }
        owner = who;
    }
    __syncthreads();
    const int p = owner;
    const double *src = p >= 0 ? bufs + ((int64_t)p * cnt + j) * (n + 4) : nullptr;
    if (threadIdx.x == 0) {
        gS[j] = src ? src[1] : 0.0;
        aS[j] = src ? src[2] : 0.0;
        if (yS) yS[j] = src ? src[3] : 0.0;
    }
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) AS[j * n + c] = src ? src[4 + c] : 0.0;
}

// Sc[p] = the first position holding S[p]: the gathered values indexed by
// position then serve the recurrence as if indexed by row, repeats included.
__global__ void first_pos_kernel(const int32_t *S, int64_t cnt, int32_t *Sc)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= cnt) return;
    const int32_t key = S[p];
    int64_t q = 0;
    while (S[q] != key) ++q;  // ends at q == p at the latest
    Sc[p] = (int32_t)q;
}

// a6 on this rank's rows: for each distinct sampled row it owns, the changes
// of all its positions summed in position order, then alpha += sum and
// g += diag * sum (the arithmetic of the single-GPU update).
__global__ void shard_update_kernel(const int32_t *S, const double *delta, int64_t cnt, double diag, int64_t row0,
                                    int64_t mloc, double *alpha, double *g)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= cnt) return;
    const int32_t key = S[p];
    const int64_t r = (int64_t)key - row0;
    if (r < 0 || r >= mloc) return;
    for (int64_t q = 0; q < p; ++q)
        if (S[q] == key) return;  // not the first position of this row
    double sum = 0.0;
    for (int64_t q = p; q < cnt; ++q)
        if (S[q] == key) sum += delta[q];
    alpha[r] += sum;
    g[r] += diag * sum;
}

// Scratch of one call, freed (stream-ordered) on return.
struct Scratch {
    void *mem = nullptr;
    cudaStream_t st = nullptr;
    ~Scratch()
    {
        if (mem) cudaFreeAsync(mem, st);
    }
};

dcd_status status_of(cudaError_t e)
{
    if (e == cudaSuccess) return DCD_OK;
    if (e == cudaErrorMemoryAllocation) return DCD_ENOMEM;
    if (e == cudaErrorInvalidValue) return DCD_EINVAL;
    return DCD_ECUDA;
}

#define SH_TRY(expr)                                  \
    do {                                              \
        cudaError_t e_ = (expr);                      \
        if (e_ != cudaSuccess) return status_of(e_);  \
    } while (0)

// Reads the error word and waits for the call's work.
dcd_status finish(int *err, cudaStream_t st)
{
    int he = 0;
    SH_TRY(cudaMemcpyAsync(&he, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SH_TRY(cudaStreamSynchronize(st));
    if (he == DEV_TIMEOUT) return DCD_ETIMEOUT;
    if (he == DEV_BAD_INDEX || he == DEV_BAD_VALUE) return DCD_EINVAL;
    if (he == DEV_NOT_SPD) return DCD_ENOTSPD;
    return he ? DCD_EINTERNAL : DCD_OK;
}

}  // namespace

cudaError_t launch_iota(int32_t *out, int64_t count, int64_t start, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    iota_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(out, count, start);
    return cudaGetLastError();
}

}  // namespace dcd

using namespace dcd;

extern "C" dcd_status dcd_shard_contribute(const dcd_matrix *A, int64_t row0, int64_t m, const int32_t *S, int64_t cnt,
                                           const double *g, const double *alpha, const double *y, double *buf,
                                           void *stream)
{
    dcd_status vs = validate_dense(A);
    if (vs != DCD_OK) return vs;
    if (A->fmt != DCD_DENSE) return DCD_EUNSUPPORTED;
    if (A->dtype == DCD_FP8E4M3) return DCD_EUNSUPPORTED;
    if (row0 < 0 || m < 1 || row0 + A->m > m || m > INT32_MAX) return DCD_EINVAL;
    if (cnt < 0 || cnt > SH_CNT_MAX || (cnt > 0 && (!S || !g || !alpha || !buf))) return DCD_EINVAL;
    if (cnt == 0) return DCD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc;
    sc.st = st;
    SH_TRY(malloc_async(&sc.mem, 256, st));
    int *err = (int *)sc.mem;
    SH_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    contribute_kernel<<<(unsigned)cnt, SH_THREADS, 0, st>>>(A->values, A->dtype, A->ld, A->m, A->n, row0, m, S, g,
                                                            alpha, y, buf, err);
    SH_TRY(cudaGetLastError());
    return finish(err, st);
}

extern "C" dcd_status dcd_shard_assemble(const double *bufs, int32_t nranks, const int32_t *S, int64_t cnt, int64_t n,
                                         double *A_S, double *g_S, double *alpha_S, double *y_S, int32_t *first_pos,
                                         void *stream)
{
    if (nranks < 1 || cnt < 0 || cnt > SH_CNT_MAX || n < 1) return DCD_EINVAL;
    if (cnt > 0 && (!bufs || !A_S || !g_S || !alpha_S || (first_pos && !S))) return DCD_EINVAL;
    if (cnt == 0) return DCD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc;
    sc.st = st;
    SH_TRY(malloc_async(&sc.mem, 256, st));
    int *err = (int *)sc.mem;
    SH_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    assemble_kernel<<<(unsigned)cnt, SH_THREADS, 0, st>>>(bufs, nranks, S, cnt, n, A_S, g_S, alpha_S, y_S, first_pos,
                                                          err);
    SH_TRY(cudaGetLastError());
    return finish(err, st);
}

extern "C" dcd_status dcd_shard_update(const int32_t *S, const double *delta, int64_t cnt, double diag, int64_t row0,
                                       int64_t m_local, double *alpha, double *g, void *stream)
{
    if (cnt < 0 || cnt > SH_CNT_MAX || row0 < 0 || m_local < 0 || !std::isfinite(diag)) return DCD_EINVAL;
    if (cnt > 0 && (!S || !delta || (m_local > 0 && (!alpha || !g)))) return DCD_EINVAL;
    if (cnt == 0 || m_local == 0) return DCD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    shard_update_kernel<<<(unsigned)((cnt + 127) / 128), 128, 0, st>>>(S, delta, cnt, diag, row0, m_local, alpha, g);
    SH_TRY(cudaGetLastError());
    SH_TRY(cudaStreamSynchronize(st));
    return DCD_OK;
}

extern "C" dcd_status dcd_bdcd_recurrence(const void *Kss, int32_t kss_f64, int64_t ldk, const int32_t *S,
                                          int64_t nblk, int32_t b, double lambda, double mdiag, const double *g_S,
                                          double *delta, double *w, void *stream)
{
    if (nblk < 0 || b < 1 || nblk * (int64_t)b > SH_CNT_MAX) return DCD_EINVAL;
    if (!(lambda > 0.0) || !std::isfinite(lambda) || !(mdiag >= 0.0) || !std::isfinite(mdiag)) return DCD_EINVAL;
    const int64_t cnt = nblk * (int64_t)b;
    if (cnt == 0) return DCD_OK;
    if (!Kss || ldk < cnt || !S || !g_S || !delta || (kss_f64 != 0 && kss_f64 != 1)) return DCD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc;
    sc.st = st;
    const size_t lb = recur_bdcd_scratch_bytes(nblk, b);
    const size_t off_sc = 256, off_l = (off_sc + sizeof(int32_t) * (size_t)cnt + 1023) / 1024 * 1024;
    SH_TRY(malloc_async(&sc.mem, off_l + lb, st));
    char *base = (char *)sc.mem;
    int *err = (int *)base;
    int32_t *Sc = (int32_t *)(base + off_sc);
    SH_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    first_pos_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(S, cnt, Sc);
    SH_TRY(cudaGetLastError());
    // the refinement setting of the single-GPU step: adaptive FP64 refinement
    // on an FP64 Gram, one refinement round on an FP32 one
    SH_TRY(launch_recur_bdcd(Kss, kss_f64, ldk, Sc, nblk, b, lambda, mdiag, g_S, kss_f64 ? 2 : 1, base + off_l, delta,
                             w, nullptr, nullptr, err, st));
    return finish(err, st);
}

extern "C" dcd_status dcd_dcd_recurrence(const void *Kss, int32_t kss_f64, int64_t ldk, const int32_t *S, int64_t cnt,
                                         const double *y_S, const double *alpha_S, const double *g_S, int32_t loss,
                                         double C, double *theta, double *w, void *stream)
{
    if (cnt < 0 || cnt > SH_CNT_MAX || (loss != 1 && loss != 2) || !(C > 0.0) || !std::isfinite(C)) return DCD_EINVAL;
    if (cnt == 0) return DCD_OK;
    if (!Kss || ldk < cnt || !S || !y_S || !alpha_S || !g_S || !theta || (kss_f64 != 0 && kss_f64 != 1))
        return DCD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc;
    sc.st = st;
    SH_TRY(malloc_async(&sc.mem, 256 + sizeof(int32_t) * (size_t)cnt, st));
    int *err = (int *)sc.mem;
    int32_t *Sc = (int32_t *)((char *)sc.mem + 256);
    SH_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    first_pos_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(S, cnt, Sc);
    SH_TRY(cudaGetLastError());
    const double omega = loss == 2 ? 1.0 / (2.0 * C) : 0.0, nu = loss == 2 ? INFINITY : C;
    SH_TRY(launch_recur_dcd(Kss, kss_f64, ldk, Sc, cnt, y_S, alpha_S, g_S, omega, nu, theta, w, nullptr, err, st));
    return finish(err, st);
}
