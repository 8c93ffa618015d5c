// static_scratch.cu -- dcd_kernel_block_static: the sampled kernel block of
// dcd_kernel_block computed without allocating any device memory.
//
// Some callers cannot allocate device memory at the point where they need a
// kernel block: a framework that has reserved the device's memory for its own
// caching pool (an extra cudaMalloc can fail, or force the pool to release
// cached blocks), or a deployment whose policy forbids dynamic device
// allocation once start-up is over (cudaMalloc / cudaFree can also
// synchronise the device and stall unrelated work).  This entry point serves
// them: its scratch -- the packed row and column operands, their norm terms
// and the error word -- lives in one file-scope device array of fixed size,
// DCD_STATIC_SCRATCH_BYTES, which every GPU that loads the library holds
// until the process exits.  The caller still provides rows, cols and out.
//
// The array's device address is looked up once per device
// (cudaGetSymbolAddress) on the first call made with that device current; the
// host-side name of the array is only a stand-in and is never passed to a
// kernel.  That first lookup is also when the CUDA runtime may load this
// file's module and commit the array's memory (lazy module loading), so a
// caller that must not allocate later makes one call at start-up -- an empty
// request (nrows or ncols 0) is enough -- before its pool reserves the
// device's memory and before any stream capture.  The cached address belongs
// to the device's primary context (the one the runtime and PyTorch use); it
// is not valid after cudaDeviceReset or under another driver context.  All
// calls share the array: each call clears what must start at zero, and two
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it.
#include "dcd_internal.cuh"

#include <mutex>

namespace dcd {
namespace {

static __device__ __align__(256) unsigned char g_static_scratch[DCD_STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_lookup_mutex;
void *g_scratch_addr[MAX_DEVICES] = {};

// Device address of g_static_scratch on the current device (looked up once).
cudaError_t scratch_address(void **addr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_lookup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        if (!p) return cudaErrorInvalidSymbol;
        g_scratch_addr[dev] = p;
    }
    *addr = g_scratch_addr[dev];
    return cudaSuccess;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

dcd_status to_status(cudaError_t e)
{
    if (e == cudaSuccess) return DCD_OK;
    if (e == cudaErrorMemoryAllocation) return DCD_ENOMEM;
    return DCD_ECUDA;
}

#define STATIC_TRY(expr)                               \
    do {                                               \
        cudaError_t e_ = (expr);                       \
        if (e_ != cudaSuccess) return to_status(e_);   \
    } while (0)

}  // namespace
}  // namespace dcd

using namespace dcd;

extern "C" dcd_status dcd_kernel_block_static(const dcd_matrix *A, const dcd_kernel *k, int32_t prec,
                                              const int32_t *rows, int64_t nrows, const int32_t *cols, int64_t ncols,
                                              void *out, int64_t ldo, void *stream)
{
    // the argument checks of dcd_kernel_block, then the two requests this entry point does not serve
    dcd_status vs = validate_dense(A);
    if (vs != DCD_OK) return vs;
    if ((vs = validate_kernel(k)) != DCD_OK) return vs;
    if (prec != DCD_PREC_FP64 && prec != DCD_PREC_BF16 && prec != DCD_PREC_TF32 && prec != DCD_PREC_BF16X3 &&
        prec != DCD_PREC_TF32X3 && prec != DCD_PREC_FP8 && prec != DCD_PREC_REFRESH && prec != DCD_PREC_FP16)
        return DCD_EINVAL;
    if (prec == DCD_PREC_REFRESH) return DCD_EUNSUPPORTED;  // an apply-only precision
    if (prec == DCD_PREC_FP16) return DCD_EUNSUPPORTED;     // its per-row scales have no place in the scratch
    if (nrows < 0 || ncols < 0 || !cols || !out || ldo < ncols) return DCD_EINVAL;
    if (!rows && nrows > A->m) return DCD_EINVAL;
    if (A->fmt == DCD_CSR) return DCD_EUNSUPPORTED;  // the CSR block's column map is sized per call
    if (A->dtype == DCD_FP8E4M3 || prec == DCD_PREC_FP8) return DCD_EUNSUPPORTED;
    // the array's address first, so that an empty request makes it resident
    void *base_v = nullptr;
    STATIC_TRY(scratch_address(&base_v));
    if (nrows == 0 || ncols == 0) return DCD_OK;
    const bool tc = prec != DCD_PREC_FP64;
    if (tc && !tc_available()) return DCD_EUNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    const KernelParams kp{k->kind, k->degree, k->gamma, k->coef0};

    // scratch layout and the size check, before touching the device
    const int pk = prec == DCD_PREC_TF32     ? PACK_TF32
                   : prec == DCD_PREC_BF16X3 ? PACK_BF16X3
                   : prec == DCD_PREC_TF32X3 ? PACK_TF32X3
                                             : PACK_BF16;
    const int kb = k_block_elems(pk);
    const int64_t n_pad = (A->n + kb - 1) / kb * kb;
    const size_t rb = (size_t)packed_row_bytes(pk, n_pad);
    const int64_t cpad = (ncols + 255) / 256 * 256;
    size_t off_a = 0, off_b = 0, off_rh = 0, off_ch = 0, need = 256;  // [0, 256): error word
    if (tc) {
        off_a = align_up(need, 1024);
        need = off_a + (size_t)nrows * rb;
        off_b = align_up(need, 1024);
        need = off_b + (size_t)ncols * rb;
        off_rh = align_up(need, 256);
        need = off_rh + sizeof(float) * (size_t)nrows;
        off_ch = align_up(need, 256);
        need = off_ch + sizeof(float) * (size_t)cpad;
    } else if (A->dtype != DCD_F64) {
        off_a = align_up(need, 1024);
        need = off_a + sizeof(double) * (size_t)A->m * (size_t)A->n;
    }
    if (need > (size_t)DCD_STATIC_SCRATCH_BYTES) return DCD_EINVAL;  // larger than the static scratch

    char *base = (char *)base_v;
    int *err = (int *)base;
    STATIC_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    if (!tc) {
        const double *a64 = (const double *)A->values;
        int64_t lda = A->ld;
        if (A->dtype != DCD_F64) {
            double *p = (double *)(base + off_a);
            STATIC_TRY(launch_pack_rows(A->values, A->dtype, A->ld, A->m, A->n, nullptr, p, PACK_F64, A->n, A->m, err,
                                        st));
            a64 = p;
            lda = A->n;
        }
        STATIC_TRY(launch_block_simt_f64(a64, lda, A->m, A->n, kp, rows, nrows, cols, ncols, nullptr, nullptr,
                                         nullptr, (double *)out, ldo, err, st));
    } else {
        void *pa = base + off_a, *pb = base + off_b;
        float *rh = (float *)(base + off_rh), *ch = (float *)(base + off_ch);
        STATIC_TRY(cudaMemsetAsync(ch, 0, sizeof(float) * (size_t)cpad, st));  // column terms past ncols read as 0
        STATIC_TRY(launch_pack_rows(A->values, A->dtype, A->ld, A->m, A->n, rows, pa, pk, n_pad, nrows, err, st));
        STATIC_TRY(launch_pack_rows(A->values, A->dtype, A->ld, A->m, A->n, cols, pb, pk, n_pad, ncols, err, st));
        STATIC_TRY(launch_row_terms(pa, pk, n_pad, nrows, kp, rh, st));
        STATIC_TRY(launch_row_terms(pb, pk, n_pad, ncols, kp, ch, st));
        TcOperand Aop{pa, nrows, n_pad, pk, nullptr, rows}, Bop{pb, ncols, n_pad, pk, nullptr, cols};
        STATIC_TRY(launch_block_tc(Aop, Bop, kp, rh, ch, nullptr, nullptr, nullptr, (float *)out, ldo, nrows, ncols,
                                   err, st));
    }
    int he = 0;
    STATIC_TRY(cudaMemcpyAsync(&he, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    STATIC_TRY(cudaStreamSynchronize(st));
    if (he == DEV_TIMEOUT) return DCD_ETIMEOUT;
    if (he == DEV_BAD_INDEX || he == DEV_BAD_VALUE) return DCD_EINVAL;
    return he ? DCD_EINTERNAL : DCD_OK;
}
