// solver.cu -- host side of libdcd_gb300.so: argument validation, workspace,
// the outer s-step loop and the C-ABI entry points of include/dcd_gb300.h.
//
// One outer step (Algorithm 2 for K-SVM, Algorithm 4 for K-RR), reordered so
// the m x sb block is never stored (its contraction with the step's
// coefficients is all the next steps need):
//   a1 sample  S = s*b indices from the counter-based stream
//   a2 gather  the sampled rows (tensor-core path) and their norms
//   a3 Gram    Kss = K(A_S, A_S), with the same kernel as a5
//   a4 recur   FP64 theta / Delta from Kss and the cached gradient g_S
//   a5 block   g += rs * K(A, A_S) w, fused, for all m rows
//   a6 update  alpha_S += delta, g_S += diag * delta; counter += s
// U_j^T alpha_sk of the paper is read from the cached gradient g, which a5/a6
// keep equal to the gradient of the current alpha.
#include "dcd_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <vector>

namespace dcd {

static bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

dcd_status validate_kernel(const dcd_kernel *k)
{
    if (!k) return DCD_EINVAL;
    switch (k->kind) {
    case DCD_LINEAR: return DCD_OK;
    case DCD_POLY:
        return (std::isfinite(k->coef0) && k->coef0 >= 0.0 && k->degree >= 2 && k->degree <= 32) ? DCD_OK : DCD_EINVAL;
    case DCD_RBF: return finite_pos(k->gamma) ? DCD_OK : DCD_EINVAL;
    default: return DCD_EINVAL;
    }
}

// Dense: row-major f64/f32/bf16, or e4m3 codes with per-row scales, with
// ld >= n.  CSR: f32/f64 values, int64 row offsets, int32 columns (checked on
// the device by the solver).
dcd_status validate_dense(const dcd_matrix *A)
{
    if (!A || A->m < 1 || A->n < 1) return DCD_EINVAL;
    if (A->fmt == DCD_CSR) {
        if (!A->row_ptr || !A->col_idx || !A->values) return DCD_EINVAL;
        if (A->dtype == DCD_BF16 || A->dtype == DCD_FP8E4M3) return DCD_EUNSUPPORTED;
        if (A->dtype != DCD_F64 && A->dtype != DCD_F32) return DCD_EINVAL;
        if (A->m > INT32_MAX || A->n > INT32_MAX) return DCD_EINVAL;
        return DCD_OK;
    }
    if (A->fmt != DCD_DENSE) return DCD_EINVAL;
    if (A->dtype != DCD_F64 && A->dtype != DCD_F32 && A->dtype != DCD_BF16 && A->dtype != DCD_FP8E4M3)
        return DCD_EINVAL;
    if (A->dtype == DCD_FP8E4M3 && !A->row_scale) return DCD_EINVAL;
    if (A->ld < A->n || !A->values) return DCD_EINVAL;
    if (A->m > INT32_MAX) return DCD_EINVAL;
    return DCD_OK;
}

namespace {

// The transposed copy of a CSR operand and the per-step scratch of the apply
// through it, kept when a step's incidences -- expected jc * (nnz / m) *
// sum_c nnz_c^2 / nnz per chunk of jc sampled rows whose columns follow the
// nonzeros -- stay below nnz / 16 (an incidence costs about 16 times the full
// pass's 4 bytes per nonzero); else nothing is kept.  maxcol_dev: one device
// int of scratch.
dcd_status csc_choose(const CsrOperand &ca, bool fp64, int64_t cnt, int maxrow, int *maxcol_dev, void **ws_csc,
                      CscOperand *C, void **ws_step, CscStep *W, CsrColMap *M, bool *use, cudaStream_t st);

constexpr int64_t SB_MAX = 8192;   // s*b per outer step
constexpr int B_MAX = 128;         // block size
constexpr int DF_XPAIRS = 8;       // CTA pairs (at most) of the deferred gradient's cross product
constexpr int DF_GRAM_CTAS = 8;    // CTAs of the Gram computed beside the deferred step's block

// Set while the batched driver and the autotuner build their plans: those
// capture many plans' steps into one graph and run without the look-ahead.
thread_local bool t_no_lookahead = false;
struct NoLookahead {
    bool prev = t_no_lookahead;
    NoLookahead() { t_no_lookahead = true; }
    ~NoLookahead() { t_no_lookahead = prev; }
};

struct Arena {
    char *base = nullptr;
    size_t used = 0, cap = 0;
    void *take(size_t bytes, size_t align = 256)
    {
        size_t off = (used + align - 1) / align * align;
        used = off + bytes;
        return base ? base + off : nullptr;
    }
};

dcd_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return DCD_OK;
    if (e == cudaErrorMemoryAllocation) return DCD_ENOMEM;
    return DCD_ECUDA;
}

#define DCD_TRY(expr)                                   \
    do {                                                \
        cudaError_t e_ = (expr);                        \
        if (e_ != cudaSuccess) return cuda_status(e_);  \
    } while (0)

dcd_status csc_choose(const CsrOperand &ca, bool fp64, int64_t cnt, int maxrow, int *maxcol_dev, void **ws_csc,
                      CscOperand *C, void **ws_step, CscStep *W, CsrColMap *M, bool *use, cudaStream_t st)
{
    *use = false;
    const int64_t jc = std::min<int64_t>(cnt, 32);
    const int64_t m = ca.m, n = ca.n;
    if (ca.nnz <= 0 || m <= 0 || jc <= 0) return DCD_OK;
    DCD_TRY(malloc_async(ws_csc, csc_bytes(n, ca.nnz, fp64), st));
    DCD_TRY(launch_csc_build(ca, fp64, *ws_csc, C, maxcol_dev, st));
    std::vector<int64_t> cp((size_t)n + 1);
    DCD_TRY(cudaMemcpyAsync(cp.data(), C->col_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st));
    DCD_TRY(cudaStreamSynchronize(st));
    double sq = 0.0;
    for (int64_t c = 0; c < n; ++c) {
        const double k = (double)(cp[c + 1] - cp[c]);
        sq += k * k;
    }
    const double nnzd = (double)ca.nnz;
    const double expect = (double)jc * (nnzd / (double)m) * (sq / nnzd);
    if (16.0 * expect > nnzd) {
        DCD_TRY(cudaFreeAsync(*ws_csc, st));
        *ws_csc = nullptr;
        return DCD_OK;
    }
    const size_t sbytes = csc_step_bytes(m, cnt, maxrow, fp64);
    DCD_TRY(malloc_async(ws_step, sbytes, st));
    DCD_TRY(cudaMemsetAsync(*ws_step, 0, sbytes, st));
    *W = csc_step_carve(*ws_step, m, cnt, maxrow, *C, M);
    *use = true;
    return DCD_OK;
}

size_t dtype_size(int dt) { return dt == DCD_F64 ? 8 : dt == DCD_F32 ? 4 : dt == DCD_BF16 ? 2 : 1; }

KernelParams to_kp(const dcd_kernel *k) { return KernelParams{k->kind, k->degree, k->gamma, k->coef0}; }

bool is_tc(int prec)
{
    return prec == DCD_PREC_BF16 || prec == DCD_PREC_TF32 || prec == DCD_PREC_BF16X3 || prec == DCD_PREC_TF32X3 ||
           prec == DCD_PREC_FP8 || prec == DCD_PREC_FP16;
}

// packed operand kind of a tensor-core precision
int pack_kind(int prec)
{
    return prec == DCD_PREC_TF32 ? PACK_TF32
           : prec == DCD_PREC_BF16X3 ? PACK_BF16X3
           : prec == DCD_PREC_TF32X3 ? PACK_TF32X3
           : prec == DCD_PREC_FP8    ? PACK_FP8
           : prec == DCD_PREC_FP16   ? PACK_FP16
                                     : PACK_BF16;
}

// Operand preparation shared by the solver and the component entry points.
struct Operand {
    // FP64 path
    const double *a64 = nullptr;
    int64_t lda = 0;
    // tensor-core path
    void *packed = nullptr;
    int64_t n_pad = 0;
    int kind = PACK_BF16;
    float *row_h = nullptr;
    float *row_s = nullptr;  // PACK_FP8, PACK_FP16: per-row scales
};

// Per-phase device times of an outer step: an event pair per phase, recorded
// back to back on the solver's stream, one synchronisation per step (flush).
struct EventTimer {
    static constexpr int MAXP = 8;
    bool on = false;
    cudaStream_t st = nullptr;
    cudaEvent_t ev[2 * MAXP] = {};
    double *acc[MAXP] = {};
    int n = 0;
    void init(bool enable, cudaStream_t s)
    {
        on = enable;
        st = s;
        if (on)
            for (auto &e : ev) cudaEventCreate(&e);
    }
    void start()
    {
        if (on && n < MAXP) cudaEventRecord(ev[2 * n], st);
    }
    void stop(double &a)
    {
        if (!on || n >= MAXP) return;
        cudaEventRecord(ev[2 * n + 1], st);
        acc[n++] = &a;
    }
    void flush()
    {
        if (!on || n == 0) return;
        cudaEventSynchronize(ev[2 * n - 1]);
        for (int i = 0; i < n; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
            *acc[i] += ms;
        }
        n = 0;
    }
    ~EventTimer()
    {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
};

struct Solver {
    // problem
    int problem = 0;  // 0: K-SVM (DCD), 1: K-RR (BDCD)
    const dcd_matrix *A = nullptr;
    KernelParams kp{};
    int loss = 1;
    double C = 1.0, lambda = 1.0, omega = 0.0, nu = 0.0, diag = 0.0;
    dcd_opts o{};
    cudaStream_t st = nullptr;
    int64_t m = 0, n = 0;
    bool tc = false;
    // caller / device arrays
    const double *y = nullptr;
    double *alpha = nullptr, *grad_out = nullptr;
    double *g = nullptr;
    // workspace
    void *ws = nullptr;
    Operand op;
    // the operand (and column buffers) of the recomputed gradient: split tf32
    // for the tensor-core modes (== op when the solve itself is split tf32)
    Operand opr;
    TcSplit tsplit;  // scratch of the balanced tensor-core apply
    void *Asr = nullptr;
    float *col_hr = nullptr;
    // literal-order steps (DCD_FLAG_LITERAL): the stored block, the U^T alpha partial sums and
    // the step's gradient values (at their positions)
    bool literal = false;
    void *Qbuf = nullptr;
    double *lit_part = nullptr, *lit_g = nullptr;
    int64_t lit_blocks = 0;
    // the accurate epilogue of the recomputed gradient: low parts of the RBF terms, and the
    // gathered columns' power-of-two scales of the sliced operand
    float *row_hlr = nullptr, *col_hlr = nullptr, *col_sr = nullptr;
    // CSR data matrix: the CUDA-core SpMM block (FP32, or FP64 in the FP64 mode)
    bool csr = false;
    CsrOperand ca;
    CsrColMap cm;
    void *ws_csr = nullptr;
    CsrColMap cm_set[3];     // the column map of each buffer set (the K-SVM look-ahead)
    void *ws_csr2[2] = {nullptr, nullptr};
    // the apply through the transposed copy (chosen at set-up when it reads far less than a full pass)
    bool use_csc = false;
    CscOperand cscop;
    CscStep cstep;
    void *ws_csc = nullptr, *ws_cstep = nullptr;
    int csr_maxrow = 0;
    // the first chunk's scatter runs on csr_st beside the Gram and the recurrence
    cudaStream_t csr_st = nullptr;
    cudaEvent_t csr_fork = nullptr, csr_join = nullptr;
    void *As = nullptr;           // packed sampled rows (tc)
    float *col_h = nullptr, *col_w = nullptr;
    float *col_s = nullptr;       // fp8, fp16: scales of the sampled rows
    const float *src_scale = nullptr;  // the row scales of an FP8 data matrix (device)
    int32_t *S = nullptr;
    void *Kss = nullptr;
    int64_t ldk = 0;
    double *delta = nullptr, *w64 = nullptr, *Lbuf = nullptr;
    uint64_t *ctr = nullptr;
    int *err = nullptr, *flag = nullptr;
    double *partials = nullptr, *result = nullptr;
    int32_t *iota = nullptr;
    // host-io copies
    void *h_vals = nullptr;
    int64_t sb = 0, col_pad = 0;
    dcd_stats stats{};

    ~Solver()
    {
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        for (auto &ge : graph_la)
            if (ge) cudaGraphExecDestroy(ge);
        if (st2) {
            cudaStreamSynchronize(st2);
            cudaStreamDestroy(st2);
        }
        if (la_fork) cudaEventDestroy(la_fork);
        if (la_join) cudaEventDestroy(la_join);
        for (auto &ge : graph_df)
            if (ge) cudaGraphExecDestroy(ge);
        for (cudaStream_t sx : {st3, st4})
            if (sx) {
                cudaStreamSynchronize(sx);
                cudaStreamDestroy(sx);
            }
        for (cudaEvent_t ev : {df_fork, df_chained, df_rows, df_gram, df_side, df_xfork, df_xjoin, df_kx})
            if (ev) cudaEventDestroy(ev);
        if (ws_csr) cudaFreeAsync(ws_csr, st);
        for (void *w : ws_csr2)
            if (w) cudaFreeAsync(w, st);
        if (csr_st) {
            cudaStreamSynchronize(csr_st);
            cudaStreamDestroy(csr_st);
        }
        if (csr_fork) cudaEventDestroy(csr_fork);
        if (csr_join) cudaEventDestroy(csr_join);
        if (ws_csc) cudaFreeAsync(ws_csc, st);
        if (ws_cstep) cudaFreeAsync(ws_cstep, st);
        if (ws) cudaFreeAsync(ws, st);
    }

    dcd_status check_device_error()
    {
        int e = 0;
        DCD_TRY(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        DCD_TRY(cudaStreamSynchronize(st));
        switch (e) {
        case DEV_OK: return DCD_OK;
        case DEV_TIMEOUT: return DCD_ETIMEOUT;
        case DEV_NOT_SPD: return DCD_ENOTSPD;
        case DEV_BAD_VALUE: return DCD_EINVAL;
        default: return DCD_EINTERNAL;
        }
    }

    dcd_status setup(const double *y_in, double *alpha_in, double *grad_in)
    {
        m = A->m;
        n = A->n;
        tc = is_tc(o.prec);
        csr = A->fmt == DCD_CSR;
        const bool host = (o.flags & DCD_FLAG_HOST_IO) != 0;
        int64_t nnz = 0;
        if (csr) {
            if (host) {
                nnz = A->row_ptr[m];
            } else {
                DCD_TRY(cudaMemcpyAsync(&nnz, A->row_ptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
                DCD_TRY(cudaStreamSynchronize(st));
            }
            if (nnz < 0) return DCD_EINVAL;
        }
        const bool tcd = tc && !csr;  // packed tensor-core operand (dense only)
        // CSR values in the block's type: FP32 (tensor-core precisions) or FP64
        const bool conv32 = csr && tc && A->dtype != DCD_F32, conv64 = csr && !tc && A->dtype != DCD_F64;
        sb = (int64_t)o.s * o.b;
        col_pad = (sb + 255) / 256 * 256;
        const int kb_elems = k_block_elems(pack_kind(o.prec));
        const int64_t n_pad = (n + kb_elems - 1) / kb_elems * kb_elems;
        const size_t row_bytes = tcd ? (size_t)packed_row_bytes(pack_kind(o.prec), n_pad) : 8 * (size_t)n;
        const bool need_pack = !csr && (tc || A->dtype != DCD_F64 || host);
        // the recomputed gradient (DCD_FLAG_REFRESH): sliced operand (exact products) for n up to
        // SLICED_N_MAX, split tf32 beyond; accurate epilogue either way
        const bool acc_ref = tcd && (o.flags & DCD_FLAG_REFRESH);
        const bool sliced_ref = acc_ref && (n + 63) / 64 * 64 <= SLICED_N_MAX;
        const bool ref_op = acc_ref && (sliced_ref || o.prec != DCD_PREC_TF32X3);
        const int kind_r = sliced_ref ? PACK_SLICED : PACK_TF32X3;
        const bool fp8 = tcd && pack_kind(o.prec) == PACK_FP8;
        const bool fp16 = tcd && pack_kind(o.prec) == PACK_FP16;
        const bool scaled = fp8 || fp16;  // per-row scales beside the packed rows
        const bool fp8in = !csr && A->dtype == DCD_FP8E4M3;
        // the look-ahead needs a stream of its own to fork from, graphs allowed, no per-phase
        // timers, and a full step that fits one cluster recurrence
        literal = (o.flags & DCD_FLAG_LITERAL) != 0;
        lit_blocks = literal ? std::min<int64_t>(std::max<int64_t>(1, (m + 255) / 256), 1024) : 0;
        const bool la_pos = !t_no_lookahead && problem == 1 && tcd && !literal &&
                            !(o.flags & (DCD_FLAG_NO_GRAPH | DCD_FLAG_PHASE_TIMERS)) && st != nullptr &&
                            st != cudaStreamLegacy && st != cudaStreamPerThread &&
                            recur_cluster_size((int)o.s, o.b, 2) > 0;
        const bool df_pos = la_pos && !(o.flags & DCD_FLAG_NO_DEFER);
        // the look-ahead of the other steps (K-SVM, dense or CSR; K-RR in FP64, on CSR or with a
        // chain longer than one cluster): the next step's sample, column map or gathers and Gram
        // on a second stream beside the recurrence and block
        const bool lag_pos = !t_no_lookahead && !la_pos && !literal &&
                             !(o.flags & (DCD_FLAG_NO_GRAPH | DCD_FLAG_PHASE_TIMERS)) && st != nullptr &&
                             st != cudaStreamLegacy && st != cudaStreamPerThread;
        const bool set2 = la_pos || lag_pos;  // a second set of step buffers
        // the deferred K-SVM step (the recurrence one step ahead of the block): a step the one-block
        // recurrence takes
        const bool dfs_pos = lag_pos && problem == 0 && o.b == 1 && o.s <= 128 && !(o.flags & DCD_FLAG_NO_DEFER);
        const bool set3 = df_pos || dfs_pos;  // a third set
        const int64_t n_pad_r = sliced_ref ? (n + 63) / 64 * 64 : (n + 31) / 32 * 32;
        const size_t row_bytes_r = ref_op ? (size_t)packed_row_bytes(kind_r, n_pad_r) : 0;

        int split_pairs = 0;
        const int split_chunks = tc_split_chunks(std::max<int64_t>(sb, 1));
        if (tcd) {
            int dev = 0, sms = 0;
            DCD_TRY(cudaGetDevice(&dev));
            DCD_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            split_pairs = std::max(sms / 2, 1);
        }
        // size the arena (two passes over the same layout)
        Arena ar;
        for (int pass = 0; pass < 2; ++pass) {
            ar.used = 0;
            char *hv = (char *)ar.take(host ? (csr ? (size_t)nnz : (size_t)m * A->ld) * dtype_size(A->dtype) : 0, 1024);
            int64_t *hrp = (int64_t *)ar.take(host && csr ? sizeof(int64_t) * (m + 1) : 0);
            int32_t *hci = (int32_t *)ar.take(host && csr ? sizeof(int32_t) * nnz : 0);
            float *cv32 = (float *)ar.take(conv32 ? sizeof(float) * nnz : 0);
            double *cv64 = (double *)ar.take(conv64 ? sizeof(double) * nnz : 0);
            float *hsc = (float *)ar.take(host && fp8in ? sizeof(float) * m : 0);
            float *rsc = (float *)ar.take(scaled ? sizeof(float) * m : 0);
            float *csc = (float *)ar.take(scaled ? sizeof(float) * col_pad : 0);
            float *nrm32 = (float *)ar.take(csr ? sizeof(float) * m : 0);
            double *nrm64 = (double *)ar.take(csr ? sizeof(double) * m : 0);
            double *yv = (double *)ar.take(host ? sizeof(double) * m : 0);
            double *av = (double *)ar.take(host ? sizeof(double) * m : 0);
            double *gv = (double *)ar.take(sizeof(double) * m);
            void *pk = ar.take(need_pack ? (size_t)m * row_bytes : 0, 1024);
            float *rh = (float *)ar.take(tcd ? sizeof(float) * m : 0);
            void *as = ar.take(tcd ? (size_t)sb * row_bytes : 0, 1024);
            float *ch = (float *)ar.take(sizeof(float) * col_pad);
            float *cw = (float *)ar.take(sizeof(float) * col_pad);
            void *pkr = ar.take((size_t)m * row_bytes_r, 1024);
            float *rhr = (float *)ar.take(ref_op ? sizeof(float) * m : 0);
            void *asr = ar.take((size_t)sb * row_bytes_r, 1024);
            float *chr = (float *)ar.take(ref_op ? sizeof(float) * col_pad : 0);
            float *rhl = (float *)ar.take(acc_ref ? sizeof(float) * m : 0);
            float *chl = (float *)ar.take(acc_ref ? sizeof(float) * col_pad : 0);
            float *rscr = (float *)ar.take(sliced_ref ? sizeof(float) * m : 0);
            float *cscr = (float *)ar.take(sliced_ref ? sizeof(float) * col_pad : 0);
            int32_t *sidx = (int32_t *)ar.take(sizeof(int32_t) * col_pad);
            void *kss = ar.take((size_t)sb * sb * (tc ? 4 : 8));
            double *dl = (double *)ar.take(sizeof(double) * col_pad);
            double *wv = (double *)ar.take(sizeof(double) * col_pad);
            double *lb = (double *)ar.take(problem == 1 ? recur_bdcd_scratch_bytes(o.s, o.b) : 0);
            uint64_t *cr = (uint64_t *)ar.take(sizeof(uint64_t));
            // the second set of step buffers and the look-ahead counter
            int32_t *sidx_b = (int32_t *)ar.take(set2 ? sizeof(int32_t) * col_pad : 0);
            void *as_b = ar.take(set2 && tcd ? (size_t)sb * row_bytes : 0, 1024);
            float *ch_b = (float *)ar.take(set2 ? sizeof(float) * col_pad : 0);
            float *cs_b = (float *)ar.take(set2 && scaled ? sizeof(float) * col_pad : 0);
            void *kss_b = ar.take(set2 ? (size_t)sb * sb * (tc ? 4 : 8) : 0);
            double *lb_b = (double *)ar.take(la_pos ? recur_bdcd_scratch_bytes(o.s, o.b) : 0);
            uint64_t *crl = (uint64_t *)ar.take(set2 ? 3 * sizeof(uint64_t) : 0);
            // the deferred gradient: a third set, the recurrence's outputs per set, x per set and the
            // cross product's split
            int32_t *sidx_c = (int32_t *)ar.take(set3 ? sizeof(int32_t) * col_pad : 0);
            void *as_c = ar.take(set3 && tcd ? (size_t)sb * row_bytes : 0, 1024);
            float *ch_c = (float *)ar.take(set3 ? sizeof(float) * col_pad : 0);
            float *cs_c = (float *)ar.take(set3 && scaled ? sizeof(float) * col_pad : 0);
            void *kss_c = ar.take(set3 ? (size_t)sb * sb * (tc ? 4 : 8) : 0);
            double *lb_c = (double *)ar.take(df_pos ? recur_bdcd_scratch_bytes(o.s, o.b) : 0);
            double *dfd = (double *)ar.take(set3 ? 4 * sizeof(double) * col_pad : 0);  // delta, w64 of sets 1, 2
            float *dfw = (float *)ar.take(set3 ? 2 * sizeof(float) * col_pad : 0);     // col_w of sets 1, 2
            // the deferred K-SVM step: per set alpha and g at its rows (snapshot, pending parts), and
            // the kernel values of the step after next's rows against the next step's
            double *dsn = (double *)ar.take(dfs_pos ? 12 * sizeof(double) * col_pad : 0);
            void *dkx = ar.take(dfs_pos ? (size_t)sb * sb * (tc ? 4 : 8) : 0);
            double *dfx = (double *)ar.take(df_pos ? 4 * sizeof(double) * col_pad : 0);  // x of sets 0-2, x2
            double *xsp =
                (double *)ar.take(df_pos ? 2 * sizeof(double) * tc_split_part_elems(DF_XPAIRS, split_chunks) : 0);
            unsigned *xsc = (unsigned *)ar.take(df_pos ? 2 * sizeof(unsigned) * 2 * DF_XPAIRS : 0);
            // the balanced split of the tensor-core apply over CTA pairs
            double *tsp = (double *)ar.take(tcd ? sizeof(double) * tc_split_part_elems(split_pairs, split_chunks) : 0);
            unsigned *tsc = (unsigned *)ar.take(tcd ? sizeof(unsigned) * 2 * split_pairs : 0);
            int *er = (int *)ar.take(sizeof(int) * 8);
            double *pt = (double *)ar.take(sizeof(double) * 4 * 256);
            double *rs = (double *)ar.take(sizeof(double) * 4);
            int64_t ichunk = std::min<int64_t>(m, SB_MAX);
            int32_t *io = (int32_t *)ar.take(sizeof(int32_t) * ichunk);
            void *qb = ar.take(literal ? (size_t)m * sb * (tc ? 4 : 8) : 0, 1024);
            double *lpart = (double *)ar.take(literal ? sizeof(double) * lit_blocks * col_pad : 0);
            double *lg = (double *)ar.take(literal ? sizeof(double) * m : 0);
            if (pass == 0) {
                cudaError_t e = malloc_async(&ws, ar.used + 1024, st);
                if (e != cudaSuccess) return cuda_status(e);
                ar.base = (char *)ws;
                continue;
            }
            h_vals = hv;
            if (csr) {
                ca.row_ptr = host ? hrp : A->row_ptr;
                ca.col_idx = host ? hci : A->col_idx;
                const void *v = host ? (const void *)hv : A->values;
                ca.vals32 = conv32 ? cv32 : (A->dtype == DCD_F32 ? (const float *)v : nullptr);
                ca.vals64 = conv64 ? cv64 : (A->dtype == DCD_F64 ? (const double *)v : nullptr);
                if (tc) ca.vals64 = nullptr;  // the FP32 block reads vals32
                ca.m = m;
                ca.n = n;
                ca.nnz = nnz;
                ca.norm32 = nrm32;
                ca.norm64 = nrm64;
                if (host) {
                    DCD_TRY(cudaMemcpyAsync(hrp, A->row_ptr, sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice, st));
                    DCD_TRY(cudaMemcpyAsync(hci, A->col_idx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
                }
            }
            g = gv;
            op.packed = pk;
            op.row_h = rh;
            op.row_s = rsc;
            col_s = csc;
            src_scale = fp8in ? (host ? hsc : A->row_scale) : nullptr;
            if (host && fp8in)
                DCD_TRY(cudaMemcpyAsync(hsc, A->row_scale, sizeof(float) * m, cudaMemcpyHostToDevice, st));
            As = as;
            col_h = ch;
            col_w = cw;
            opr.packed = pkr;
            opr.row_h = rhr;
            Asr = asr;
            col_hr = chr;
            row_hlr = rhl;
            col_hlr = chl;
            opr.row_s = rscr;
            col_sr = cscr;
            S = sidx;
            Kss = kss;
            ldk = sb;
            delta = dl;
            w64 = wv;
            Lbuf = lb;
            ctr = cr;
            err = er;
            flag = er + 1;
            partials = pt;
            result = rs;
            iota = io;
            Qbuf = qb;
            lit_part = lpart;
            lit_g = lg;
            sbuf[0].S = sidx;
            sbuf[0].As = as;
            sbuf[0].col_h = ch;
            sbuf[0].col_s = csc;
            sbuf[0].Kss = kss;
            sbuf[0].Lbuf = lb;
            sbuf[1].S = sidx_b;
            sbuf[1].As = as_b;
            sbuf[1].col_h = ch_b;
            sbuf[1].col_s = cs_b;
            sbuf[1].Kss = kss_b;
            sbuf[1].Lbuf = la_pos ? lb_b : lb;  // off the cluster path only the main stream uses the scratch
            sbuf[2].S = sidx_c;
            sbuf[2].As = as_c;
            sbuf[2].col_h = ch_c;
            sbuf[2].col_s = cs_c;
            sbuf[2].Kss = kss_c;
            sbuf[2].Lbuf = lb_c;
            sbuf[0].delta = dl;
            sbuf[0].w64 = wv;
            sbuf[0].col_w = cw;
            if (set3)
                for (int q = 1; q < 3; ++q) {
                    sbuf[q].delta = dfd + (size_t)(2 * q - 2) * col_pad;
                    sbuf[q].w64 = dfd + (size_t)(2 * q - 1) * col_pad;
                    sbuf[q].col_w = dfw + (size_t)(q - 1) * col_pad;
                }
            for (int q = 0; q < 3; ++q) df_x[q] = df_pos ? dfx + (size_t)q * col_pad : nullptr;
            for (int q = 0; q < 3; ++q)
                for (int k = 0; k < 4; ++k) dfs_v[q][k] = dfs_pos ? dsn + (size_t)(4 * q + k) * col_pad : nullptr;
            dfs_kx = dkx;
            df_x2 = df_pos ? dfx + 3 * (size_t)col_pad : nullptr;
            xsplit2.part = df_pos ? xsp + tc_split_part_elems(DF_XPAIRS, split_chunks) : nullptr;
            xsplit2.cnt = df_pos ? xsc + 2 * DF_XPAIRS : nullptr;
            xsplit2.pairs = df_pos ? DF_XPAIRS : 0;
            xsplit.part = xsp;
            xsplit.cnt = xsc;
            xsplit.pairs = df_pos ? DF_XPAIRS : 0;
            xsplit.chunks = df_pos ? split_chunks : 0;
            xsplit2.chunks = df_pos ? split_chunks : 0;
            ctr_la = crl;
            if (tcd) {
                tsplit.part = tsp;
                tsplit.cnt = tsc;
                tsplit.pairs = split_pairs;
                tsplit.chunks = split_chunks;
            }
            if (host) {
                DCD_TRY(cudaMemcpyAsync(hv, A->values,
                                        (csr ? (size_t)nnz : (size_t)m * A->ld) * dtype_size(A->dtype),
                                        cudaMemcpyHostToDevice, st));
                DCD_TRY(cudaMemcpyAsync(yv, y_in, sizeof(double) * m, cudaMemcpyHostToDevice, st));
                DCD_TRY(cudaMemcpyAsync(av, alpha_in, sizeof(double) * m, cudaMemcpyHostToDevice, st));
                y = yv;
                alpha = av;
            } else {
                y = y_in;
                alpha = alpha_in;
            }
        }
        const void *vals = host ? h_vals : A->values;
        DCD_TRY(cudaMemsetAsync(err, 0, sizeof(int) * 8, st));
        if (tcd) DCD_TRY(cudaMemsetAsync(tsplit.cnt, 0, sizeof(unsigned) * 2 * split_pairs, st));
        DCD_TRY(cudaMemsetAsync(col_h, 0, sizeof(float) * col_pad, st));
        DCD_TRY(cudaMemsetAsync(col_w, 0, sizeof(float) * col_pad, st));
        DCD_TRY(cudaMemsetAsync(S, 0, sizeof(int32_t) * col_pad, st));
        if (tcd) DCD_TRY(cudaMemsetAsync(As, 0, (size_t)sb * row_bytes, st));
        if (scaled) DCD_TRY(cudaMemsetAsync(col_s, 0, sizeof(float) * col_pad, st));
        if (set2) {
            DCD_TRY(cudaMemsetAsync(sbuf[1].S, 0, sizeof(int32_t) * col_pad, st));
            DCD_TRY(cudaMemsetAsync(sbuf[1].col_h, 0, sizeof(float) * col_pad, st));
            if (tcd) DCD_TRY(cudaMemsetAsync(sbuf[1].As, 0, (size_t)sb * row_bytes, st));
            if (scaled) DCD_TRY(cudaMemsetAsync(sbuf[1].col_s, 0, sizeof(float) * col_pad, st));
            DCD_TRY(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking));
            DCD_TRY(cudaEventCreateWithFlags(&la_fork, cudaEventDisableTiming));
            DCD_TRY(cudaEventCreateWithFlags(&la_join, cudaEventDisableTiming));
            la = la_pos;
            lag = lag_pos;
        }
        if (df_pos) {
            for (int q = 1; q < 3; ++q) DCD_TRY(cudaMemsetAsync(sbuf[q].col_w, 0, sizeof(float) * col_pad, st));
            DCD_TRY(cudaMemsetAsync(sbuf[2].S, 0, sizeof(int32_t) * col_pad, st));
            DCD_TRY(cudaMemsetAsync(sbuf[2].col_h, 0, sizeof(float) * col_pad, st));
            DCD_TRY(cudaMemsetAsync(sbuf[2].As, 0, (size_t)sb * row_bytes, st));
            if (scaled) DCD_TRY(cudaMemsetAsync(sbuf[2].col_s, 0, sizeof(float) * col_pad, st));
            DCD_TRY(cudaMemsetAsync(xsplit.cnt, 0, 2 * sizeof(unsigned) * 2 * DF_XPAIRS, st));
            DCD_TRY(cudaEventCreateWithFlags(&df_fork, cudaEventDisableTiming));
            DCD_TRY(cudaEventCreateWithFlags(&df_chained, cudaEventDisableTiming));
            DCD_TRY(cudaEventCreateWithFlags(&df_side, cudaEventDisableTiming));
            DCD_TRY(cudaEventCreateWithFlags(&df_rows, cudaEventDisableTiming));
            DCD_TRY(cudaEventCreateWithFlags(&df_gram, cudaEventDisableTiming));
            DCD_TRY(cudaStreamCreateWithFlags(&st3, cudaStreamNonBlocking));
            DCD_TRY(cudaStreamCreateWithFlags(&st4, cudaStreamNonBlocking));
            DCD_TRY(cudaEventCreateWithFlags(&df_xfork, cudaEventDisableTiming));
            DCD_TRY(cudaEventCreateWithFlags(&df_xjoin, cudaEventDisableTiming));
            // the block leaves SMs for the recurrence ahead (one cluster) and the next step's Gram
            // (measured at config 2: 64 of 76 pairs 88.0 us per step, 66 90.0, 68 100.5, 60 88.8)
            const int P = recur_cluster_size((int)o.s, o.b, 2);
            df_pairs = std::max(split_pairs - (P + 1) / 2 - DF_GRAM_CTAS / 2, 1);
            int p_least = 0, p_greatest = 0;
            DCD_TRY(cudaDeviceGetStreamPriorityRange(&p_least, &p_greatest));
            df_prio = p_greatest;
            df = true;
        }
        if (dfs_pos) {
            for (int q = 1; q < 3; ++q) DCD_TRY(cudaMemsetAsync(sbuf[q].col_w, 0, sizeof(float) * col_pad, st));
            DCD_TRY(cudaMemsetAsync(sbuf[2].S, 0, sizeof(int32_t) * col_pad, st));
            DCD_TRY(cudaMemsetAsync(sbuf[2].col_h, 0, sizeof(float) * col_pad, st));
            if (tcd) DCD_TRY(cudaMemsetAsync(sbuf[2].As, 0, (size_t)sb * row_bytes, st));
            if (scaled) DCD_TRY(cudaMemsetAsync(sbuf[2].col_s, 0, sizeof(float) * col_pad, st));
            DCD_TRY(cudaMemsetAsync(dfs_v[0][0], 0, 12 * sizeof(double) * col_pad, st));
            for (cudaEvent_t *ev : {&df_fork, &df_chained, &df_rows, &df_side, &df_kx})
                DCD_TRY(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
            DCD_TRY(cudaStreamCreateWithFlags(&st3, cudaStreamNonBlocking));
            DCD_TRY(cudaStreamCreateWithFlags(&st4, cudaStreamNonBlocking));
            dfs = true;
        }
        DCD_TRY(cudaMemcpyAsync(ctr, &o.start_iter, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
        // the recurrence scratch starts zeroed (the FP64 form keeps its refinement state there)
        if (problem == 1) DCD_TRY(cudaMemsetAsync(Lbuf, 0, recur_bdcd_scratch_bytes(o.s, o.b), st));

        // operand
        if (csr) {
            const void *v = host ? (const void *)h_vals : A->values;
            if (conv32) DCD_TRY(launch_f64_to_f32((const double *)v, nnz, (float *)ca.vals32, st));
            if (conv64)
                DCD_TRY(launch_pack_rows(v, A->dtype, nnz, 1, nnz, nullptr, (double *)ca.vals64, PACK_F64, nnz, 1,
                                         err, st));
            // CSR checks, squared row norms and the longest row (err[2] = bad entries, err[3] = max length)
            int *bad = err + 2, *maxlen = err + 3;
            CsrOperand chk = ca;
            if (!chk.vals64 && !chk.vals32) return DCD_EINTERNAL;
            DCD_TRY(launch_csr_prep(chk, bad, maxlen, st));
            int h[2] = {0, 0};
            DCD_TRY(cudaMemcpyAsync(h, bad, sizeof(h), cudaMemcpyDeviceToHost, st));
            DCD_TRY(cudaStreamSynchronize(st));
            if (h[0]) return DCD_EINVAL;
            const int64_t cap = std::max<int64_t>(1, sb * (int64_t)h[1]);
            const size_t cmb = csr_colmap_bytes(n, cap);
            DCD_TRY(malloc_async(&ws_csr, cmb, st));
            DCD_TRY(cudaMemsetAsync(ws_csr, 0, cmb, st));
            cm = csr_colmap_carve(ws_csr, n, cap);
            csr_maxrow = h[1];
            if (!(o.flags & DCD_FLAG_CSR_FULL_PASS) && !literal) {
                dcd_status cs = setup_csc();
                if (cs != DCD_OK) return cs;
            }
            cm_set[0] = cm;
            // the look-ahead's second column map and pair table (and the deferred step's third)
            for (int q = 1; q < (dfs ? 3 : lag ? 2 : 1); ++q) {
                const int64_t pairs = sb * (int64_t)std::max(csr_maxrow, 1);
                const size_t pb = (size_t)pairs * (8 + 8 + 4) + 256 * 3;
                DCD_TRY(malloc_async(&ws_csr2[q - 1], cmb + pb, st));
                DCD_TRY(cudaMemsetAsync(ws_csr2[q - 1], 0, cmb + pb, st));
                CsrColMap c2 = csr_colmap_carve(ws_csr2[q - 1], n, cap);
                char *pp = (char *)ws_csr2[q - 1] + (cmb + 255) / 256 * 256;
                c2.pstart = (int64_t *)pp;
                pp += ((size_t)pairs * 8 + 255) / 256 * 256;
                c2.pval = (double *)pp;
                pp += ((size_t)pairs * 8 + 255) / 256 * 256;
                c2.plen = (int32_t *)pp;
                c2.pmax = cm.pmax;
                c2.csc_col_ptr = cm.csc_col_ptr;
                cm_set[q] = c2;
            }
        } else if (tc) {
            op.n_pad = n_pad;
            op.kind = pack_kind(o.prec);
            if (fp8) {
                DCD_TRY(launch_quantize_rows(vals, A->dtype, A->ld, m, n, nullptr, src_scale, (uint8_t *)op.packed,
                                             n_pad, op.row_s, m, err, st));
                dcd_status qs = check_device_error();  // non-finite values or scales: EINVAL
                if (qs != DCD_OK) return qs;
            } else if (fp16) {
                // one power-of-two scale for the matrix, from its largest magnitude (err[5], zeroed above)
                unsigned *gbits = (unsigned *)(err + 5);
                DCD_TRY(launch_absmax_rows(vals, A->dtype, A->ld, m, n, nullptr, m, gbits, err, st, src_scale));
                DCD_TRY(launch_pack_fp16(vals, A->dtype, A->ld, m, n, nullptr, op.packed, n_pad, m, op.row_s, gbits, err,
                                         st, src_scale));
                dcd_status qs = check_device_error();  // non-finite values: EINVAL
                if (qs != DCD_OK) return qs;
            } else {
                DCD_TRY(launch_pack_rows(vals, A->dtype, A->ld, m, n, nullptr, op.packed, op.kind, n_pad, m, err, st,
                                         src_scale));
            }
            DCD_TRY(launch_row_terms(op.packed, op.kind, n_pad, m, kp, op.row_h, st, op.row_s));
            if (ref_op) {
                opr.n_pad = n_pad_r;
                opr.kind = kind_r;
                if (sliced_ref) {
                    DCD_TRY(launch_pack_sliced(vals, A->dtype, A->ld, m, n, nullptr, opr.packed, n_pad_r, m, opr.row_s,
                                               err, st, src_scale));
                    DCD_TRY(cudaMemsetAsync(col_sr, 0, sizeof(float) * col_pad, st));
                } else {
                    opr.row_s = nullptr;
                    DCD_TRY(launch_pack_rows(vals, A->dtype, A->ld, m, n, nullptr, opr.packed, opr.kind, n_pad_r, m,
                                             err, st, src_scale));
                }
                DCD_TRY(cudaMemsetAsync(col_hr, 0, sizeof(float) * col_pad, st));
            } else {
                opr = op;
                Asr = As;
                col_hr = col_h;
                ref_shared = true;
            }
            if (acc_ref) {  // the RBF terms of the recomputed gradient's operand, as hi + lo pairs
                DCD_TRY(launch_row_terms(opr.packed, opr.kind, opr.n_pad, m, kp, opr.row_h, st,
                                         opr.kind == PACK_SLICED ? opr.row_s : nullptr, row_hlr));
                DCD_TRY(cudaMemsetAsync(col_hlr, 0, sizeof(float) * col_pad, st));
            }
        } else if (need_pack) {
            DCD_TRY(launch_pack_rows(vals, A->dtype, A->ld, m, n, nullptr, op.packed, 2, n, m, err, st, src_scale));
            op.a64 = (const double *)op.packed;
            op.lda = n;
        } else {
            op.a64 = (const double *)vals;
            op.lda = A->ld;
        }

        // labels
        if (problem == 0) {
            DCD_TRY(launch_label_check(y, m, flag, st));
            int bad = 0;
            DCD_TRY(cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
            DCD_TRY(cudaStreamSynchronize(st));
            if (bad) return DCD_EINVAL;
        }

        // cached gradient: with device io and a caller array, the solver works
        // on that array directly
        if (!host && grad_in) g = grad_in;
        if (o.flags & DCD_FLAG_GRAD_VALID) {
            if (!grad_in) return DCD_EINVAL;
            if (host)
                DCD_TRY(cudaMemcpyAsync(g, grad_in, sizeof(double) * m, cudaMemcpyHostToDevice, st));
        } else {
            DCD_TRY(launch_init_grad(problem, y, alpha, diag, m, g, st));
            DCD_TRY(launch_nnz_count(alpha, m, flag, st));
            int nnz = 0;
            DCD_TRY(cudaMemcpyAsync(&nnz, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
            DCD_TRY(cudaStreamSynchronize(st));
            if (nnz > 0) {
                dcd_status s2 = full_pass();
                if (s2 != DCD_OK) return s2;
            }
        }
        return DCD_OK;
    }

    // Recomputes the cached gradient of the current alpha from scratch (the
    // steps update it incrementally, so it drifts by the kernel block's
    // rounding): the constant and diagonal part, then full kernel passes.
    dcd_status refresh()
    {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
        dcd_status s0 = cuda_status(launch_init_grad(problem, y, alpha, diag, m, g, st));
        if (s0 == DCD_OK) s0 = full_pass(true);
        df_chain = false;  // a chain computed ahead read the gradient before the recomputation
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        stats.ms_refresh += ms;
        ++stats.refreshes;
        return s0;
    }

    // Convergence test at a check point: the metric of the cached gradient,
    // confirmed on a recomputed gradient with DCD_FLAG_REFRESH.
    // After a recomputed gradient misses tol, the next recomputation waits
    // for twice as many check points as the previous wait (bounded cost when
    // the precision's floor lies above tol).
    int64_t refresh_wait = 0, refresh_gap = 1;

    // final: the check at the end of the budget, which always confirms (a
    // reported metric is then never the cached gradient's alone)
    dcd_status check_converged(bool final = false)
    {
        dcd_status s0 = measure(metric, primal, dual, ynorm2);
        if (s0 != DCD_OK || !(metric <= o.tol)) return s0;
        if (o.flags & DCD_FLAG_REFRESH) {
            if (refresh_wait > 0 && !final) {
                --refresh_wait;
                return DCD_OK;
            }
            if ((s0 = refresh()) != DCD_OK) return s0;
            if ((s0 = measure(metric, primal, dual, ynorm2)) != DCD_OK) return s0;
            if (!(metric <= o.tol)) {
                refresh_wait = refresh_gap;
                refresh_gap *= 2;
            }
        }
        if (metric <= o.tol) conv = true;
        return DCD_OK;
    }

    // g += rs * K(A, A_cols) w over all columns, in chunks of SB_MAX: the
    // kernel part of the gradient for a nonzero alpha_0.
    dcd_status full_pass(bool ref = false)
    {
        std::vector<int32_t> hidx;
        const int64_t chunk = std::min<int64_t>(m, std::min<int64_t>(SB_MAX, sb));
        for (int64_t c0 = 0; c0 < m; c0 += chunk) {
            const int64_t cnt = std::min(chunk, m - c0);
            hidx.resize(cnt);
            for (int64_t j = 0; j < cnt; ++j) hidx[j] = (int32_t)(c0 + j);
            DCD_TRY(cudaMemcpyAsync(S, hidx.data(), sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, st));
            DCD_TRY(launch_coef(problem == 0 ? y : nullptr, alpha, S, cnt, 1.0 / lambda, w64, st));
            dcd_status s2 = apply_block(cnt, ref);
            if (s2 != DCD_OK) return s2;
            DCD_TRY(cudaStreamSynchronize(st));  // hidx is reused
        }
        return DCD_OK;
    }

    // gather A_S for the tensor-core path (of the step operand, or of x)
    cudaError_t gather(int64_t ncols)
    {
        if (csr) return launch_csr_colmap(ca, S, ncols, cm, err, st);
        return gather_op(ncols, op, As, col_h);
    }
    cudaError_t gather_op(int64_t ncols, const Operand &x, void *Asx, float *chx)
    {
        if (!tc) return cudaSuccess;
        const bool f8 = x.kind == PACK_FP8 || x.kind == PACK_FP16;  // per-row scales gathered too
        return launch_gather_rows(x.packed, packed_row_bytes(x.kind, x.n_pad), S, ncols, m, Asx, err, st, x.row_h,
                                  chx, f8 ? x.row_s : nullptr, f8 ? col_s : nullptr);
    }

    cudaError_t gram(int64_t ncols)
    {
        if (csr)
            return launch_csr_block(ca, cm, !tc, kp, S, ncols, S, ncols, nullptr, nullptr, nullptr, nullptr, Kss, ldk,
                                    st);
        if (tc) {
            // the cluster and blocked recurrences read the lower triangle only
            const bool lower = problem == 1 && recur_bdcd_lower_gram(ncols / o.b, o.b, 1, ldk);
            TcOperand B{As, ncols, op.n_pad, op.kind, col_s, S};
            return launch_block_tc(B, B, kp, col_h, col_h, nullptr, nullptr, nullptr, (float *)Kss, ldk, ncols, ncols,
                                   err, st, lower);
        }
        return launch_block_simt_f64(op.a64, op.lda, m, n, kp, S, ncols, S, ncols, nullptr, nullptr, nullptr,
                                     (double *)Kss, ldk, err, st);
    }

    // g += rs * K(A, A_S) w64 with the step operand, or (ref) with the
    // operand of the recomputed gradient
    dcd_status apply_block(int64_t ncols, bool ref = false)
    {
        const double *rs = problem == 0 ? y : nullptr;
        if (csr) {  // the same CSR block in every case (ref has no other operand)
            DCD_TRY(gather(ncols));
            if (tc) DCD_TRY(launch_f64_to_f32(w64, ncols, col_w, st));
            return cuda_status(csr_apply(ncols, rs));
        }
        if (tc && ref && row_hlr) {
            // the recomputed gradient: sliced (or split-tf32) products, accurate epilogue, FP64 coefficients
            const bool sl = opr.kind == PACK_SLICED;
            cudaError_t e = launch_gather_rows(opr.packed, packed_row_bytes(opr.kind, opr.n_pad), S, ncols, m, Asr,
                                               err, st, opr.row_h, col_hr, row_hlr, col_hlr, sl ? opr.row_s : nullptr,
                                               sl ? col_sr : nullptr);
            if (e != cudaSuccess) return cuda_status(e);
            TcOperand Aop{opr.packed, m, opr.n_pad, opr.kind, sl ? opr.row_s : nullptr};
            TcOperand Bop{Asr, ncols, opr.n_pad, opr.kind, sl ? col_sr : nullptr, S};
            TcAccurate acc;
            acc.w64 = w64;
            acc.row_hl = row_hlr;
            acc.col_hl = col_hlr;
            return cuda_status(launch_block_tc(Aop, Bop, kp, opr.row_h, col_hr, col_w, rs, g, nullptr, 0, m, ncols,
                                               err, st, false, &tsplit, false, 0, &acc));
        }
        if (tc) {
            const Operand &x = ref ? opr : op;
            void *Asx = ref ? Asr : As;
            float *chx = ref ? col_hr : col_h;
            // the coefficients in w64 (FP64) go to the FP32 column buffer
            cudaError_t e = gather_op(ncols, x, Asx, chx);
            if (e != cudaSuccess) return cuda_status(e);
            e = launch_f64_to_f32(w64, ncols, col_w, st);
            if (e != cudaSuccess) return cuda_status(e);
            e = clear_col_w_tail(ncols);
            if (e != cudaSuccess) return cuda_status(e);
            TcOperand Aop{x.packed, m, x.n_pad, x.kind, x.row_s};
            TcOperand Bop{Asx, ncols, x.n_pad, x.kind, x.kind == PACK_FP8 || x.kind == PACK_FP16 ? col_s : nullptr,
                          S};
            return cuda_status(
                launch_block_tc(Aop, Bop, kp, x.row_h, chx, col_w, rs, g, nullptr, 0, m, ncols, err, st, false, &tsplit));
        }
        return cuda_status(launch_block_simt_f64(op.a64, op.lda, m, n, kp, nullptr, m, S, ncols, w64, rs, g, nullptr,
                                                 0, err, st));
    }

    // Columns past ncols of the FP32 coefficient buffer must be zero: the
    // tensor-core epilogue reads whole 32-column groups.
    int64_t col_w_hi = 0;  // entries [0, col_w_hi) may be nonzero
    cudaError_t clear_col_w_tail(int64_t ncols)
    {
        cudaError_t e = cudaSuccess;
        if (col_w_hi > ncols) e = cudaMemsetAsync(col_w + ncols, 0, sizeof(float) * (col_w_hi - ncols), st);
        col_w_hi = ncols;
        return e;
    }

    dcd_status setup_csc()
    {
        bool use = false;
        dcd_status r =
            csc_choose(ca, !tc, sb, csr_maxrow, err + 4, &ws_csc, &cscop, &ws_cstep, &cstep, &cm, &use, st);
        use_csc = use;
        if (r == DCD_OK && use) {
            DCD_TRY(cudaStreamCreateWithFlags(&csr_st, cudaStreamNonBlocking));
            DCD_TRY(cudaEventCreateWithFlags(&csr_fork, cudaEventDisableTiming));
            DCD_TRY(cudaEventCreateWithFlags(&csr_join, cudaEventDisableTiming));
        }
        return r;
    }

    // The first chunk's scatter forked onto csr_st after the column map (it
    // runs beside the Gram and the recurrence); csr_apply joins it.
    bool csr_forked = false;
    cudaError_t csr_fork_scatter(int64_t ncols)
    {
        cudaError_t e = cudaEventRecord(csr_fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(csr_st, csr_fork, 0);
        if (e == cudaSuccess) e = launch_csr_csc_scatter_first(cm, cscop, cstep, !tc, csr_maxrow, ncols, csr_st);
        if (e == cudaSuccess) e = cudaEventRecord(csr_join, csr_st);
        csr_forked = e == cudaSuccess;
        return e;
    }

    cudaError_t csr_apply(int64_t ncols, const double *rs)
    {
        if (use_csc) {
            const bool first = csr_forked;
            csr_forked = false;
            if (first) {
                const cudaError_t e = cudaStreamWaitEvent(st, csr_join, 0);
                if (e != cudaSuccess) return e;
            }
            return launch_csr_apply_csc(ca, cm, cscop, cstep, !tc, csr_maxrow, kp, S, ncols, col_w, w64, rs, g, st,
                                        first);
        }
        return launch_csr_block(ca, cm, !tc, kp, nullptr, m, S, ncols, col_w, w64, rs, g, nullptr, 0, st);
    }

    cudaError_t block_tc_apply(int64_t ncols, const double *rs)
    {
        TcOperand Aop{op.packed, m, op.n_pad, op.kind, op.row_s};
        TcOperand Bop{As, ncols, op.n_pad, op.kind, col_s, S};
        return launch_block_tc(Aop, Bop, kp, op.row_h, col_h, col_w, rs, g, nullptr, 0, m, ncols, err, st, false,
                               &tsplit);
    }

    // Convergence measure from the cached gradient (reads back 4 doubles).
    dcd_status measure(double &metric, double &primal, double &dual, double ynorm2)
    {
        double r[4];
        DCD_TRY(measure_enqueue(r));
        DCD_TRY(cudaStreamSynchronize(st));
        measure_finish(r, metric, primal, dual, ynorm2);
        return DCD_OK;
    }

    // the two halves of measure, for checks of many solves with one synchronisation
    cudaError_t measure_enqueue(double *r4)
    {
        cudaError_t e = launch_check(problem, g, alpha, y, m, C, loss, partials, result, st);
        if (e != cudaSuccess) return e;
        return cudaMemcpyAsync(r4, result, 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
    }

    void measure_finish(const double *r, double &metric, double &primal, double &dual, double ynorm2) const
    {
        if (problem == 1) {
            metric = std::sqrt(r[0]) / std::sqrt(ynorm2 > 0 ? ynorm2 : 1.0);
            primal = dual = 0.0;
        } else {
            // r = {a^T Q a, sum a, ||a||^2, hinge}; gap = P - D, reported relative to |P|
            primal = 0.5 * r[0] + C * r[3];
            dual = r[1] - 0.5 * r[0] - (loss == 2 ? r[2] / (4.0 * C) : 0.0);
            metric = (primal - dual) / std::max(std::fabs(primal), 1e-300);
        }
    }

    // ---- outer-step loop, resumable (the plan API runs it in pieces) ----
    double ynorm2 = 1.0;
    int64_t done = 0, steps = 0;
    double metric = 0.0, primal = 0.0, dual = 0.0;
    bool conv = false, begun = false;
    double ms_accum = 0.0;

    dcd_status begin()
    {
        if (begun) return DCD_OK;
        begun = true;
        if (problem == 1) {  // ||y||^2 by the same reduction as the residual
            DCD_TRY(launch_check(1, y, alpha, y, m, C, loss, partials, result, st));
            DCD_TRY(cudaMemcpyAsync(&ynorm2, result, sizeof(double), cudaMemcpyDeviceToHost, st));
            DCD_TRY(cudaStreamSynchronize(st));
        }
        // kernels per outer step: sample, [gather rows, gather terms,] Gram,
        // recurrence, block, update -- counted exactly from the graph once a
        // full step has been captured; the recurrence is taken as the
        // cluster (K-RR) or single-warp (K-SVM) form until then
        stats.gpu_launches_per_step = (tc ? 3 : 1) + 1 + (problem == 0 ? 1 : 2) + 2;
        stats.s_used = o.s;
        return DCD_OK;
    }

    bool finished() const { return conv || done >= o.max_iters; }

    // One outer s-step (a1..a6) of cnt inner iterations.  Full steps
    // (cnt == s) are captured once into a CUDA graph and replayed: every
    // kernel argument is the same from step to step (the stream position
    // lives in device memory), so one capture serves the whole solve.
    cudaGraphExec_t graph_exec = nullptr;
    int direct_full_steps = 0;
    bool graph_failed = false;

    // ---- look-ahead (dense tensor-core K-RR on the single-cluster recurrence) ----
    // Step k+1's sample, gathers, Gram and recurrence prep depend on its
    // indices only, not on alpha or g, so they run on a second stream beside
    // step k's chain (which occupies one cluster of SMs) and fused block.
    // The step products live in two buffer sets used alternately; ctr_la[q]
    // holds the index-stream position of the step to be sampled into set q,
    // one step ahead of ctr (which the chain's a6 advances as before); the
    // sample into set q leaves the following position in ctr_la[1 - q].
    struct StepBufs {
        int32_t *S = nullptr;
        void *As = nullptr;
        float *col_h = nullptr, *col_s = nullptr;
        void *Kss = nullptr;
        double *Lbuf = nullptr;
        // the chain's outputs (per set with the deferred gradient; shared otherwise)
        double *delta = nullptr, *w64 = nullptr;
        float *col_w = nullptr;
    };
    bool la = false;
    bool lag = false;  // the K-SVM look-ahead (in-order: products of step k+1 beside step k)
    StepBufs sbuf[3];
    cudaStream_t st2 = nullptr;
    cudaEvent_t la_fork = nullptr, la_join = nullptr;
    uint64_t *ctr_la = nullptr;
    int la_par = 0;        // the buffer set holding the next step's products
    int64_t la_cnt = 0;    // their step size (0: none pending)
    bool ref_shared = false;  // the recomputed gradient uses the step operand's buffers
    cudaGraphExec_t graph_la[2] = {nullptr, nullptr};
    int la_direct[2] = {0, 0};

    // the step members point at buffer set p
    void use_bufs(int p)
    {
        S = sbuf[p].S;
        As = sbuf[p].As;
        col_h = sbuf[p].col_h;
        col_s = sbuf[p].col_s;
        Kss = sbuf[p].Kss;
        Lbuf = sbuf[p].Lbuf;
        if (df || dfs) {
            delta = sbuf[p].delta;
            w64 = sbuf[p].w64;
            col_w = sbuf[p].col_w;
        }
        if (lag && csr) cm = cm_set[p];
        if (ref_shared) {
            Asr = As;
            col_hr = col_h;
        }
    }

    // step products of a step of cnt blocks into buffer set q, on stream s2: the sample and the
    // gathers (la_rows), then the Gram and the prep (la_gram)
    dcd_status la_side(int q, int64_t cnt, cudaStream_t s2, int qnext = -1, int max_ctas = 0)
    {
        dcd_status r = la_rows(q, cnt, s2, qnext);
        return r != DCD_OK ? r : la_gram(q, cnt, s2, max_ctas);
    }

    dcd_status la_rows(int q, int64_t cnt, cudaStream_t s2, int qnext = -1)
    {
        const StepBufs &Bq = sbuf[q];
        const int64_t ncols = cnt * o.b;
        if (qnext < 0) qnext = 1 - q;
        // the sample reads the position in ctr_la[q] and leaves the next one in ctr_la[qnext]
        DCD_TRY(launch_sample(problem, o.seed, ctr_la + q, 0, m, o.b, cnt, Bq.S, err, s2, ctr_la + qnext));
        const bool f8 = op.kind == PACK_FP8 || op.kind == PACK_FP16;  // per-row scales gathered too
        DCD_TRY(launch_gather_rows(op.packed, packed_row_bytes(op.kind, op.n_pad), Bq.S, ncols, m, Bq.As, err, s2,
                                   op.row_h, Bq.col_h, f8 ? op.row_s : nullptr, f8 ? Bq.col_s : nullptr));
        return DCD_OK;
    }

    dcd_status la_gram(int q, int64_t cnt, cudaStream_t s2, int max_ctas = 0)
    {
        const StepBufs &Bq = sbuf[q];
        const int64_t ncols = cnt * o.b;
        TcOperand Bo{Bq.As, ncols, op.n_pad, op.kind, Bq.col_s, Bq.S};
        DCD_TRY(launch_block_tc(Bo, Bo, kp, Bq.col_h, Bq.col_h, nullptr, nullptr, nullptr, (float *)Bq.Kss, ldk, ncols,
                                ncols, err, s2, true, nullptr, false, max_ctas));
        DCD_TRY(launch_recur_cluster_prep((const float *)Bq.Kss, ldk, Bq.S, (int)cnt, o.b, lambda, (double)m, Bq.Lbuf,
                                          err, s2));
        return DCD_OK;
    }

    // one look-ahead step, products in set p: the chain (with the a6 update) on st, then the fused
    // block as its programmatic dependent on the SMs the chain's cluster leaves free: its
    // tensor-core products start beside the chain, its epilogue waits for it.  The next full step's
    // products (next > 0) go to set 1 - p on st2, forked before the chain and joined back into st
    // after the block: the sample and the gathers fit beside the block's CTAs, the Gram and the
    // prep take the chain's SMs once it ends.
    dcd_status la_body(int p, int64_t cnt, int64_t next)
    {
        const StepBufs &Bp = sbuf[p];
        const int64_t ncols = cnt * o.b;
        FusedUpdate fu;
        fu.alpha = alpha;
        fu.ctr = ctr;
        fu.ctr_advance = (uint64_t)cnt;
        const int P = recur_cluster_size((int)cnt, o.b, 2);
        if (P <= 0) return DCD_EINTERNAL;
        // the fork is recorded first and the chain launched before the side kernels (its cluster
        // takes SMs first); the block may start once the side kernels are done: about 5/8 of the
        // chain
        if (next) DCD_TRY(cudaEventRecord(la_fork, st));
        const int trig = next ? (int)((cnt * o.b / 32) * 5 / 8) : -1;
        DCD_TRY(launch_recur_cluster_chain((const float *)Bp.Kss, ldk, Bp.S, (int)cnt, o.b, P, lambda, (double)m, g, 2,
                                           Bp.Lbuf, delta, w64, col_w, &fu, err, st, nullptr, trig));
        if (next) {
            DCD_TRY(cudaStreamWaitEvent(st2, la_fork, 0));
            dcd_status r = la_side(1 - p, next, st2);
            if (r != DCD_OK) return r;
            DCD_TRY(cudaEventRecord(la_join, st2));
        }
        DCD_TRY(clear_col_w_tail(ncols));
        TcOperand Aop{op.packed, m, op.n_pad, op.kind, op.row_s};
        TcOperand Bop{Bp.As, ncols, op.n_pad, op.kind, Bp.col_s, Bp.S};
        // the chain writes only delta, the coefficients, alpha, g and the counter: the block's
        // products read none of them.  The pairs that land on the chain's SMs (the grid's last,
        // launched once the chain ends) take two units fewer: the others fill both tensor-memory
        // accumulators while the chain runs.
        TcSplit sp = tsplit;
        sp.late_pairs = (P + 1) / 2;
        sp.late_units = 2;
        DCD_TRY(launch_block_tc(Aop, Bop, kp, op.row_h, Bp.col_h, col_w, nullptr, g, nullptr, 0, m, ncols, err, st,
                                false, &sp, true));
        if (next) DCD_TRY(cudaStreamWaitEvent(st, la_join, 0));
        return DCD_OK;
    }

    dcd_status la_step(int64_t cnt)
    {
        if (la_cnt != cnt) {  // nothing pending: this step's products first, on st
            DCD_TRY(cudaMemcpyAsync(ctr_la + la_par, ctr, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
            dcd_status r = la_side(la_par, cnt, st);
            if (r != DCD_OK) return r;
            la_cnt = cnt;
        }
        const int p = la_par;
        const int64_t next = (o.max_iters - done - cnt) >= o.s ? o.s : 0;  // only full steps are prepared ahead
        if (next && cnt == o.s && !graph_failed) {
            if (graph_la[p]) {
                DCD_TRY(cudaGraphLaunch(graph_la[p], st));
            } else if (la_direct[p] >= 1) {
                DCD_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                const dcd_status sc = la_body(p, cnt, next);
                cudaGraph_t graph = nullptr;
                const cudaError_t ec = cudaStreamEndCapture(st, &graph);
                const bool ok = sc == DCD_OK && ec == cudaSuccess && graph != nullptr &&
                                cudaGraphInstantiate(&graph_la[p], graph, 0) == cudaSuccess;
                if (ok) stats.gpu_launches_per_step = count_kernel_nodes(graph);
                if (graph) cudaGraphDestroy(graph);
                if (!ok) {
                    cudaGetLastError();
                    graph_la[p] = nullptr;
                    graph_failed = true;
                    dcd_status r = la_body(p, cnt, next);
                    if (r != DCD_OK) return r;
                } else {
                    DCD_TRY(cudaGraphLaunch(graph_la[p], st));
                }
            } else {
                dcd_status r = la_body(p, cnt, next);
                if (r != DCD_OK) return r;
                ++la_direct[p];
            }
        } else {
            dcd_status r = la_body(p, cnt, next);
            if (r != DCD_OK) return r;
        }
        la_par = 1 - p;
        la_cnt = next;
        use_bufs(p);  // the set just used is free (for a gradient recomputation) while the other holds products
        return DCD_OK;
    }

    // ---- deferred gradient (the look-ahead with the recurrence one step ahead of the block) ----
    // The recurrence of step k+1 reads g at its sampled rows after step k's block and update.
    // That is g before block k plus x(k+1), block k's and update k's part at those rows:
    // K(A_S(k+1), A_S(k)) w(k) (an s b x s b product) plus m Delta(k) summed over the positions of
    // S(k) holding the same row.  x(k+1) needs only step k's coefficients and step k+1's rows, so it
    // is formed a step early, and the recurrence of step k+1 runs beside block k, reading
    // -(g[S] + x) before that block writes g.  One captured body per step k, buffer sets in
    // rotation (cur: step k with its recurrence outputs; nxt: step k+1's products and x(k+1);
    // nn: step k+2's):
    //   st : recurrence k+1 (one cluster, launched first), block k as its programmatic dependent
    //        on the SMs the others leave (its epilogue does not wait: it reads nothing the
    //        recurrence writes), update k;
    //   st2: step k+2's sample and gathers, then its Gram (a few CTAs) and prep, into nn;
    //   st3, st4: after the gathers and recurrence k+1, x(k+2) into nn (two column halves).
    // The association of the gradient's sums differs from the in-order step's; results agree to
    // rounding.  A gradient recomputation invalidates the recurrence and x computed ahead.
    bool df = false;
    int df_cur = 0;            // the set of the next step to run
    bool df_chain = false;     // its recurrence outputs (and x of the step after it) are in place
    int64_t df_prod = 0;       // step size of the products in (df_cur + 1) % 3 (0: none)
    double *df_x[3] = {nullptr, nullptr, nullptr};  // per set: x of its step (col_pad doubles)
    cudaStream_t st3 = nullptr, st4 = nullptr;  // x of the step after next, beside its Gram and prep
    cudaEvent_t df_fork = nullptr, df_chained = nullptr, df_rows = nullptr, df_gram = nullptr, df_side = nullptr,
                df_xfork = nullptr, df_xjoin = nullptr;
    double *df_x2 = nullptr;   // the second column half's part of x
    TcSplit xsplit, xsplit2;   // the cross product's halves' splits (they run beside the block)
    int df_pairs = 0;          // CTA pairs of the block
    int df_prio = 0;           // launch priority of the recurrence and the block
    cudaGraphExec_t graph_df[3] = {nullptr, nullptr, nullptr};
    int df_direct[3] = {0, 0, 0};

    // the recurrence of the step in set q on stream s, right-hand side -(g[S] + x) (x: nullptr for
    // -g[S]), no fused update
    dcd_status df_chain_of(int q, int64_t cnt, const double *x, cudaStream_t s, int prio = 0)
    {
        const StepBufs &Bq = sbuf[q];
        const int P = recur_cluster_size((int)cnt, o.b, 2);
        if (P <= 0) return DCD_EINTERNAL;
        DCD_TRY(launch_recur_cluster_chain((const float *)Bq.Kss, ldk, Bq.S, (int)cnt, o.b, P, lambda, (double)m, g,
                                           2, Bq.Lbuf, Bq.delta, Bq.w64, Bq.col_w, nullptr, err, s, x, -1, x != nullptr,
                                           prio));
        return DCD_OK;
    }

    // x of the step in set r (full) from the step in set c (full, its recurrence done), on stream
    // s; the product's columns in two launches (the second on sb, joined back), each on as many
    // CTA pairs as row tiles, and the halves added in the repeat kernel
    dcd_status df_cross(int r, int c, cudaStream_t s, cudaStream_t sb2)
    {
        const StepBufs &Br = sbuf[r], &Bc = sbuf[c];
        const int64_t nc = o.s * o.b;
        // split at a multiple of the 256-column chunk, so that neither launch reads the other's columns
        const int64_t h = nc >= 512 ? nc / 2 / 256 * 256 : nc;
        TcOperand Ax{Br.As, nc, op.n_pad, op.kind, Br.col_s, Br.S};
        if (h < nc) {
            if (sb2 != s) {
                DCD_TRY(cudaEventRecord(df_xfork, s));
                DCD_TRY(cudaStreamWaitEvent(sb2, df_xfork, 0));
            }
            const size_t rb = (size_t)packed_row_bytes(op.kind, op.n_pad);
            DCD_TRY(cudaMemsetAsync(df_x2, 0, sizeof(double) * nc, sb2));
            TcOperand Bx{(const char *)Bc.As + h * rb, nc - h, op.n_pad, op.kind, Bc.col_s ? Bc.col_s + h : nullptr,
                         Bc.S + h};
            DCD_TRY(launch_block_tc(Ax, Bx, kp, Br.col_h, Bc.col_h + h, Bc.col_w + h, nullptr, df_x2, nullptr, 0, nc,
                                    nc - h, err, sb2, false, &xsplit2, false, DF_XPAIRS));
            if (sb2 != s) DCD_TRY(cudaEventRecord(df_xjoin, sb2));
        }
        DCD_TRY(cudaMemsetAsync(df_x[r], 0, sizeof(double) * nc, s));
        TcOperand Bx{Bc.As, h, op.n_pad, op.kind, Bc.col_s, Bc.S};
        DCD_TRY(launch_block_tc(Ax, Bx, kp, Br.col_h, Bc.col_h, Bc.col_w, nullptr, df_x[r], nullptr, 0, nc, h, err, s,
                                false, &xsplit, false, DF_XPAIRS));
        if (h < nc && sb2 != s) DCD_TRY(cudaStreamWaitEvent(s, df_xjoin, 0));
        DCD_TRY(launch_defer_repeat(Br.S, nc, Bc.S, Bc.delta, nc, diag, h < nc ? df_x2 : nullptr, df_x[r], s));
        return DCD_OK;
    }

    dcd_status df_body(int cur, int64_t cnt, bool has1, bool has2)
    {
        const int nxt = (cur + 1) % 3, nn = (cur + 2) % 3;
        const StepBufs &Bc = sbuf[cur];
        const int64_t ncols = cnt * o.b;
        // the fork is recorded first and the recurrence launched before the side streams' kernels,
        // so that its cluster takes SMs first
        if (has2) DCD_TRY(cudaEventRecord(df_fork, st));
        if (has1) {
            dcd_status r = df_chain_of(nxt, o.s, df_x[nxt], st, df_prio);
            if (r != DCD_OK) return r;
        }
        if (has2) {
            DCD_TRY(cudaStreamWaitEvent(st2, df_fork, 0));
            dcd_status r = la_rows(nn, o.s, st2, (nn + 1) % 3);
            if (r != DCD_OK) return r;
            DCD_TRY(cudaEventRecord(df_rows, st2));
            DCD_TRY(cudaStreamWaitEvent(st3, df_rows, 0));
            r = la_gram(nn, o.s, st2, DF_GRAM_CTAS);
            if (r != DCD_OK) return r;
            DCD_TRY(cudaEventRecord(df_gram, st2));
        }
        if (has1 && has2) {
            // x of step k+2 waits for recurrence k+1.  Under capture the recurrence's node (still
            // st's last) is added to the side stream's dependencies directly: an event recorded on
            // st between the recurrence and the block would stand between the two kernels of the
            // programmatic launch
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            const cudaGraphNode_t *deps = nullptr;
            size_t nd = 0;
            DCD_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd));
            if (cs == cudaStreamCaptureStatusActive) {
                std::vector<cudaGraphNode_t> dv(deps, deps + nd);
                DCD_TRY(cudaStreamUpdateCaptureDependencies(st3, dv.data(), nullptr, dv.size(),
                                                            cudaStreamAddCaptureDependencies));
            } else {
                DCD_TRY(cudaEventRecord(df_chained, st));
                DCD_TRY(cudaStreamWaitEvent(st3, df_chained, 0));
            }
            const dcd_status r = df_cross(nn, nxt, st3, st4);
            if (r != DCD_OK) return r;
            DCD_TRY(cudaEventRecord(df_side, st3));
        }
        // block k as the programmatic dependent of recurrence k+1 (which read g before signalling):
        // its epilogue does not wait, it reads nothing the recurrence writes; the recurrence and
        // the block take SMs before the side kernels (higher launch priority).  (Update k before
        // the block, as a dependent of the recurrence, would make the block's epilogue wait for
        // the recurrence too: a grid's completion as a programmatic prerequisite includes its own
        // prerequisite's.)
        TcOperand Aop{op.packed, m, op.n_pad, op.kind, op.row_s};
        TcOperand Bop{Bc.As, ncols, op.n_pad, op.kind, Bc.col_s, Bc.S};
        DCD_TRY(launch_block_tc(Aop, Bop, kp, op.row_h, Bc.col_h, Bc.col_w, nullptr, g, nullptr, 0, m, ncols, err, st,
                                false, &tsplit, has1, has1 ? df_pairs : 0, nullptr, false, df_prio));
        DCD_TRY(launch_update(Bc.S, Bc.delta, ncols, diag, alpha, g, ctr, (uint64_t)cnt, m, err, st));
        if (has2) {
            DCD_TRY(cudaStreamWaitEvent(st, df_gram, 0));
            DCD_TRY(cudaStreamWaitEvent(st, df_side, 0));
        }
        return DCD_OK;
    }

    // one full step through the deferred bodies
    dcd_status df_step(int64_t cnt)
    {
        const int cur = df_cur, nxt = (cur + 1) % 3, nn = (cur + 2) % 3;
        const int64_t rem1 = o.max_iters - done - cnt, rem2 = rem1 - o.s;
        const bool has1 = rem1 >= o.s, has2 = has1 && rem2 >= o.s;
        if (!df_chain) {  // prologue: this step's products (unless prepared), its recurrence on g itself
            if (la_cnt != cnt) {
                DCD_TRY(cudaMemcpyAsync(ctr_la + cur, ctr, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
                dcd_status r = la_side(cur, cnt, st, nxt);
                if (r != DCD_OK) return r;
                la_cnt = cnt;
                df_prod = 0;  // the position after this step is in ctr_la[nxt]; nothing sampled there
            }
            dcd_status r = df_chain_of(cur, cnt, nullptr, st);
            if (r != DCD_OK) return r;
            if (has1) {  // step k+1's products and x
                if (df_prod != o.s) {
                    r = la_side(nxt, o.s, st, nn);
                    if (r != DCD_OK) return r;
                    df_prod = o.s;
                }
                r = df_cross(nxt, cur, st, st);
                if (r != DCD_OK) return r;
            }
            df_chain = true;
        }
        const bool graphable = !graph_failed && has1 && has2;  // the steady state replays three graphs
        if (graphable && graph_df[cur]) {
            DCD_TRY(cudaGraphLaunch(graph_df[cur], st));
        } else if (graphable && df_direct[cur] >= 1) {
            DCD_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            const dcd_status sc = df_body(cur, cnt, has1, has2);
            cudaGraph_t graph = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(st, &graph);
            const bool ok = sc == DCD_OK && ec == cudaSuccess && graph != nullptr &&
                            cudaGraphInstantiate(&graph_df[cur], graph, 0) == cudaSuccess;
            if (ok) stats.gpu_launches_per_step = count_kernel_nodes(graph);
            if (graph) cudaGraphDestroy(graph);
            if (!ok) {
                cudaGetLastError();
                graph_df[cur] = nullptr;
                graph_failed = true;
                dcd_status r = df_body(cur, cnt, has1, has2);
                if (r != DCD_OK) return r;
            } else {
                DCD_TRY(cudaGraphLaunch(graph_df[cur], st));
            }
        } else {
            dcd_status r = df_body(cur, cnt, has1, has2);
            if (r != DCD_OK) return r;
            if (graphable) ++df_direct[cur];
        }
        df_cur = nxt;
        df_chain = has1;
        df_prod = has2 ? o.s : 0;
        la_cnt = has1 ? o.s : 0;  // the products of the next step are in place
        use_bufs(cur);  // the set just used is free (for a gradient recomputation)
        col_w_hi = std::max<int64_t>(col_w_hi, sb);  // any set's coefficients may fill sb entries
        return DCD_OK;
    }

    // ---- the deferred K-SVM step (the recurrence one step ahead of the block and update) ----
    // The recurrence of step k+1 needs alpha and g at its rows S(k+1) after step k's block and
    // update.  Those are the values before block k (a snapshot taken once update k-1 is done)
    // plus step k's part, which needs only step k's steps theta(k) and coefficients w(k) = y theta(k):
    //   alpha: the sum of theta(k) over the positions of S(k) holding the same row,
    //   g:     y_i K(a_i, A_S(k)) w(k) (an s x s product) plus diag times that sum.
    // Step k+2's part is formed as soon as recurrence k+1 ends, so each body runs recurrence k+1
    // beside block k.  One captured body per step k, buffer sets in rotation (cur: step k with its
    // recurrence outputs; nxt: step k+1's products and pending parts; nn: step k+2's):
    //   st : the snapshot at S(k+1), block k (the CSR block's first scatter forked beside it), update k;
    //   st3: recurrence k+1 on the snapshot plus the pending parts, then step k+2's pending parts;
    //   st2: step k+2's sample, column map (CSR) and Gram, into nn;
    //   st4: after that sample, K(A_S(k+2), A_S(k+1)) for the pending parts.
    // The sums are associated differently from the in-order step's; results agree to rounding.
    // A gradient recomputation invalidates the recurrence and the parts computed ahead.
    bool dfs = false;
    double *dfs_v[3][4] = {};  // per set: alpha snapshot, alpha pending, g snapshot, g pending
    void *dfs_kx = nullptr;    // s x s kernel values (FP32 when tc, else FP64), row-major
    cudaEvent_t df_kx = nullptr;

    // K(A_S(q2) rows, A_S(q) columns) into dfs_kx on stream s2 (CSR: the column map of set q;
    // tensor-core form: both sets' gathered rows)
    cudaError_t dfs_cross(int q2, int q, int64_t cnt, cudaStream_t s2)
    {
        if (csr)
            return launch_csr_block(ca, cm_set[q], !tc, kp, sbuf[q2].S, cnt, sbuf[q].S, cnt, nullptr, nullptr,
                                    nullptr, nullptr, dfs_kx, cnt, s2);
        if (tc) {
            const StepBufs &R = sbuf[q2], &Cq = sbuf[q];
            TcOperand Ro{R.As, cnt, op.n_pad, op.kind, R.col_s, R.S};
            TcOperand Co{Cq.As, cnt, op.n_pad, op.kind, Cq.col_s, Cq.S};
            return launch_block_tc(Ro, Co, kp, R.col_h, Cq.col_h, nullptr, nullptr, nullptr, (float *)dfs_kx, cnt, cnt,
                                   cnt, err, s2);
        }
        return launch_block_simt_f64(op.a64, op.lda, m, n, kp, sbuf[q2].S, cnt, sbuf[q].S, cnt, nullptr, nullptr,
                                     nullptr, (double *)dfs_kx, cnt, err, s2);
    }

    // the pending parts of set q2 (the step after set q's) from set q's recurrence outputs
    cudaError_t dfs_pending(int q2, int q, int64_t cnt, cudaStream_t s2)
    {
        return launch_dcd_pending(sbuf[q2].S, cnt, y, dfs_kx, !tc, cnt, sbuf[q].S, sbuf[q].delta, sbuf[q].w64, cnt,
                                  diag, dfs_v[q2][1], dfs_v[q2][3], s2);
    }

    // the recurrence of the step in set q on stream s2 (pend: from the snapshot and pending parts)
    cudaError_t dfs_chain_of(int q, int64_t cnt, bool pend, cudaStream_t s2)
    {
        const StepBufs &Bq = sbuf[q];
        DcdPending pd{dfs_v[q][0], dfs_v[q][1], dfs_v[q][2], dfs_v[q][3]};
        return launch_recur_dcd(Bq.Kss, tc ? 0 : 1, ldk, Bq.S, cnt, y, alpha, g, omega, nu, Bq.delta, Bq.w64,
                                tc ? Bq.col_w : nullptr, err, s2, pend ? &pd : nullptr);
    }

    dcd_status dfs_body(int cur, int64_t cnt, bool has1, bool has2)
    {
        const int nxt = (cur + 1) % 3, nn = (cur + 2) % 3;
        const bool scatter = csr && use_csc;
        if (has1) {
            DCD_TRY(launch_dcd_snapshot(sbuf[nxt].S, o.s, m, alpha, g, dfs_v[nxt][0], dfs_v[nxt][2], st));
            DCD_TRY(cudaEventRecord(df_fork, st));
        }
        if (scatter) DCD_TRY(cudaEventRecord(csr_fork, st));
        if (has1) {  // the recurrence first, so that it is the first of the step's kernels to take an SM
            DCD_TRY(cudaStreamWaitEvent(st3, df_fork, 0));
            DCD_TRY(dfs_chain_of(nxt, o.s, true, st3));
        }
        if (has2) {
            DCD_TRY(cudaStreamWaitEvent(st2, df_fork, 0));
            dcd_status r = lag_side(nn, o.s, st2, (nn + 1) % 3, df_rows);
            if (r != DCD_OK) return r;
            DCD_TRY(cudaEventRecord(la_join, st2));
            DCD_TRY(cudaStreamWaitEvent(st4, df_rows, 0));
            DCD_TRY(dfs_cross(nn, nxt, o.s, st4));
            DCD_TRY(cudaEventRecord(df_kx, st4));
            DCD_TRY(cudaStreamWaitEvent(st3, df_kx, 0));
            DCD_TRY(dfs_pending(nn, nxt, o.s, st3));
        }
        if (has1) DCD_TRY(cudaEventRecord(df_side, st3));
        use_bufs(cur);
        const int64_t ncols = cnt * o.b;
        if (scatter) {  // this step's first scatter through the transposed copy, beside the block's start
            DCD_TRY(cudaStreamWaitEvent(csr_st, csr_fork, 0));
            DCD_TRY(launch_csr_csc_scatter_first(cm, cscop, cstep, !tc, csr_maxrow, ncols, csr_st));
            DCD_TRY(cudaEventRecord(csr_join, csr_st));
            csr_forked = true;
        }
        const double *rs = y;
        if (csr)
            DCD_TRY(csr_apply(ncols, rs));
        else if (tc)
            DCD_TRY(block_tc_apply(ncols, rs));  // (every set's coefficients past sb stay zero)
        else
            DCD_TRY(launch_block_simt_f64(op.a64, op.lda, m, n, kp, nullptr, m, S, ncols, w64, rs, g, nullptr, 0,
                                          err, st));
        DCD_TRY(launch_update(S, delta, ncols, diag, alpha, g, ctr, (uint64_t)cnt, m, err, st));
        if (has2) DCD_TRY(cudaStreamWaitEvent(st, la_join, 0));
        if (has1) DCD_TRY(cudaStreamWaitEvent(st, df_side, 0));
        return DCD_OK;
    }

    // one full step through the deferred bodies
    dcd_status dfs_step(int64_t cnt)
    {
        const int cur = df_cur, nxt = (cur + 1) % 3, nn = (cur + 2) % 3;
        const int64_t rem1 = o.max_iters - done - cnt, rem2 = rem1 - o.s;
        const bool has1 = rem1 >= o.s, has2 = has1 && rem2 >= o.s;
        if (!df_chain) {  // prologue: this step's products (unless prepared), its recurrence on alpha and g
            if (la_cnt != cnt) {
                DCD_TRY(cudaMemcpyAsync(ctr_la + cur, ctr, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
                dcd_status r = lag_side(cur, cnt, st, nxt);
                if (r != DCD_OK) return r;
                la_cnt = cnt;
                df_prod = 0;  // the position after this step is in ctr_la[nxt]; nothing sampled there
            }
            DCD_TRY(dfs_chain_of(cur, cnt, false, st));
            if (has1) {  // step k+1's products and pending parts
                if (df_prod != o.s) {
                    dcd_status r = lag_side(nxt, o.s, st, nn);
                    if (r != DCD_OK) return r;
                    df_prod = o.s;
                }
                DCD_TRY(dfs_cross(nxt, cur, o.s, st));
                DCD_TRY(dfs_pending(nxt, cur, o.s, st));
            }
            df_chain = true;
        }
        const bool graphable = !graph_failed && has1 && has2;  // the steady state replays three graphs
        if (graphable && graph_df[cur]) {
            DCD_TRY(cudaGraphLaunch(graph_df[cur], st));
        } else if (graphable && df_direct[cur] >= 1) {
            DCD_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            const dcd_status sc = dfs_body(cur, cnt, has1, has2);
            cudaGraph_t graph = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(st, &graph);
            const bool ok = sc == DCD_OK && ec == cudaSuccess && graph != nullptr &&
                            cudaGraphInstantiate(&graph_df[cur], graph, 0) == cudaSuccess;
            if (ok) stats.gpu_launches_per_step = count_kernel_nodes(graph);
            if (graph) cudaGraphDestroy(graph);
            if (!ok) {
                cudaGetLastError();
                graph_df[cur] = nullptr;
                graph_failed = true;
                dcd_status r = dfs_body(cur, cnt, has1, has2);
                if (r != DCD_OK) return r;
            } else {
                DCD_TRY(cudaGraphLaunch(graph_df[cur], st));
            }
        } else {
            dcd_status r = dfs_body(cur, cnt, has1, has2);
            if (r != DCD_OK) return r;
            if (graphable) ++df_direct[cur];
        }
        df_cur = nxt;
        df_chain = has1;
        df_prod = has2 ? o.s : 0;
        la_cnt = has1 ? o.s : 0;  // the products of the next step are in place
        la_par = nxt < 2 ? nxt : 0;
        use_bufs(cur);  // the set just used is free (for a gradient recomputation)
        col_w_hi = std::max<int64_t>(col_w_hi, sb);  // any set's coefficients may fill sb entries
        return DCD_OK;
    }

    // ---- the look-ahead of the other steps (K-SVM; K-RR off the single-cluster path) ----
    // Step k+1's sample (from ctr_la, as above), its column map (CSR) or gathered rows (dense
    // tensor-core form) and its Gram, into buffer set q on stream s2; the helpers enqueue on the
    // plan's stream member, pointed at s2 meanwhile.  The sample leaves the following position in
    // ctr_la[qnext] (1 - q by default); `sampled` (optional) is recorded after it (after the
    // gathered rows in the dense tensor-core form).
    dcd_status lag_side(int q, int64_t cnt, cudaStream_t s2, int qnext = -1, cudaEvent_t sampled = nullptr)
    {
        const cudaStream_t keep = st;
        st = s2;
        use_bufs(q);
        const int64_t ncols = cnt * o.b;
        cudaError_t e =
            launch_sample(problem, o.seed, ctr_la + q, 0, m, o.b, cnt, S, err, st, ctr_la + (qnext < 0 ? 1 - q : qnext));
        const bool rows_gathered = tc && !csr;  // the cross product reads the gathered rows
        if (e == cudaSuccess && sampled && !rows_gathered) e = cudaEventRecord(sampled, st);
        if (e == cudaSuccess) e = gather(ncols);
        if (e == cudaSuccess && sampled && rows_gathered) e = cudaEventRecord(sampled, st);
        if (e == cudaSuccess) e = gram(ncols);
        st = keep;
        return cuda_status(e);
    }

    // one look-ahead step with products in set p: the recurrence, the block and the update on
    // st (the CSR block's first scatter forked beside the recurrence); the next step's products
    // (next > 0) into set 1 - p on st2, forked first and joined after the update
    dcd_status lag_body(int p, int64_t cnt, int64_t next)
    {
        // the forks are recorded first and the recurrence is launched before the kernels that
        // branch off them, so that it is the first of the step's kernels to take an SM
        const bool scatter = csr && use_csc;
        if (next) DCD_TRY(cudaEventRecord(la_fork, st));
        if (scatter) DCD_TRY(cudaEventRecord(csr_fork, st));
        use_bufs(p);
        const int64_t ncols = cnt * o.b;
        const double *rs = problem == 0 ? y : nullptr;
        FusedUpdate fu;  // a6 done by the K-RR recurrence when it can
        fu.alpha = alpha;
        fu.ctr = ctr;
        fu.ctr_advance = (uint64_t)cnt;
        if (problem == 0)
            DCD_TRY(launch_recur_dcd(Kss, tc ? 0 : 1, ldk, S, cnt, y, alpha, g, omega, nu, delta, w64,
                                     tc ? col_w : nullptr, err, st));
        else
            DCD_TRY(launch_recur_bdcd(Kss, tc ? 0 : 1, ldk, S, cnt, o.b, lambda, (double)m, g, tc ? 1 : 2, Lbuf,
                                      delta, w64, tc ? col_w : nullptr, &fu, err, st));
        if (next) {
            DCD_TRY(cudaStreamWaitEvent(st2, la_fork, 0));
            dcd_status r = lag_side(1 - p, next, st2);
            if (r != DCD_OK) return r;
            DCD_TRY(cudaEventRecord(la_join, st2));
            use_bufs(p);
        }
        if (scatter) {  // this step's first scatter through the transposed copy, beside the recurrence
            DCD_TRY(cudaStreamWaitEvent(csr_st, csr_fork, 0));
            DCD_TRY(launch_csr_csc_scatter_first(cm, cscop, cstep, !tc, csr_maxrow, ncols, csr_st));
            DCD_TRY(cudaEventRecord(csr_join, csr_st));
            csr_forked = true;
        }
        if (tc) DCD_TRY(clear_col_w_tail(ncols));
        if (csr)
            DCD_TRY(csr_apply(ncols, rs));
        else if (tc)
            DCD_TRY(block_tc_apply(ncols, rs));
        else
            DCD_TRY(launch_block_simt_f64(op.a64, op.lda, m, n, kp, nullptr, m, S, ncols, w64, rs, g, nullptr, 0,
                                          err, st));
        if (!fu.done) DCD_TRY(launch_update(S, delta, ncols, diag, alpha, g, ctr, (uint64_t)cnt, m, err, st));
        if (next) DCD_TRY(cudaStreamWaitEvent(st, la_join, 0));
        return DCD_OK;
    }

    dcd_status lag_step(int64_t cnt)
    {
        if (la_cnt != cnt) {  // nothing pending: this step's products first, on st
            DCD_TRY(cudaMemcpyAsync(ctr_la + la_par, ctr, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
            dcd_status r = lag_side(la_par, cnt, st);
            if (r != DCD_OK) return r;
            la_cnt = cnt;
        }
        const int p = la_par;
        const int64_t next = (o.max_iters - done - cnt) >= o.s ? o.s : 0;  // only full steps are prepared ahead
        if (next && cnt == o.s && !graph_failed) {
            if (graph_la[p]) {
                DCD_TRY(cudaGraphLaunch(graph_la[p], st));
            } else if (la_direct[p] >= 1) {
                DCD_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                const dcd_status sc = lag_body(p, cnt, next);
                cudaGraph_t graph = nullptr;
                const cudaError_t ec = cudaStreamEndCapture(st, &graph);
                const bool ok = sc == DCD_OK && ec == cudaSuccess && graph != nullptr &&
                                cudaGraphInstantiate(&graph_la[p], graph, 0) == cudaSuccess;
                if (ok) stats.gpu_launches_per_step = count_kernel_nodes(graph);
                if (graph) cudaGraphDestroy(graph);
                if (!ok) {
                    cudaGetLastError();
                    graph_la[p] = nullptr;
                    graph_failed = true;
                    dcd_status r = lag_body(p, cnt, next);
                    if (r != DCD_OK) return r;
                } else {
                    DCD_TRY(cudaGraphLaunch(graph_la[p], st));
                }
            } else {
                dcd_status r = lag_body(p, cnt, next);
                if (r != DCD_OK) return r;
                ++la_direct[p];
            }
        } else {
            dcd_status r = lag_body(p, cnt, next);
            if (r != DCD_OK) return r;
        }
        la_par = 1 - p;
        la_cnt = next;
        use_bufs(p);  // the set just used is free (for a gradient recomputation)
        return DCD_OK;
    }

    dcd_status outer_step(int64_t cnt, EventTimer &tm)
    {
        if (dfs && !tm.on && cnt == o.s) {
            dcd_status r = dfs_step(cnt);
            if (r != DCD_OK) return r;
            done += cnt;
            ++steps;
            return DCD_OK;
        }
        if (lag && !tm.on) {
            dcd_status r = lag_step(cnt);
            if (r != DCD_OK) return r;
            done += cnt;
            ++steps;
            return DCD_OK;
        }
        if (df && !tm.on && cnt == o.s) {
            dcd_status r = df_step(cnt);
            if (r != DCD_OK) return r;
            done += cnt;
            ++steps;
            return DCD_OK;
        }
        if (la && !df && !tm.on && recur_cluster_size((int)cnt, o.b, 2) > 0) {
            dcd_status r = la_step(cnt);
            if (r != DCD_OK) return r;
            done += cnt;
            ++steps;
            return DCD_OK;
        }
        if (la_cnt) return DCD_EINTERNAL;  // prepared products would be skipped
        const bool graphable = !tm.on && !(o.flags & DCD_FLAG_NO_GRAPH) && cnt == o.s && st != nullptr &&
                               st != cudaStreamLegacy && st != cudaStreamPerThread && !graph_failed;
        if (graphable && graph_exec) {
            DCD_TRY(cudaGraphLaunch(graph_exec, st));
        } else if (graphable && direct_full_steps >= 1) {
            // capture after one direct full step has set every kernel attribute
            DCD_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            EventTimer off;
            off.init(false, st);
            const dcd_status sc = enqueue_step(cnt, off);
            cudaGraph_t graph = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(st, &graph);
            bool ok = sc == DCD_OK && ec == cudaSuccess && graph != nullptr &&
                      cudaGraphInstantiate(&graph_exec, graph, 0) == cudaSuccess;
            if (ok) stats.gpu_launches_per_step = count_kernel_nodes(graph);
            if (graph) cudaGraphDestroy(graph);
            if (!ok) {
                cudaGetLastError();
                graph_exec = nullptr;
                graph_failed = true;
                dcd_status s2 = enqueue_step(cnt, tm);
                if (s2 != DCD_OK) return s2;
            } else {
                DCD_TRY(cudaGraphLaunch(graph_exec, st));
            }
        } else {
            dcd_status s2 = enqueue_step(cnt, tm);
            if (s2 != DCD_OK) return s2;
            if (graphable) ++direct_full_steps;
        }
        done += cnt;
        ++steps;
        return DCD_OK;
    }

    static int count_kernel_nodes(cudaGraph_t graph)
    {
        size_t nn = 0;
        if (cudaGraphGetNodes(graph, nullptr, &nn) != cudaSuccess || nn == 0) return 0;
        std::vector<cudaGraphNode_t> nodes(nn);
        if (cudaGraphGetNodes(graph, nodes.data(), &nn) != cudaSuccess) return 0;
        int k = 0;
        for (size_t i = 0; i < nn; ++i) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
        }
        return k;
    }

    // One outer step in the printed order of Algorithms 2 / 4: Q_k = K(A, A_S) stored (m x ncols),
    // the step's gradient values from Q_k^T alpha, the Gram from the rows of Q_k at S, the
    // recurrence, alpha_S += delta.  The cached gradient is not used.
    dcd_status literal_step(int64_t cnt, EventTimer &tm)
    {
        const int64_t ncols = cnt * o.b;
        tm.start();
        DCD_TRY(launch_sample(problem, o.seed, ctr, 0, m, o.b, cnt, S, err, st));
        DCD_TRY(gather(ncols));
        tm.stop(stats.ms_sample);
        tm.start();
        if (tc) {
            TcOperand Aop{op.packed, m, op.n_pad, op.kind, op.row_s};
            TcOperand Bop{As, ncols, op.n_pad, op.kind, col_s, S};
            DCD_TRY(launch_block_tc(Aop, Bop, kp, op.row_h, col_h, nullptr, nullptr, nullptr, (float *)Qbuf, sb, m,
                                    ncols, err, st));
        } else {
            DCD_TRY(launch_block_simt_f64(op.a64, op.lda, m, n, kp, nullptr, m, S, ncols, nullptr, nullptr, nullptr,
                                          (double *)Qbuf, sb, err, st));
        }
        tm.stop(stats.ms_block);
        tm.start();
        DCD_TRY(launch_literal_terms(Qbuf, tc ? 0 : 1, sb, m, ncols, S, problem, y, alpha, 1.0 / lambda, diag,
                                     lit_part, lit_blocks, lit_g, Kss, ldk, st));
        tm.stop(stats.ms_gram);
        tm.start();
        FusedUpdate fu;
        fu.alpha = alpha;
        fu.ctr = ctr;
        fu.ctr_advance = (uint64_t)cnt;
        if (problem == 0)
            DCD_TRY(launch_recur_dcd(Kss, tc ? 0 : 1, ldk, S, cnt, y, alpha, lit_g, omega, nu, delta, w64,
                                     tc ? col_w : nullptr, err, st));
        else
            DCD_TRY(launch_recur_bdcd(Kss, tc ? 0 : 1, ldk, S, cnt, o.b, lambda, (double)m, lit_g, tc ? 1 : 2, Lbuf,
                                      delta, w64, tc ? col_w : nullptr, &fu, err, st));
        tm.stop(stats.ms_recur);
        tm.start();
        if (!fu.done) DCD_TRY(launch_update(S, delta, ncols, diag, alpha, lit_g, ctr, (uint64_t)cnt, m, err, st));
        tm.stop(stats.ms_update);
        tm.flush();
        return DCD_OK;
    }

    dcd_status enqueue_step(int64_t cnt, EventTimer &tm)
    {
        if (literal) return literal_step(cnt, tm);
        const int64_t ncols = cnt * o.b;
        const double *rs = problem == 0 ? y : nullptr;
        tm.start();
        DCD_TRY(launch_sample(problem, o.seed, ctr, 0, m, o.b, cnt, S, err, st));
        DCD_TRY(gather(ncols));
        tm.stop(stats.ms_sample);
        // CSR through the transposed copy: the first chunk's incidences are gathered beside the
        // Gram and the recurrence (not under the phase timers, which time the block as a whole)
        if (csr && use_csc && !tm.on) DCD_TRY(csr_fork_scatter(ncols));
        tm.start();
        DCD_TRY(gram(ncols));
        tm.stop(stats.ms_gram);
        tm.start();
        FusedUpdate fu;  // a6 done by the recurrence when it can
        fu.alpha = alpha;
        fu.ctr = ctr;
        fu.ctr_advance = (uint64_t)cnt;
        if (problem == 0)
            DCD_TRY(launch_recur_dcd(Kss, tc ? 0 : 1, ldk, S, cnt, y, alpha, g, omega, nu, delta, w64,
                                     tc ? col_w : nullptr, err, st));
        else
            DCD_TRY(launch_recur_bdcd(Kss, tc ? 0 : 1, ldk, S, cnt, o.b, lambda, (double)m, g, tc ? 1 : 2, Lbuf,
                                      delta, w64, tc ? col_w : nullptr, &fu, err, st));
        if (tc) DCD_TRY(clear_col_w_tail(ncols));
        tm.stop(stats.ms_recur);
        tm.start();
        if (csr)
            DCD_TRY(csr_apply(ncols, rs));
        else if (tc)
            DCD_TRY(block_tc_apply(ncols, rs));
        else
            DCD_TRY(launch_block_simt_f64(op.a64, op.lda, m, n, kp, nullptr, m, S, ncols, w64, rs, g, nullptr, 0, err,
                                          st));
        tm.stop(stats.ms_block);
        tm.start();
        if (!fu.done) DCD_TRY(launch_update(S, delta, ncols, diag, alpha, g, ctr, (uint64_t)cnt, m, err, st));
        tm.stop(stats.ms_update);
        tm.flush();
        return DCD_OK;
    }

    // Runs up to max_steps outer steps (all remaining if < 0), then measures
    // the convergence metric and publishes alpha / grad / stats.
    dcd_status run_steps(int64_t max_steps, dcd_stats *st_out)
    {
        dcd_status s0 = begin();
        if (s0 != DCD_OK) return s0;
        EventTimer tm;
        tm.init((o.flags & DCD_FLAG_PHASE_TIMERS) != 0, st);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
        const int check_every = o.check_every > 0 ? o.check_every : 0;
        for (int64_t k = 0; !finished() && (max_steps < 0 || k < max_steps); ++k) {
            const int64_t cnt = std::min<int64_t>(o.s, o.max_iters - done);
            s0 = outer_step(cnt, tm);
            if (s0 != DCD_OK) break;
            if (check_every && o.tol > 0 && steps % check_every == 0 && done < o.max_iters) {
                tm.start();
                s0 = check_converged();
                tm.stop(stats.ms_check);
                tm.flush();
                if (s0 != DCD_OK) break;
            }
        }
        // the literal order keeps no gradient between steps: recompute it from alpha
        if (s0 == DCD_OK && literal) {
            s0 = cuda_status(launch_init_grad(problem, y, alpha, diag, m, g, st));
            if (s0 == DCD_OK) s0 = full_pass();
        }
        // the metric is measured at check points and when the budget ends;
        // an intermediate dcd_plan_run without a tolerance leaves it NaN
        if (s0 == DCD_OK && (finished() || o.tol > 0)) {
            if (conv)
                ;  // measured (and confirmed) at the check point that converged
            else if (o.tol > 0)
                s0 = check_converged(finished());
            else
                s0 = measure(metric, primal, dual, ynorm2);
        } else if (s0 == DCD_OK) {
            metric = primal = dual = NAN;
        }
        dcd_status se = check_device_error();
        if (s0 == DCD_OK) s0 = se;
        if (s0 == DCD_OK) s0 = publish();
        cudaEventRecord(e1, st);
        cudaStreamSynchronize(st);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ms_accum += ms;
        stats.iters_done = done;
        stats.outer_steps = steps;
        stats.converged = conv ? 1 : 0;
        stats.final_metric = metric;
        stats.primal = primal;
        stats.dual = dual;
        stats.ms_total = ms_accum;
        if (st_out) *st_out = stats;
        if (s0 != DCD_OK) return s0;
        if (o.tol > 0 && !conv && done >= o.max_iters) return DCD_ENOTCONV;
        return DCD_OK;
    }

    // alpha (host-io only) and the cached gradient back to the caller.
    dcd_status publish()
    {
        const bool host = (o.flags & DCD_FLAG_HOST_IO) != 0;
        if (host) {
            DCD_TRY(cudaMemcpyAsync(alpha_host, alpha, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
            if (grad_out) DCD_TRY(cudaMemcpyAsync(grad_out, g, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
        }
        return DCD_OK;  // device io: g is the caller's grad array (or internal)
    }

    dcd_status run(dcd_stats *st_out) { return run_steps(-1, st_out); }

    // Enqueues up to max_steps outer steps with no host synchronisation and
    // no convergence check; device-side errors surface at the next run_steps.
    dcd_status enqueue_steps(int64_t max_steps, int64_t *enqueued)
    {
        int64_t k = 0;
        dcd_status s0 = begin();
        if (s0 == DCD_OK) {
            EventTimer off;
            off.init(false, st);
            for (; !finished() && k < max_steps; ++k) {
                s0 = outer_step(std::min<int64_t>(o.s, o.max_iters - done), off);
                if (s0 != DCD_OK) break;
            }
        }
        stats.iters_done = done;
        stats.outer_steps = steps;
        if (enqueued) *enqueued = k;
        return s0;
    }

    double *alpha_host = nullptr;
};

dcd_status validate_opts(const dcd_opts *o, int64_t m, int problem, bool csr)
{
    if (!o) return DCD_EINVAL;
    if (o->s < 1 || o->b < 1 || o->max_iters < 0) return DCD_EINVAL;
    if (problem == 0 && o->b != 1) return DCD_EINVAL;
    if (o->b > B_MAX || o->b > m) return DCD_EINVAL;
    if ((int64_t)o->s * o->b > SB_MAX) return DCD_EINVAL;
    if (!(std::isfinite(o->tol) && o->tol >= 0.0) || o->check_every < 0) return DCD_EINVAL;
    if (o->prec == DCD_PREC_REFRESH) return DCD_EUNSUPPORTED;  // an apply-only precision
    if ((o->flags & DCD_FLAG_LITERAL) && (csr || o->tol != 0.0)) return DCD_EINVAL;
    if (o->prec != DCD_PREC_FP64 && !is_tc(o->prec)) return DCD_EINVAL;
    if (o->prec == DCD_PREC_FP8 && csr) return DCD_EUNSUPPORTED;  // the CSR block has no fp8 form
    if (is_tc(o->prec) && !csr && !tc_available()) return DCD_EUNSUPPORTED;  // CSR: CUDA cores
    return DCD_OK;
}

dcd_status prepare(Solver &sv, const double *y, double *alpha, double *grad)
{
    if (!y || !alpha) return DCD_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DCD_ECUDA;
    if (sv.o.flags & DCD_FLAG_HOST_IO) sv.alpha_host = alpha;
    sv.grad_out = grad;
    return sv.setup(y, alpha, grad);
}

dcd_status init_svm(Solver &sv, const dcd_matrix *A, const dcd_kernel *k, int32_t loss, double C, const dcd_opts *o,
                    void *stream)
{
    dcd_status s = validate_dense(A);
    if (s != DCD_OK) return s;
    if ((s = validate_kernel(k)) != DCD_OK) return s;
    if (loss != 1 && loss != 2) return DCD_EINVAL;
    if (!finite_pos(C)) return DCD_EINVAL;
    if ((s = validate_opts(o, A->m, 0, A->fmt == DCD_CSR)) != DCD_OK) return s;
    sv.problem = 0;
    sv.A = A;
    sv.kp = to_kp(k);
    sv.loss = loss;
    sv.C = C;
    sv.omega = loss == 2 ? 1.0 / (2.0 * C) : 0.0;
    sv.nu = loss == 2 ? INFINITY : C;
    sv.diag = sv.omega;
    sv.o = *o;
    sv.st = (cudaStream_t)stream;
    return DCD_OK;
}

dcd_status init_krr(Solver &sv, const dcd_matrix *A, const dcd_kernel *k, double lambda, const dcd_opts *o,
                    void *stream)
{
    dcd_status s = validate_dense(A);
    if (s != DCD_OK) return s;
    if ((s = validate_kernel(k)) != DCD_OK) return s;
    if (!finite_pos(lambda)) return DCD_EINVAL;
    if ((s = validate_opts(o, A->m, 1, A->fmt == DCD_CSR)) != DCD_OK) return s;
    sv.problem = 1;
    sv.A = A;
    sv.kp = to_kp(k);
    sv.lambda = lambda;
    sv.diag = (double)A->m;
    sv.o = *o;
    sv.st = (cudaStream_t)stream;
    return DCD_OK;
}

}  // namespace
}  // namespace dcd

using namespace dcd;

struct dcd_plan {
    Solver sv;
};

extern "C" dcd_status dcd_svm_solve(const dcd_matrix *A, const double *y, const dcd_kernel *k, int32_t loss, double C,
                                    const dcd_opts *o, double *alpha, double *grad, dcd_stats *st, void *stream)
{
    Solver sv;
    dcd_status s = init_svm(sv, A, k, loss, C, o, stream);
    if (s == DCD_OK) s = prepare(sv, y, alpha, grad);
    if (s == DCD_OK) s = sv.run(st);
    return s;
}

extern "C" dcd_status bdcd_krr_solve(const dcd_matrix *A, const double *y, const dcd_kernel *k, double lambda,
                                     const dcd_opts *o, double *alpha, double *grad, dcd_stats *st, void *stream)
{
    Solver sv;
    dcd_status s = init_krr(sv, A, k, lambda, o, stream);
    if (s == DCD_OK) s = prepare(sv, y, alpha, grad);
    if (s == DCD_OK) s = sv.run(st);
    return s;
}

extern "C" dcd_status dcd_svm_plan_create(const dcd_matrix *A, const double *y, const dcd_kernel *k, int32_t loss,
                                          double C, const dcd_opts *o, double *alpha, double *grad, void *stream,
                                          dcd_plan **plan)
{
    if (!plan) return DCD_EINVAL;
    *plan = nullptr;
    dcd_plan *p = new (std::nothrow) dcd_plan;
    if (!p) return DCD_ENOMEM;
    dcd_status s = init_svm(p->sv, A, k, loss, C, o, stream);
    if (s == DCD_OK) s = prepare(p->sv, y, alpha, grad);
    if (s != DCD_OK) {
        delete p;
        return s;
    }
    *plan = p;
    return DCD_OK;
}

extern "C" dcd_status bdcd_krr_plan_create(const dcd_matrix *A, const double *y, const dcd_kernel *k, double lambda,
                                           const dcd_opts *o, double *alpha, double *grad, void *stream,
                                           dcd_plan **plan)
{
    if (!plan) return DCD_EINVAL;
    *plan = nullptr;
    dcd_plan *p = new (std::nothrow) dcd_plan;
    if (!p) return DCD_ENOMEM;
    dcd_status s = init_krr(p->sv, A, k, lambda, o, stream);
    if (s == DCD_OK) s = prepare(p->sv, y, alpha, grad);
    if (s != DCD_OK) {
        delete p;
        return s;
    }
    *plan = p;
    return DCD_OK;
}

extern "C" dcd_status dcd_plan_run(dcd_plan *plan, int64_t max_outer_steps, dcd_stats *st)
{
    if (!plan) return DCD_EINVAL;
    return plan->sv.run_steps(max_outer_steps, st);
}

extern "C" dcd_status dcd_plan_enqueue(dcd_plan *plan, int64_t outer_steps, int64_t *enqueued)
{
    if (enqueued) *enqueued = 0;
    if (!plan || outer_steps < 0) return DCD_EINVAL;
    return plan->sv.enqueue_steps(outer_steps, enqueued);
}

extern "C" dcd_status dcd_plan_destroy(dcd_plan *plan)
{
    if (!plan) return DCD_OK;
    cudaStream_t st = plan->sv.st;
    delete plan;
    return cuda_status(cudaStreamSynchronize(st));
}

extern "C" const char *dcd_status_string(int32_t s)
{
    switch (s) {
    case DCD_OK: return "DCD_OK";
    case DCD_EINVAL: return "DCD_EINVAL: invalid argument";
    case DCD_ENOMEM: return "DCD_ENOMEM: device allocation failed";
    case DCD_ECUDA: return "DCD_ECUDA: CUDA runtime error";
    case DCD_ETIMEOUT: return "DCD_ETIMEOUT: bounded device wait expired";
    case DCD_ENOTCONV: return "DCD_ENOTCONV: iteration budget reached before tolerance";
    case DCD_EINTERNAL: return "DCD_EINTERNAL: device-side check failed";
    case DCD_ENOTSPD: return "DCD_ENOTSPD: block system not positive definite";
    case DCD_EUNSUPPORTED: return "DCD_EUNSUPPORTED: not implemented in this build";
    default: return "unknown dcd_status";
    }
}

extern "C" dcd_status dcd_sample_indices(int32_t method, uint64_t seed, int64_t m, int32_t b, uint64_t first,
                                         int64_t count, int32_t *out, void *stream)
{
    if ((method != 0 && method != 1) || m < 1 || m > INT32_MAX || count < 0 || !out) return DCD_EINVAL;
    if (method == 1 && (b < 1 || b > m)) return DCD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = launch_sample(method, seed, nullptr, first, m, method == 1 ? b : 1, count, out, nullptr, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_status(e);
}

namespace {

// Scratch memory of one component call, freed (stream-ordered) on return.
struct ComponentBufs {
    void *mem = nullptr;
    cudaStream_t st = nullptr;
    ~ComponentBufs()
    {
        if (mem) cudaFreeAsync(mem, st);
    }
};

size_t place(size_t &cur, size_t bytes, size_t align = 1024)
{
    size_t off = (cur + align - 1) / align * align;
    cur = off + bytes;
    return off;
}

dcd_status component_check(const dcd_matrix *A, const dcd_kernel *k, int32_t prec, bool apply = false)
{
    dcd_status s = validate_dense(A);
    if (s != DCD_OK) return s;
    if ((s = validate_kernel(k)) != DCD_OK) return s;
    if (prec == DCD_PREC_REFRESH) {  // the accurate epilogue: dense apply form only
        if (!apply || A->fmt == DCD_CSR || A->dtype == DCD_FP8E4M3) return DCD_EUNSUPPORTED;
        return tc_available() ? DCD_OK : DCD_EUNSUPPORTED;
    }
    if (prec != DCD_PREC_FP64 && !is_tc(prec)) return DCD_EINVAL;
    if (prec == DCD_PREC_FP8 && A->fmt == DCD_CSR) return DCD_EUNSUPPORTED;
    if (is_tc(prec) && A->fmt != DCD_CSR && !tc_available()) return DCD_EUNSUPPORTED;
    return DCD_OK;
}

dcd_status finish_component(int *err, cudaStream_t st)
{
    int he = 0;
    DCD_TRY(cudaMemcpyAsync(&he, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    DCD_TRY(cudaStreamSynchronize(st));
    if (he == DEV_TIMEOUT) return DCD_ETIMEOUT;
    if (he == DEV_BAD_INDEX || he == DEV_BAD_VALUE) return DCD_EINVAL;
    return he ? DCD_EINTERNAL : DCD_OK;
}

// The CSR form of component_block: the CUDA-core SpMM block, FP64 in the
// FP64 mode and FP32 otherwise (device arrays only).
dcd_status component_block_csr(const dcd_matrix *A, const KernelParams &kp, int32_t prec, const int32_t *rows,
                               int64_t nrows, const int32_t *cols, int64_t ncols, const double *w, const double *rs,
                               double *g, void *out, int64_t ldo, cudaStream_t st)
{
    const bool fp64 = !is_tc(prec);
    const int64_t m = A->m;
    int64_t nnz = 0;
    DCD_TRY(cudaMemcpyAsync(&nnz, A->row_ptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    DCD_TRY(cudaStreamSynchronize(st));
    if (nnz < 0) return DCD_EINVAL;
    const bool conv32 = !fp64 && A->dtype != DCD_F32, conv64 = fp64 && A->dtype != DCD_F64;
    ComponentBufs cb, cb2;
    cb.st = cb2.st = st;
    size_t cur = 0;
    const size_t oe = place(cur, 256), ov = place(cur, conv32 ? 4 * (size_t)nnz : conv64 ? 8 * (size_t)nnz : 0);
    const size_t on32 = place(cur, 4 * (size_t)m), on64 = place(cur, 8 * (size_t)m);
    const size_t ow = place(cur, (w && !fp64) ? 4 * (size_t)ncols : 0);
    DCD_TRY(malloc_async(&cb.mem, cur + 1024, st));
    char *base = (char *)cb.mem;
    int *err = (int *)(base + oe);
    DCD_TRY(cudaMemsetAsync(err, 0, 4 * sizeof(int), st));
    CsrOperand ca;
    ca.row_ptr = A->row_ptr;
    ca.col_idx = A->col_idx;
    ca.m = m;
    ca.n = A->n;
    ca.nnz = nnz;
    ca.norm32 = (float *)(base + on32);
    ca.norm64 = (double *)(base + on64);
    if (fp64) {
        ca.vals64 = conv64 ? (const double *)(base + ov) : (const double *)A->values;
        if (conv64)
            DCD_TRY(launch_pack_rows(A->values, A->dtype, nnz, 1, nnz, nullptr, base + ov, PACK_F64, nnz, 1, err, st));
    } else {
        ca.vals32 = conv32 ? (const float *)(base + ov) : (const float *)A->values;
        if (conv32) DCD_TRY(launch_f64_to_f32((const double *)A->values, nnz, (float *)(base + ov), st));
    }
    DCD_TRY(launch_csr_prep(ca, err + 2, err + 3, st));
    int h[2] = {0, 0};
    DCD_TRY(cudaMemcpyAsync(h, err + 2, sizeof(h), cudaMemcpyDeviceToHost, st));
    DCD_TRY(cudaStreamSynchronize(st));
    if (h[0]) return DCD_EINVAL;
    const int64_t cap = std::max<int64_t>(1, ncols * (int64_t)h[1]);
    const size_t cmb = csr_colmap_bytes(A->n, cap);
    DCD_TRY(malloc_async(&cb2.mem, cmb, st));
    DCD_TRY(cudaMemsetAsync(cb2.mem, 0, cmb, st));
    CsrColMap cm = csr_colmap_carve(cb2.mem, A->n, cap);
    float *w32 = (w && !fp64) ? (float *)(base + ow) : nullptr;
    if (w32) DCD_TRY(launch_f64_to_f32(w, ncols, w32, st));
    // the apply over every row: through the transposed copy when it pays (its pair table comes
    // with the column map)
    ComponentBufs cb3, cb4;
    cb3.st = cb4.st = st;
    CscOperand C;
    CscStep W;
    bool use = false;
    if (!out && !rows && nrows == m) {
        dcd_status cs = csc_choose(ca, fp64, ncols, h[1], err + 1, &cb3.mem, &C, &cb4.mem, &W, &cm, &use, st);
        if (cs != DCD_OK) return cs;
    }
    DCD_TRY(launch_csr_colmap(ca, cols, ncols, cm, err, st));
    if (use) {
        DCD_TRY(launch_csr_apply_csc(ca, cm, C, W, fp64, h[1], kp, cols, ncols, w32, w, rs, g, st));
        return finish_component(err, st);
    }
    DCD_TRY(launch_csr_block(ca, cm, fp64, kp, rows, nrows, cols, ncols, w32, w, rs, g, out, ldo, st));
    return finish_component(err, st);
}

// Column points given as a matrix of their own: rows 0..ncols-1 of P stand
// for the columns, and the own-sample rule of the tensor-core epilogue (a
// squared distance of exactly 0 between a row and itself) compares global
// ids: row_id0 + i for row i of A, col_ids[c] for row c of P (no column
// matches when col_ids is null).  The FP64 form sums coordinate differences
// and needs no ids.
struct PointsArg {
    const dcd_matrix *P = nullptr;
    int64_t row_id0 = 0;
    const int32_t *col_ids = nullptr;
};

// Runs the kernel block on rows `rows` (or the first nrows) against columns
// `cols` (or against the rows of pts->P): store into `out` (w == nullptr) or
// apply into g.
dcd_status component_block(const dcd_matrix *A, const dcd_kernel *k, int32_t prec, const int32_t *rows,
                           int64_t nrows, const int32_t *cols, int64_t ncols, const double *w, const double *rs,
                           double *g, void *out, int64_t ldo, cudaStream_t st, const PointsArg *pts = nullptr)
{
    const KernelParams kp = to_kp(k);
    if (A->fmt == DCD_CSR) return component_block_csr(A, kp, prec, rows, nrows, cols, ncols, w, rs, g, out, ldo, st);
    const dcd_matrix *P = pts ? pts->P : A;  // the matrix holding the column points
    ComponentBufs cb;
    cb.st = st;
    if (!is_tc(prec) && prec != DCD_PREC_REFRESH) {
        const bool pack = A->dtype != DCD_F64, packp = pts && P->dtype != DCD_F64;
        size_t cur = 0;
        size_t oe = place(cur, 256);
        size_t op64 = place(cur, pack ? sizeof(double) * A->m * A->n : 0);
        size_t opp = place(cur, packp ? sizeof(double) * P->m * P->n : 0);
        DCD_TRY(malloc_async(&cb.mem, cur + 1024, st));
        char *base = (char *)cb.mem;
        int *err = (int *)(base + oe);
        DCD_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
        const double *a64 = (const double *)A->values;
        int64_t lda = A->ld;
        if (pack) {
            double *p = (double *)(base + op64);
            DCD_TRY(launch_pack_rows(A->values, A->dtype, A->ld, A->m, A->n, nullptr, p, 2, A->n, A->m, err, st,
                                     A->row_scale));
            a64 = p;
            lda = A->n;
        }
        const double *p64 = nullptr;
        int64_t ldp = 0;
        if (pts) {
            p64 = (const double *)P->values;
            ldp = P->ld;
            if (packp) {
                double *p = (double *)(base + opp);
                DCD_TRY(launch_pack_rows(P->values, P->dtype, P->ld, P->m, P->n, nullptr, p, 2, P->n, P->m, err, st,
                                         P->row_scale));
                p64 = p;
                ldp = P->n;
            }
        }
        DCD_TRY(launch_block_simt_f64(a64, lda, A->m, A->n, kp, rows, nrows, pts ? nullptr : cols, ncols, w, rs, g,
                                      (double *)out, ldo, err, st, p64, ldp, pts ? P->m : 0));
        return finish_component(err, st);
    }
    const bool accurate = prec == DCD_PREC_REFRESH;
    const bool sliced = accurate && (A->n + 63) / 64 * 64 <= SLICED_N_MAX;
    const int pk = sliced ? PACK_SLICED : accurate ? PACK_TF32X3 : pack_kind(prec);
    const int kb = k_block_elems(pk);
    const int64_t n_pad = (A->n + kb - 1) / kb * kb;
    const size_t rb = (size_t)packed_row_bytes(pk, n_pad);
    const int64_t cpad = (ncols + 255) / 256 * 256;
    size_t cur = 0;
    size_t oe = place(cur, 256);
    size_t oa = place(cur, (size_t)nrows * rb);
    size_t ob = place(cur, (size_t)ncols * rb);
    size_t orh = place(cur, sizeof(float) * nrows);
    size_t och = place(cur, sizeof(float) * cpad);
    size_t ocw = place(cur, sizeof(float) * cpad);
    const bool fp8 = pk == PACK_FP8, fp16 = pk == PACK_FP16;
    size_t ors = place(cur, (fp8 || fp16 || sliced) ? sizeof(float) * nrows : 0);
    size_t ocs = place(cur, (fp8 || fp16 || sliced) ? sizeof(float) * cpad : 0);
    size_t orl = place(cur, accurate ? sizeof(float) * nrows : 0);
    size_t ocl = place(cur, accurate ? sizeof(float) * cpad : 0);
    // points form: global row ids (when offset) and column ids (-1 without col_ids)
    const bool rid = pts && pts->row_id0 != 0, cid = pts && !pts->col_ids;
    size_t ori = place(cur, rid ? sizeof(int32_t) * nrows : 0);
    size_t oci = place(cur, cid ? sizeof(int32_t) * ncols : 0);
    // the apply form's balanced split over CTA pairs
    TcSplit sp;
    if (!out) {
        int dev = 0, sms = 0;
        DCD_TRY(cudaGetDevice(&dev));
        DCD_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        sp.pairs = std::max(sms / 2, 1);
        sp.chunks = tc_split_chunks(ncols);
    }
    size_t osp = place(cur, sizeof(double) * tc_split_part_elems(sp.pairs, sp.chunks));
    size_t osc = place(cur, sizeof(unsigned) * 2 * sp.pairs);
    DCD_TRY(malloc_async(&cb.mem, cur + 1024, st));
    char *base = (char *)cb.mem;
    int *err = (int *)(base + oe);
    void *pa = base + oa, *pb = base + ob;
    float *rh = (float *)(base + orh), *ch = (float *)(base + och), *cw = (float *)(base + ocw);
    float *rsa = (fp8 || fp16 || sliced) ? (float *)(base + ors) : nullptr;
    float *rsb = (fp8 || fp16 || sliced) ? (float *)(base + ocs) : nullptr;
    DCD_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    DCD_TRY(cudaMemsetAsync(ch, 0, sizeof(float) * cpad, st));
    DCD_TRY(cudaMemsetAsync(cw, 0, sizeof(float) * cpad, st));
    if (!out) {
        sp.part = (double *)(base + osp);
        sp.cnt = (unsigned *)(base + osc);
        DCD_TRY(cudaMemsetAsync(sp.cnt, 0, sizeof(unsigned) * 2 * sp.pairs, st));
    }
    const int32_t *pcols = pts ? nullptr : cols;  // rows of P: the first ncols
    if (sliced) {
        DCD_TRY(cudaMemsetAsync(rsb, 0, sizeof(float) * cpad, st));
        DCD_TRY(launch_pack_sliced(A->values, A->dtype, A->ld, A->m, A->n, rows, pa, n_pad, nrows, rsa, err, st,
                                   A->row_scale));
        DCD_TRY(launch_pack_sliced(P->values, P->dtype, P->ld, P->m, P->n, pcols, pb, n_pad, ncols, rsb, err, st,
                                   P->row_scale));
    } else if (fp8) {
        DCD_TRY(cudaMemsetAsync(rsb, 0, sizeof(float) * cpad, st));
        DCD_TRY(launch_quantize_rows(A->values, A->dtype, A->ld, A->m, A->n, rows, A->row_scale, (uint8_t *)pa, n_pad,
                                     rsa, nrows, err, st));
        DCD_TRY(launch_quantize_rows(P->values, P->dtype, P->ld, P->m, P->n, pcols, P->row_scale, (uint8_t *)pb,
                                     n_pad, rsb, ncols, err, st));
    } else if (fp16) {
        // one power-of-two scale for both operands: the largest magnitude over every row of A (the
        // scale the solver's operand takes) and of the points (err[2])
        unsigned *gbits = (unsigned *)(err + 2);
        DCD_TRY(cudaMemsetAsync(gbits, 0, sizeof(unsigned), st));
        DCD_TRY(cudaMemsetAsync(rsb, 0, sizeof(float) * cpad, st));
        DCD_TRY(launch_absmax_rows(A->values, A->dtype, A->ld, A->m, A->n, nullptr, A->m, gbits, err, st,
                                   A->row_scale));
        if (pts)
            DCD_TRY(launch_absmax_rows(P->values, P->dtype, P->ld, P->m, P->n, nullptr, P->m, gbits, err, st,
                                       P->row_scale));
        DCD_TRY(launch_pack_fp16(A->values, A->dtype, A->ld, A->m, A->n, rows, pa, n_pad, nrows, rsa, gbits, err, st,
                                 A->row_scale));
        DCD_TRY(launch_pack_fp16(P->values, P->dtype, P->ld, P->m, P->n, pcols, pb, n_pad, ncols, rsb, gbits, err,
                                 st, P->row_scale));
    } else {
        DCD_TRY(launch_pack_rows(A->values, A->dtype, A->ld, A->m, A->n, rows, pa, pk, n_pad, nrows, err, st,
                                 A->row_scale));
        DCD_TRY(launch_pack_rows(P->values, P->dtype, P->ld, P->m, P->n, pcols, pb, pk, n_pad, ncols, err, st,
                                 P->row_scale));
    }
    float *rl = accurate ? (float *)(base + orl) : nullptr, *cl = accurate ? (float *)(base + ocl) : nullptr;
    if (cl) DCD_TRY(cudaMemsetAsync(cl, 0, sizeof(float) * cpad, st));
    DCD_TRY(launch_row_terms(pa, pk, n_pad, nrows, kp, rh, st, rsa, rl));
    DCD_TRY(launch_row_terms(pb, pk, n_pad, ncols, kp, ch, st, rsb, cl));
    if (w) DCD_TRY(launch_f64_to_f32(w, ncols, cw, st));
    const int32_t *aids = rows, *bids = cols;
    if (pts) {
        aids = nullptr;  // row i: id i, or row_id0 + i from the array below
        bids = pts->col_ids;
        if (rid) {
            int32_t *ids = (int32_t *)(base + ori);
            DCD_TRY(launch_iota(ids, nrows, pts->row_id0, st));
            aids = ids;
        }
        if (cid) {
            int32_t *ids = (int32_t *)(base + oci);
            DCD_TRY(cudaMemsetAsync(ids, 0xff, sizeof(int32_t) * ncols, st));  // -1: matches no row
            bids = ids;
        }
    }
    TcOperand Aop{pa, nrows, n_pad, pk, rsa, aids}, Bop{pb, ncols, n_pad, pk, rsb, bids};
    TcAccurate acc;
    acc.w64 = w;
    acc.row_hl = rl;
    acc.col_hl = cl;
    DCD_TRY(launch_block_tc(Aop, Bop, kp, rh, ch, w ? cw : nullptr, rs, g, (float *)out, ldo, nrows, ncols, err, st,
                            false, &sp, false, 0, accurate ? &acc : nullptr));
    return finish_component(err, st);
}

}  // namespace

extern "C" dcd_status dcd_quantize_e4m3(const dcd_matrix *A, uint8_t *q, int64_t ldq, float *row_scale,
                                        void *stream)
{
    if (!A || A->fmt != DCD_DENSE || A->m < 1 || A->n < 1 || A->ld < A->n || !A->values || A->m > INT32_MAX)
        return DCD_EINVAL;
    if (A->dtype != DCD_F64 && A->dtype != DCD_F32 && A->dtype != DCD_BF16) return DCD_EINVAL;
    if (!q || !row_scale || ldq < A->n) return DCD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    ComponentBufs cb;
    cb.st = st;
    DCD_TRY(malloc_async(&cb.mem, 256, st));
    int *err = (int *)cb.mem;
    DCD_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    DCD_TRY(launch_quantize_rows(A->values, A->dtype, A->ld, A->m, A->n, nullptr, nullptr, q, ldq, row_scale, A->m, err,
                                 st));
    return finish_component(err, st);
}

extern "C" dcd_status dcd_kernel_block(const dcd_matrix *A, const dcd_kernel *k, int32_t prec, const int32_t *rows,
                                       int64_t nrows, const int32_t *cols, int64_t ncols, void *out, int64_t ldo,
                                       void *stream)
{
    dcd_status s = component_check(A, k, prec);
    if (s != DCD_OK) return s;
    if (nrows < 0 || ncols < 0 || !cols || !out || ldo < ncols) return DCD_EINVAL;
    if (!rows && nrows > A->m) return DCD_EINVAL;
    if (nrows == 0 || ncols == 0) return DCD_OK;
    return component_block(A, k, prec, rows, nrows, cols, ncols, nullptr, nullptr, nullptr, out, ldo,
                           (cudaStream_t)stream);
}

extern "C" dcd_status dcd_kernel_block_apply(const dcd_matrix *A, const dcd_kernel *k, int32_t prec,
                                             const int32_t *cols, int64_t ncols, const double *w,
                                             const double *rowscale, double *g, void *stream)
{
    dcd_status s = component_check(A, k, prec, true);
    if (s != DCD_OK) return s;
    if (ncols < 0 || (ncols > 0 && (!cols || !w)) || !g) return DCD_EINVAL;
    if (ncols == 0) return DCD_OK;
    return component_block(A, k, prec, nullptr, A->m, cols, ncols, w, rowscale, g, nullptr, 0, (cudaStream_t)stream);
}

extern "C" dcd_status dcd_kernel_block_apply_points(const dcd_matrix *A, int64_t row_id0, const dcd_matrix *P,
                                                    const int32_t *col_ids, const dcd_kernel *k, int32_t prec,
                                                    const double *w, const double *rowscale, double *g, void *stream)
{
    dcd_status s = component_check(A, k, prec, true);
    if (s != DCD_OK) return s;
    if (A->fmt != DCD_DENSE || !P || !g) return DCD_EINVAL;
    if ((s = validate_dense(P)) != DCD_OK) return s;
    if (P->fmt != DCD_DENSE || P->n != A->n) return DCD_EINVAL;
    if (row_id0 < 0 || row_id0 + A->m > (int64_t)INT32_MAX) return DCD_EINVAL;
    if (A->dtype == DCD_FP8E4M3 || P->dtype == DCD_FP8E4M3 || prec == DCD_PREC_FP8) return DCD_EUNSUPPORTED;
    if (!w) return DCD_EINVAL;
    PointsArg pts;
    pts.P = P;
    pts.row_id0 = row_id0;
    pts.col_ids = col_ids;
    return component_block(A, k, prec, nullptr, A->m, nullptr, P->m, w, rowscale, g, nullptr, 0, (cudaStream_t)stream,
                           &pts);
}

// ------------------------------------------------------------- batched --
namespace dcd {
namespace {

struct StreamSet {
    std::vector<cudaStream_t> s;
    std::vector<cudaEvent_t> ev;
    cudaEvent_t fork = nullptr;
    ~StreamSet()
    {
        for (auto x : s) cudaStreamDestroy(x);
        for (auto e : ev) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
    }
    cudaError_t create(int n)
    {
        s.resize(n, nullptr);
        ev.resize(n, nullptr);
        for (int i = 0; i < n; ++i) {
            cudaError_t e = cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking);
            if (e != cudaSuccess) return e;
            e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
        return cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    }
};

struct DevBuf {
    void *p = nullptr;
    cudaStream_t st = nullptr;
    ~DevBuf()
    {
        if (p) cudaFreeAsync(p, st);
    }
};

// Device time per block update of s-step BDCD with this s (a few outer
// steps after a warm-up one; alpha starts at 0 in scratch arrays).
dcd_status time_per_update(const dcd_matrix *A, const double *y, const dcd_kernel *k, double lambda, int b, int s,
                           int prec, double *alpha, double *grad, cudaStream_t st, double &ms_per)
{
    const int warm = 2, timed = 3;  // warm-up: one direct step and the step that is captured
    NoLookahead nla;  // timed as the batched driver runs it
    dcd_opts o{};
    o.s = s;
    o.b = b;
    o.max_iters = (int64_t)(warm + timed) * s;
    o.prec = prec;
    DCD_TRY(cudaMemsetAsync(alpha, 0, sizeof(double) * A->m, st));
    Solver sv;
    dcd_status r = init_krr(sv, A, k, lambda, &o, st);
    if (r == DCD_OK) r = prepare(sv, y, alpha, grad);
    if (r != DCD_OK) return r;
    dcd_stats a{}, c{};
    if ((r = sv.run_steps(warm, &a)) != DCD_OK) return r;
    if ((r = sv.run_steps(timed, &c)) != DCD_OK) return r;
    ms_per = (c.ms_total - a.ms_total) / ((double)timed * s);
    return DCD_OK;
}

}  // namespace
}  // namespace dcd

namespace dcd {
namespace {
// The autotuner over s = 1, 2, 4, ... while s*b <= max_sb.
dcd_status autotune_s(const dcd_matrix *A, const double *y, const dcd_kernel *k, double lambda, int32_t b,
                      int32_t prec, int32_t *s_out, void *stream, int64_t max_sb)
{
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf buf;
    buf.st = st;
    DCD_TRY(malloc_async(&buf.p, 2 * sizeof(double) * A->m, st));
    double *alpha = (double *)buf.p, *grad = alpha + A->m;
    double best = 1e300;
    int best_s = 1;
    for (int s = 1; s <= 128 && (int64_t)s * b <= max_sb; s *= 2) {
        double ms = 0.0;
        const dcd_status r = time_per_update(A, y, k, lambda, b, s, prec, alpha, grad, st, ms);
        if (r != DCD_OK) return r;
        if (ms < best * 0.98) {  // a larger s must win by more than the timing noise
            best = ms;
            best_s = s;
        }
    }
    *s_out = best_s;
    return DCD_OK;
}
}  // namespace
}  // namespace dcd

extern "C" dcd_status dcd_krr_autotune_s(const dcd_matrix *A, const double *y, const dcd_kernel *k, double lambda,
                                         int32_t b, int32_t prec, int32_t *s_out, void *stream)
{
    using namespace dcd;
    if (!A || !y || !k || !s_out || b < 1 || b > B_MAX || b > A->m) return DCD_EINVAL;
    return autotune_s(A, y, k, lambda, b, prec, s_out, stream, SB_MAX);
}

extern "C" dcd_status bdcd_krr_solve_batched(const dcd_krr_problem *probs, int32_t count, const dcd_batch_opts *bo,
                                             dcd_stats *st_out, void *stream)
{
    using namespace dcd;
    if (!probs || !bo || count < 0) return DCD_EINVAL;
    if (count == 0) return DCD_OK;
    if (!(std::isfinite(bo->tol) && bo->tol >= 0.0) || bo->check_every < 0 || bo->streams < 0 ||
        bo->rounds_per_graph < 0)
        return DCD_EINVAL;
    cudaStream_t main = (cudaStream_t)stream;
    const int nstreams = bo->streams > 0 ? std::min(bo->streams, 64) : 16;
    const int R = bo->rounds_per_graph > 0 ? bo->rounds_per_graph : 8;
    StreamSet ss;
    DCD_TRY(ss.create(nstreams));

    // s per problem: given, or the autotuner's per (m bucket, b)
    std::vector<int> s_of(count);
    std::map<std::pair<int, int>, int> tuned;
    for (int i = 0; i < count; ++i) {
        if (probs[i].s > 0) {
            s_of[i] = probs[i].s;
            continue;
        }
        int bucket = 0;
        while ((2LL << bucket) <= probs[i].A.m) ++bucket;
        const auto key = std::make_pair(bucket, (int)probs[i].b);
        auto it = tuned.find(key);
        if (it == tuned.end()) {
            // beside other problems the blocked recurrence of shapes above one cluster (s*b > 1024
            // rows) packs worse than it runs alone (measured on the sweep: 27.7 against 31.8 M
            // coordinate updates/s), so the candidates stop at the largest single-cluster shape
            int64_t max_sb = SB_MAX;
            for (int s = 128; s >= 1; s /= 2)
                if (recur_cluster_size(s, (int)probs[i].b, 2) > 0) {
                    max_sb = (int64_t)s * probs[i].b;
                    break;
                }
            int32_t s = 1;
            const dcd_status r = (probs[i].b < 1 || probs[i].b > B_MAX || probs[i].b > probs[i].A.m)
                                     ? DCD_EINVAL
                                     : autotune_s(&probs[i].A, probs[i].y, &probs[i].k, probs[i].lambda, probs[i].b,
                                                  bo->prec, &s, ss.s[0], max_sb);
            if (r != DCD_OK) return r;
            it = tuned.emplace(key, s).first;
        }
        s_of[i] = it->second;
    }

    // one plan per problem, round-robin over the worker streams
    NoLookahead nla;  // the batch graph captures rounds of many plans' steps
    std::vector<std::unique_ptr<dcd_plan>> plans(count);
    for (int i = 0; i < count; ++i) {
        dcd_opts o{};
        o.s = s_of[i];
        o.b = probs[i].b;
        o.max_iters = probs[i].max_iters;
        o.seed = probs[i].seed;
        o.tol = bo->tol;
        o.prec = bo->prec;
        o.flags = bo->flags & (DCD_FLAG_REFRESH | DCD_FLAG_NO_GRAPH);
        dcd_plan *p = nullptr;
        const dcd_status r = bdcd_krr_plan_create(&probs[i].A, probs[i].y, &probs[i].k, probs[i].lambda, &o,
                                                  probs[i].alpha, probs[i].grad, ss.s[i % nstreams], &p);
        if (r != DCD_OK) return r;
        plans[i].reset(p);
    }
    // a first direct step per problem sets every kernel attribute and cached
    // launch shape before any capture
    std::vector<char> active(count, 1);
    EventTimer off;
    off.init(false, nullptr);
    for (int i = 0; i < count; ++i) {
        Solver &sv = plans[i]->sv;
        dcd_status r = sv.begin();
        if (r != DCD_OK) return r;
        if (sv.finished()) {
            active[i] = 0;
            continue;
        }
        const int64_t cnt = std::min<int64_t>(sv.o.s, sv.o.max_iters - sv.done);
        if ((r = sv.enqueue_step(cnt, off)) != DCD_OK) return r;
        sv.done += cnt;
        ++sv.steps;
    }
    for (auto x : ss.s) DCD_TRY(cudaStreamSynchronize(x));

    // pinned buffer for the batched convergence checks
    double *hres = nullptr;
    DCD_TRY(cudaMallocHost(&hres, sizeof(double) * 4 * count));
    struct HostFree {
        double *p;
        ~HostFree() { cudaFreeHost(p); }
    } hf{hres};

    cudaGraphExec_t gexec = nullptr;
    struct GraphFree {
        cudaGraphExec_t *g;
        ~GraphFree()
        {
            if (*g) cudaGraphExecDestroy(*g);
        }
    } gf{&gexec};
    std::vector<int> rounds_in_graph(count, 0);
    bool dirty = true;
    const bool use_graph = !(bo->flags & DCD_FLAG_NO_GRAPH) && main != nullptr && main != cudaStreamLegacy &&
                           main != cudaStreamPerThread;
    int64_t replays = 0;
    for (;;) {
        // full outer steps each active problem can take in this replay
        bool any = false;
        for (int i = 0; i < count; ++i) {
            if (!active[i]) continue;
            Solver &sv = plans[i]->sv;
            const int64_t full = (sv.o.max_iters - sv.done) / sv.o.s;
            const int r = (int)std::min<int64_t>(R, full);
            if (r != rounds_in_graph[i]) dirty = true;
            rounds_in_graph[i] = r;
            any = any || r > 0;
        }
        if (!any) break;
        if (use_graph) {
            if (dirty) {
                if (gexec) {
                    cudaGraphExecDestroy(gexec);
                    gexec = nullptr;
                }
                DCD_TRY(cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal));
                cudaError_t ce = cudaEventRecord(ss.fork, main);
                for (int k = 0; k < nstreams && ce == cudaSuccess; ++k) ce = cudaStreamWaitEvent(ss.s[k], ss.fork, 0);
                dcd_status r = ce == cudaSuccess ? DCD_OK : DCD_ECUDA;
                for (int rr = 0; rr < R && r == DCD_OK; ++rr)
                    for (int i = 0; i < count && r == DCD_OK; ++i)
                        if (active[i] && rr < rounds_in_graph[i]) r = plans[i]->sv.enqueue_step(plans[i]->sv.o.s, off);
                for (int k = 0; k < nstreams && ce == cudaSuccess; ++k) {
                    ce = cudaEventRecord(ss.ev[k], ss.s[k]);
                    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(main, ss.ev[k], 0);
                }
                cudaGraph_t graph = nullptr;
                const cudaError_t ee = cudaStreamEndCapture(main, &graph);
                const bool ok = r == DCD_OK && ce == cudaSuccess && ee == cudaSuccess && graph &&
                                cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess;
                if (graph) cudaGraphDestroy(graph);
                if (!ok) {
                    cudaGetLastError();
                    return r != DCD_OK ? r : DCD_ECUDA;
                }
                dirty = false;
            }
            DCD_TRY(cudaGraphLaunch(gexec, main));
        } else {
            for (int rr = 0; rr < R; ++rr)
                for (int i = 0; i < count; ++i)
                    if (active[i] && rr < rounds_in_graph[i]) {
                        const dcd_status r = plans[i]->sv.enqueue_step(plans[i]->sv.o.s, off);
                        if (r != DCD_OK) return r;
                    }
        }
        for (int i = 0; i < count; ++i)
            if (active[i]) {
                plans[i]->sv.done += (int64_t)rounds_in_graph[i] * plans[i]->sv.o.s;
                plans[i]->sv.steps += rounds_in_graph[i];
            }
        ++replays;
        // convergence of every active problem, one synchronisation
        if (bo->tol > 0 && bo->check_every > 0 && replays % bo->check_every == 0) {
            if (use_graph) DCD_TRY(cudaStreamSynchronize(main));
            for (int i = 0; i < count; ++i)
                if (active[i]) DCD_TRY(plans[i]->sv.measure_enqueue(hres + 4 * i));
            for (auto x : ss.s) DCD_TRY(cudaStreamSynchronize(x));
            for (int i = 0; i < count; ++i) {
                if (!active[i]) continue;
                Solver &sv = plans[i]->sv;
                sv.measure_finish(hres + 4 * i, sv.metric, sv.primal, sv.dual, sv.ynorm2);
                if (sv.metric <= bo->tol) {
                    // confirmed (on a recomputed gradient with DCD_FLAG_REFRESH) by the solver's own test
                    const dcd_status r = sv.check_converged();
                    if (r != DCD_OK) return r;
                    if (sv.conv) {
                        active[i] = 0;
                        dirty = true;
                    }
                }
            }
        }
    }
    if (use_graph) DCD_TRY(cudaStreamSynchronize(main));
    // the last, shorter outer steps, then each problem's final measure, publish and statistics
    dcd_status first_err = DCD_OK;
    for (int i = 0; i < count; ++i) {
        dcd_stats st{};
        const dcd_status r = dcd_plan_run(plans[i].get(), -1, &st);
        if (st_out) st_out[i] = st;
        if (r != DCD_OK && r != DCD_ENOTCONV && first_err == DCD_OK) first_err = r;
        if (r == DCD_ENOTCONV && first_err == DCD_OK) first_err = r;
    }
    for (auto x : ss.s) DCD_TRY(cudaStreamSynchronize(x));
    return first_err;
}
