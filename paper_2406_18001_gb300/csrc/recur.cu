// recur.cu -- the FP64 s-step inner recurrence.
//
// The sampled Gram Kss[t][j] = K(a_{S_t}, a_{S_j}) is computed beforehand by
// the same block kernel that later applies the whole m x sb block, and the
// cached gradient g supplies U_j^T alpha_sk (g_S = V^T (Q alpha - 1 + omega
// alpha) for K-SVM, V^T((K/lambda + mI) alpha - y) for K-RR), so only the
// unrolled correction sums of Sections 3.2 and 3.4 remain:
//   DCD  (Algorithm 2): g_j = g_S[j] + sum_{t<j} Q(i_t,i_j) theta_t + omega sum_{t<j, i_t=i_j} theta_t
//                       rho_j = alpha_S[j] + sum_{t<j, i_t=i_j} theta_t
//                       theta_j = clip(rho_j - g_j/eta_j, 0, nu) - rho_j  (0 if the projected gradient is 0)
//   BDCD (eq. bdcd-sstep): G_jj Delta_j = -g_S[j] - sum_{t<j} G_jt Delta_t,
//                       G_jt = Kss_jt / lambda + m [S_j = S_t]   (Algorithm 4)
// All arithmetic here is FP64.
#include "dcd_internal.cuh"

namespace dcd {

namespace {

template <typename KT>
__device__ __forceinline__ double kval(const KT *K, int64_t ld, int64_t r, int64_t c)
{
    return (double)K[r * ld + c];
}

// ------------------------------------------------------------------ DCD ---
// One CTA.  All threads stage the sampled data (and, when it fits, the Gram
// transposed so that column j is a contiguous smem row); warp 0 then runs the
// sequential chain, each lane owning the future coordinates t = lane mod 32
// and folding every new theta_j into their pending corrections.
constexpr int DCD_THREADS = 256;
constexpr int DCD_SMEM_GRAM_MAX = 128;   // cnt <= 128: Gram staged in shared memory

template <typename KT>
__global__ void __launch_bounds__(DCD_THREADS) recur_dcd_kernel(const KT *Kss, int64_t ldk, const int32_t *S,
                                                                int cnt, const double *y, const double *alpha,
                                                                const double *g, double omega, double nu,
                                                                double *delta, double *w64, float *w32, int *err)
{
    extern __shared__ double sm[];
    double *corr = sm;               // pending gradient corrections
    double *rcorr = corr + cnt;      // pending corrections of rho
    double *gS = rcorr + cnt;
    double *aS = gS + cnt;
    double *yS = aS + cnt;
    double *ieta = yS + cnt;         // 1 / eta_j (0 marks eta <= 0)
    double *theta = ieta + cnt;
    int32_t *sI = (int32_t *)(theta + cnt);
    double *KT_s = (double *)(sI + ((cnt + 1) & ~1));  // cnt x cnt, KT_s[j*cnt + t] = Kss[t][j]
    const bool staged = cnt <= DCD_SMEM_GRAM_MAX;

    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        int32_t i = S[t];
        sI[t] = i;
        gS[t] = g[i];
        aS[t] = alpha[i];
        yS[t] = y[i];
        corr[t] = 0.0;
        rcorr[t] = 0.0;
        double eta = kval(Kss, ldk, t, t) + omega;  // G_k = V^T U_k + omega I, y_t^2 = 1
        ieta[t] = eta > 0.0 ? 1.0 / eta : 0.0;
    }
    if (staged)
        for (int e = threadIdx.x; e < cnt * cnt; e += blockDim.x) {
            int t = e / cnt, j = e % cnt;
            KT_s[j * cnt + t] = kval(Kss, ldk, t, j);
        }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    for (int j = 0; j < cnt; ++j) {
        double th = 0.0;
        if (lane == (j & 31)) {
            double rho = aS[j] + rcorr[j];
            double gj = gS[j] + corr[j];
            double gt = fabs(fmin(fmax(rho - gj, 0.0), nu) - rho);
            if (gt != 0.0 && ieta[j] != 0.0) th = fmin(fmax(rho - gj * ieta[j], 0.0), nu) - rho;
            theta[j] = th;
        }
        th = __shfl_sync(0xffffffffu, th, j & 31);
        if (th != 0.0) {
            const int32_t ij = sI[j];
            const double yj = yS[j];
            for (int t = j + 1 + ((lane - (j + 1)) & 31); t < cnt; t += 32) {
                double kt = staged ? KT_s[j * cnt + t] : kval(Kss, ldk, t, j);
                double c = yS[t] * yj * kt * th;
                if (sI[t] == ij) {
                    c += omega * th;
                    rcorr[t] += th;
                }
                corr[t] += c;
            }
        }
        __syncwarp();
    }
    for (int t = lane; t < cnt; t += 32) {
        double th = theta[t];
        delta[t] = th;
        double wv = yS[t] * th;
        if (w64) w64[t] = wv;
        if (w32) w32[t] = (float)wv;
    }
}

// ----------------------------------------------------------------- BDCD ---
// (1) factor: one CTA per diagonal block G_jj = Kss_jj/lambda + m I; writes
//     the Cholesky factor L_j (row-major b x b, lower) and 1/L_j[p][p].
// (2) forward: one CTA runs j = 0..nblk-1: solve L L^T Delta_j = r_j with one
//     warp, then every thread subtracts G_tj Delta_j from the right-hand
//     sides r_t of the later blocks t > j.
constexpr int FAC_THREADS = 128;

template <typename KT>
__global__ void __launch_bounds__(FAC_THREADS) bdcd_factor_kernel(const KT *Kss, int64_t ldk, int b, double lambda,
                                                                  double mdiag, double *Lbuf, int *err)
{
    extern __shared__ double G[];  // b x b
    const int j = blockIdx.x;
    const int64_t o = (int64_t)j * b;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        int p = e / b, q = e % b;
        G[e] = kval(Kss, ldk, o + p, o + q) / lambda + (p == q ? mdiag : 0.0);
    }
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < b; ++k) {
        if (threadIdx.x == 0) {
            double d = G[k * b + k];
            if (!(d > 0.0)) {
                bad = 1;
                d = 1.0;
            }
            G[k * b + k] = sqrt(d);
        }
        __syncthreads();
        const double dk = G[k * b + k];
        for (int p = k + 1 + threadIdx.x; p < b; p += blockDim.x) G[p * b + k] /= dk;
        __syncthreads();
        const int rem = b - k - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            int p = k + 1 + e / rem, q = k + 1 + e % rem;
            if (q <= p) G[p * b + q] -= G[p * b + k] * G[q * b + k];
        }
        __syncthreads();
    }
    double *L = Lbuf + (int64_t)j * b * (b + 1);
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        int p = e / b, q = e % b;
        L[e] = (q <= p) ? G[e] : 0.0;
    }
    for (int p = threadIdx.x; p < b; p += blockDim.x) L[b * b + p] = 1.0 / G[p * b + p];
    if (threadIdx.x == 0 && bad) set_error(err, DEV_NOT_SPD);
}

constexpr int FWD_THREADS = 256;

template <typename KT>
__global__ void __launch_bounds__(FWD_THREADS) bdcd_forward_kernel(const KT *Kss, int64_t ldk, const int32_t *S,
                                                                   int nblk, int b, double lambda, double mdiag,
                                                                   const double *g, const double *Lbuf,
                                                                   double *delta, double *w64, float *w32)
{
    extern __shared__ double smd[];
    const int sb = nblk * b;
    double *r = smd;             // right-hand sides, then solutions
    double *z = r + sb;          // b scratch
    int32_t *sI = (int32_t *)(z + b);
    for (int p = threadIdx.x; p < sb; p += blockDim.x) {
        int32_t i = S[p];
        sI[p] = i;
        r[p] = -g[i];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = 0; j < nblk; ++j) {
        const int64_t o = (int64_t)j * b;
        const double *L = Lbuf + (int64_t)j * b * (b + 1);
        const double *Ld = L + b * b;
        if (warp == 0) {
            // forward: L z = r_j (column-oriented; lane p owns rows p mod 32)
            for (int p = lane; p < b; p += 32) z[p] = r[o + p];
            __syncwarp();
            for (int q = 0; q < b; ++q) {
                double zq = z[q] * Ld[q];
                __syncwarp();
                for (int p = q + 1 + lane; p < b; p += 32) z[p] -= L[p * b + q] * zq;
                if (lane == 0) z[q] = zq;
                __syncwarp();
            }
            // backward: L^T x = z
            for (int q = b - 1; q >= 0; --q) {
                double xq = z[q] * Ld[q];
                __syncwarp();
                for (int p = lane; p < q; p += 32) z[p] -= L[q * b + p] * xq;
                if (lane == 0) z[q] = xq;
                __syncwarp();
            }
            for (int p = lane; p < b; p += 32) r[o + p] = z[p];
        }
        __syncthreads();
        // r_t -= G_tj Delta_j for rows of later blocks
        for (int p = (int)o + b + threadIdx.x; p < sb; p += blockDim.x) {
            double acc = 0.0;
            const int32_t ip = sI[p];
            for (int q = 0; q < b; ++q) {
                double gq = kval(Kss, ldk, p, o + q) / lambda + (sI[o + q] == ip ? mdiag : 0.0);
                acc = fma(gq, r[o + q], acc);
            }
            r[p] -= acc;
        }
        __syncthreads();
    }
    for (int p = threadIdx.x; p < sb; p += blockDim.x) {
        double d = r[p];
        delta[p] = d;
        if (w64) w64[p] = d / lambda;
        if (w32) w32[p] = (float)(d / lambda);
    }
}

}  // namespace

cudaError_t launch_recur_dcd(const void *Kss, int kss_f64, int64_t ldk, const int32_t *S, int64_t cnt,
                             const double *y, const double *alpha, const double *g, double omega, double nu,
                             double *delta, double *w64, float *w32, int *err, cudaStream_t st)
{
    if (cnt <= 0) return cudaSuccess;
    size_t sm = sizeof(double) * 7 * cnt + sizeof(int32_t) * ((cnt + 1) & ~1);
    if (cnt <= DCD_SMEM_GRAM_MAX) sm += sizeof(double) * cnt * cnt;
    cudaError_t e;
    if (kss_f64) {
        e = cudaFuncSetAttribute(recur_dcd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        recur_dcd_kernel<double><<<1, DCD_THREADS, sm, st>>>((const double *)Kss, ldk, S, (int)cnt, y, alpha, g,
                                                             omega, nu, delta, w64, w32, err);
    } else {
        e = cudaFuncSetAttribute(recur_dcd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        recur_dcd_kernel<float><<<1, DCD_THREADS, sm, st>>>((const float *)Kss, ldk, S, (int)cnt, y, alpha, g, omega,
                                                            nu, delta, w64, w32, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_recur_bdcd(const void *Kss, int kss_f64, int64_t ldk, const int32_t *S, int64_t nblk, int b,
                              double lambda, double mdiag, const double *g, double *Lbuf, double *delta, double *w64,
                              float *w32, int *err, cudaStream_t st)
{
    if (nblk <= 0) return cudaSuccess;
    size_t smf = sizeof(double) * (size_t)b * b;
    size_t smw = sizeof(double) * ((size_t)nblk * b + b) + sizeof(int32_t) * (size_t)nblk * b;
    cudaError_t e;
    if (kss_f64) {
        e = cudaFuncSetAttribute(bdcd_factor_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(bdcd_forward_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
        if (e != cudaSuccess) return e;
        bdcd_factor_kernel<double><<<(unsigned)nblk, FAC_THREADS, smf, st>>>((const double *)Kss, ldk, b, lambda,
                                                                             mdiag, Lbuf, err);
        bdcd_forward_kernel<double><<<1, FWD_THREADS, smw, st>>>((const double *)Kss, ldk, S, (int)nblk, b, lambda,
                                                                 mdiag, g, Lbuf, delta, w64, w32);
    } else {
        e = cudaFuncSetAttribute(bdcd_factor_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(bdcd_forward_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
        if (e != cudaSuccess) return e;
        bdcd_factor_kernel<float><<<(unsigned)nblk, FAC_THREADS, smf, st>>>((const float *)Kss, ldk, b, lambda, mdiag,
                                                                            Lbuf, err);
        bdcd_forward_kernel<float><<<1, FWD_THREADS, smw, st>>>((const float *)Kss, ldk, S, (int)nblk, b, lambda,
                                                                mdiag, g, Lbuf, delta, w64, w32);
    }
    return cudaGetLastError();
}

}  // namespace dcd
