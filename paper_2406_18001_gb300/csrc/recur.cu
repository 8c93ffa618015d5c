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
#include "ptx.cuh"

#include <algorithm>

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
constexpr size_t DCD_SMEM_LIMIT = 224 * 1024;

// Refinement state of one FP64-form outer step (the last 256 bytes of the
// recurrence scratch).  The FP64 form does not fix its number of refinement
// rounds: after each round the chain kernel compares the size of the
// correction it added with the size of Delta and with the previous round's
// correction, and decides on the device whether to
//   stop      (the correction is below 2^-44 |Delta|: the error left is that
//              times the contraction factor),
//   go on     (the correction shrank by more than 10x: one more round), or
//   fall back (no contraction, or REFINE_MAX rounds without reaching the
//              stop test while the correction is still above 1e-10 |Delta|:
//              cond(L) * 2^-24 is too close to 1 for the FP32 chain), in which
//              case the FP64 factor / forward kernels solve the step instead.
// Kernels of rounds after the stop, and the fallback kernels when there is
// no fallback, return at once (they stay in the launch sequence, so a
// captured step graph is the same for every step).
struct RefineState {
    int done;        // no further refinement round runs
    int fallback;    // the FP64 factor / forward kernels run
    int inv_bad;     // the FP32 inverse met a non-positive pivot (reset by round 0)
    int rounds;      // refinement rounds run (statistics)
    double prev_corr;
};
constexpr int REFINE_MAX = 4;
constexpr size_t REFINE_STATE_BYTES = 256;

// max that keeps a NaN (fmax drops it), so a non-finite round takes the fallback
__device__ __forceinline__ double nanmax(double a, double b) { return (a != a || b != b) ? a + b : fmax(a, b); }


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
                                                                  double mdiag, double *Lbuf, int *err,
                                                                  const RefineState *rs = nullptr)
{
    if (rs && !*(volatile const int *)&rs->fallback) return;  // the refined chain solved this step
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
                                                                   double *delta, double *w64, float *w32,
                                                                   const RefineState *rs = nullptr)
{
    if (rs && !*(volatile const int *)&rs->fallback) return;  // the refined chain solved this step
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

// ------------------------------------------- BDCD, refined FP32 chain ---
// On GB300 an FP64 FMA has a 64-cycle dependent latency and 1/64 of the FP32
// rate, so the sequential block forward substitution is run in FP32 and made
// FP64-accurate by iterative refinement with FP64 residuals:
//   round 0:  Delta = L32^-1 rhs,                    rhs = -g_S
//   round k:  rho   = rhs - L Delta      (FP64, all rows in parallel)
//             Delta += L32^-1 rho
// L is the block lower triangle of G (G_jt = Kss_jt/lambda + m [S_j = S_t]),
// L32 its FP32 rounding.  Each round multiplies the error by about
// cond(L) * 2^-24, so one refinement reaches ~1e-13 and two reach FP64
// rounding for the well-conditioned blocks of K-RR (G_jj >= m I).

// W_j = G_jj^-1 in FP32 for every diagonal block, one warp per block,
// Gauss-Jordan with lane p holding row p of [G_jj | I]; only the columns that
// can still change at pivot k are touched (left half k.., right half ..k).
template <typename KT, int BT>
__global__ void __launch_bounds__(128) bdcd_inverse_kernel(const KT *Kss, int64_t ldk, int nblk, int b, float inv_lam,
                                                           float mf, float *W32, int *err, RefineState *rs)
{
    const int j = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= nblk) return;
    const int jb = j * b;
    float aug[2 * BT];
#pragma unroll
    for (int q = 0; q < BT; ++q) {
        float gv = 0.f;
        if (lane < b && q < b) gv = (float)Kss[(int64_t)(jb + q) * ldk + jb + lane] * inv_lam + (q == lane ? mf : 0.f);
        aug[q] = gv;
        aug[BT + q] = (q == lane) ? 1.f : 0.f;
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < BT; ++k) {
        if (k < b) {
            float piv = __shfl_sync(0xffffffffu, aug[k], k);
            if (!(piv > 0.f)) {
                bad = true;
                piv = 1.f;
            }
            const float ip = 1.f / piv;
            if (lane == k) {
#pragma unroll
                for (int q = k; q < BT + k + 1; ++q) aug[q] *= ip;
            }
            const float f = (lane == k) ? 0.f : aug[k];
#pragma unroll
            for (int q = k; q < BT + k + 1; ++q) {
                const float rk = __shfl_sync(0xffffffffu, aug[q], k);
                aug[q] = fmaf(-f, rk, aug[q]);
            }
        }
    }
    // with a refinement state the FP64 factorisation decides (the FP32 pivots may fail first)
    if (bad && lane == 0) {
        if (rs) atomicExch(&rs->inv_bad, 1);
        else set_error(err, DEV_NOT_SPD);
    }
    if (lane < b)
#pragma unroll
        for (int q = 0; q < BT; ++q)
            if (q < b) W32[((int64_t)jb + lane) * b + q] = aug[BT + q];
}

// One CTA walks the blocks: the warp owning block t forms delta_t = W_t r_t
// (W_t from shared memory), and all threads subtract G_pt delta_t from the
// right-hand sides r_p of the later rows p, one row per thread.  The Gram
// entries G_{p,tb+q} are read as Kss[tb+q][p] -- the kernel matrix is
// symmetric (up to the last FP32 bit in the tensor-core modes, which the FP64
// residual absorbs) -- so consecutive threads read consecutive addresses; with
// fp32 storage the b rows of step t+1 are streamed into shared memory by bulk
// copies while step t computes.  The m [S_p = S_q] terms follow a per-row
// chain of earlier occurrences of the same index, built once with a
// shared-memory hash table (repeated indices are rare).
constexpr size_t CHAIN_SMEM_MAX = 224 * 1024;  // dynamic shared memory of the chain kernel
constexpr int NBUF = 3;                        // streamed Gram panels in flight

struct ChainLayout {
    size_t pan_off, bar_off, total;
    bool tma;
};

__host__ __device__ inline ChainLayout chain_layout(int sb, int b, int kss_bytes, int64_t ldk)
{
    ChainLayout L;
    size_t cur = (size_t)sb * 20;  // r32, d32, dl32 (fp32) and sI, prev (int32)
    cur = (cur + 15) & ~(size_t)15;
    L.pan_off = cur;
    size_t T = 2;
    while (T < 2 * (size_t)sb) T <<= 1;
    const size_t hash_bytes = 8 * T;  // keys + counts, T entries each
    const size_t with_tma = cur + NBUF * (size_t)b * sb * 4 + 8 * NBUF;
    L.tma = kss_bytes == 4 && b % 4 == 0 && ldk % 4 == 0 && sb > b && with_tma <= CHAIN_SMEM_MAX &&
            (size_t)b * sb * 4 >= hash_bytes;
    if (L.tma) {
        L.bar_off = cur + NBUF * (size_t)b * sb * 4;
        L.total = with_tma;
    } else {
        L.bar_off = 0;
        L.total = cur + hash_bytes;  // hash table lives where the panels would be
    }
    return L;
}

template <typename KT, int BT, int NT>
__global__ void __launch_bounds__(NT) bdcd_chain_kernel(const KT *Kss, int64_t ldk, const int32_t *S, int nblk, int b,
                                                        double lambda, double mdiag, const double *g,
                                                        const double *rho, const float *W32, double *rhs64,
                                                        double *delta, int round, int final_round, double *w64,
                                                        float *w32, int *err, RefineState *rs)
{
    extern __shared__ __align__(16) unsigned char csm_raw[];
    if (rs && round > 0 && *(volatile int *)&rs->done) return;  // refinement already stopped
    const int sb = nblk * b;
    const ChainLayout L = chain_layout(sb, b, (int)sizeof(KT), ldk);
    float *r32 = (float *)csm_raw;
    float *d32 = r32 + sb;
    float *dl32 = d32 + sb;   // delta / lambda
    int32_t *sI = (int32_t *)(dl32 + sb);
    int32_t *prev = sI + sb;  // previous position with the same index, or -1
    float *panels = (float *)(csm_raw + L.pan_off);  // NBUF x (b rows x sb)
    uint64_t *pbar = (uint64_t *)(csm_raw + L.bar_off);
    __shared__ int abort_chain;
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float inv_lam = (float)(1.0 / lambda);
    const float mf = (float)mdiag;

    // hash table for the repeated-index chains (in the last panel's space)
    int T = 2;
    while (T < 2 * sb) T <<= 1;
    int32_t *hkey = (int32_t *)(panels + (L.tma ? (size_t)(NBUF - 1) * b * sb : 0));
    int32_t *hcnt = hkey + T;
    for (int e = tid; e < T; e += NT) {
        hkey[e] = -1;
        hcnt[e] = 0;
    }
    for (int p = tid; p < sb; p += NT) {
        const int32_t i = S[p];
        sI[p] = i;
        double rhs;
        if (round == 0) {
            rhs = -g[i];
            rhs64[p] = rhs;
        } else {
            rhs = rho[p];
        }
        r32[p] = (float)rhs;
    }
    if (tid == 0) abort_chain = 0;
    __syncthreads();
    for (int p = tid; p < sb; p += NT) {
        const int32_t key = sI[p];
        int h = (int)(((uint32_t)key * 2654435761u) & (uint32_t)(T - 1));
        for (int probe = 0; probe < T; ++probe) {
            const int32_t old = atomicCAS(&hkey[h], -1, key);
            if (old == -1 || old == key) break;
            h = (h + 1) & (T - 1);
        }
        prev[p] = h;
        atomicAdd(&hcnt[h], 1);
    }
    __syncthreads();
    for (int p = tid; p < sb; p += NT) {
        int pv = -1;
        if (hcnt[prev[p]] > 1) {
            const int32_t key = sI[p];
            for (int q = p - 1; q >= 0; --q)
                if (sI[q] == key) {
                    pv = q;
                    break;
                }
        }
        prev[p] = pv;
    }
    if (L.tma && tid == 0) {
        for (int k = 0; k < NBUF; ++k) ptx::mbar_init(&pbar[k], 1);
        ptx::mbar_init_fence();
    }
    __syncthreads();

    // Panel of step t (rows tb..tb+b-1 of Kss from column (t+1)b on) into
    // buffer t % NBUF; warp 0 issues it, one row per lane.
    int issued_upto = -1;  // warp 0: last step whose panel was issued
    auto issue = [&](int t) {
        const int ps = (t + 1) * b;
        if (ps >= sb) return;
        issued_upto = t;
        const int k = t % NBUF;
        float *pan = panels + (size_t)k * b * sb;
        const uint32_t row_bytes = (uint32_t)(sb - ps) * 4u;
        if (lane == 0) ptx::mbar_expect_tx(&pbar[k], row_bytes * (uint32_t)b);
        __syncwarp();
        for (int q = lane; q < b; q += 32)
            ptx::bulk_g2s(pan + (size_t)q * sb + ps, (const float *)Kss + ((int64_t)t * b + q) * ldk + ps, row_bytes,
                          &pbar[k]);
    };
    if (L.tma && warp == 0)
        for (int t = 0; t < NBUF - 1 && t < nblk; ++t) issue(t);

    // owner warp: inverse row of its next block (lane p: row p of W_t)
    float wrow[BT];
    auto load_w = [&](int t) {
#pragma unroll
        for (int q = 0; q < BT; ++q) wrow[q] = (lane < b && q < b) ? W32[((int64_t)t * b + lane) * b + q] : 0.f;
    };
    if (warp < nblk) load_w(warp);

    for (int t = 0; t < nblk; ++t) {
        const int tb = t * b;
        if (L.tma && warp == 0 && t + NBUF - 1 < nblk) issue(t + NBUF - 1);
        if (warp == t % NW) {
            if (lane < b) {
                float a0 = 0.f, a1 = 0.f;
#pragma unroll
                for (int q = 0; q < BT; q += 2) {
                    if (q < b) a0 = fmaf(wrow[q], r32[tb + q], a0);
                    if (q + 1 < b) a1 = fmaf(wrow[q + 1], r32[tb + q + 1], a1);
                }
                const float d = a0 + a1;
                d32[tb + lane] = d;
                dl32[tb + lane] = d * inv_lam;
            }
            if (t + NW < nblk) load_w(t + NW);
        }
        const bool has_rows = (t + 1) * b < sb;
        if (L.tma && has_rows &&
            !ptx::mbar_wait_bounded(&pbar[t % NBUF], (uint32_t)((t / NBUF) & 1), 2000000000ull))
            abort_chain = 1;
        __syncthreads();
        if (abort_chain) break;
        if (has_rows) {
            const float *pan = panels + (size_t)(t % NBUF) * b * sb;
            for (int p = (t + 1) * b + tid; p < sb; p += NT) {
                float s0 = 0.f, s1 = 0.f;
                if (L.tma) {
#pragma unroll
                    for (int q = 0; q < BT; q += 2) {
                        if (q < b) s0 = fmaf(pan[(size_t)q * sb + p], dl32[tb + q], s0);
                        if (q + 1 < b) s1 = fmaf(pan[(size_t)(q + 1) * sb + p], dl32[tb + q + 1], s1);
                    }
                } else {
                    for (int q = 0; q < b; ++q) s0 = fmaf((float)Kss[((int64_t)tb + q) * ldk + p], dl32[tb + q], s0);
                }
                for (int q = prev[p]; q >= tb; q = prev[q])
                    if (q < tb + b) s1 = fmaf(mf, d32[q], s1);
                r32[p] -= s0 + s1;
            }
        }
        __syncthreads();
    }
    if (abort_chain) {
        if (tid == 0) {
            // Every panel issued but not consumed is still in flight: wait
            // (bounded) for the last phase armed on each buffer.
            set_error(err, DEV_TIMEOUT);
            for (int k = 0; k < NBUF; ++k) {
                int last = -1;  // the last issued step that used buffer k
                for (int t = k; t <= issued_upto; t += NBUF) last = t;
                if (last >= 0) ptx::mbar_wait_bounded(&pbar[k], (uint32_t)((last / NBUF) & 1), 2000000000ull);
            }
        }
        __syncthreads();
    }
    double cmax = 0.0, dmax = 0.0;  // this round's correction and the new Delta, max norms
    for (int p = tid; p < sb; p += NT) {
        const double c = (double)d32[p];
        double d = c;
        if (round > 0) d += delta[p];
        delta[p] = d;
        cmax = nanmax(cmax, fabs(c));
        dmax = nanmax(dmax, fabs(d));
        if (final_round || rs) {  // adaptive rounds: every round may be the last
            if (w64) w64[p] = d / lambda;
            if (w32) w32[p] = (float)(d / lambda);
        }
    }
    if (rs) {
        __shared__ double red[2][NT / 32];
        for (int o = 16; o > 0; o >>= 1) {
            cmax = nanmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
            dmax = nanmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        }
        if (lane == 0) {
            red[0][warp] = cmax;
            red[1][warp] = dmax;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < NT / 32; ++w) {
                cmax = nanmax(cmax, red[0][w]);
                dmax = nanmax(dmax, red[1][w]);
            }
            int done = 0, fb = 0;
            if (round == 0) {
                fb = rs->inv_bad;  // the FP32 inverse failed: the FP64 factorisation decides
                rs->inv_bad = 0;
                done = fb;
                rs->rounds = 0;
            } else {
                rs->rounds = round;
                const bool small = cmax <= 0x1p-44 * dmax;          // converged to FP64 working accuracy
                const bool floor = cmax <= 1e-10 * dmax;            // at a conditioning floor, still accurate
                const bool stalled = !(cmax <= 0.1 * rs->prev_corr);  // no contraction (or not finite)
                if (small) done = 1;
                else if (stalled || round >= REFINE_MAX) {
                    done = 1;
                    fb = floor ? 0 : 1;
                }
            }
            rs->prev_corr = cmax;
            rs->fallback = fb;
            __threadfence();
            *(volatile int *)&rs->done = done;
        }
    }
}

// rho = rhs - L Delta in FP64, one warp per row, rows of all blocks at once.
template <typename KT>
__global__ void __launch_bounds__(256) bdcd_residual_kernel(const KT *Kss, int64_t ldk, const int32_t *S, int nblk,
                                                            int b, double inv_lambda, double mdiag,
                                                            const double *rhs64, const double *delta, double *rho,
                                                            const RefineState *rs)
{
    if (rs && *(volatile const int *)&rs->done) return;  // refinement already stopped
    const int sb = nblk * b;
    const int p = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (p >= sb) return;
    const int end = (p / b + 1) * b;
    const int32_t ip = S[p];
    const KT *kr = Kss + (int64_t)p * ldk;
    // sum_q Kss_pq delta_q and sum_{q: S_q = S_p} delta_q kept apart, so each
    // term costs one conversion and one FP64 FMA; four accumulators hide the
    // 64-cycle FP64 latency
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, dm = 0.0;
    int q = lane;
    for (; q + 96 < end; q += 128) {
        const double d0 = delta[q], d1 = delta[q + 32], d2 = delta[q + 64], d3 = delta[q + 96];
        a0 = fma((double)kr[q], d0, a0);
        a1 = fma((double)kr[q + 32], d1, a1);
        a2 = fma((double)kr[q + 64], d2, a2);
        a3 = fma((double)kr[q + 96], d3, a3);
        if (S[q] == ip) dm += d0;
        if (S[q + 32] == ip) dm += d1;
        if (S[q + 64] == ip) dm += d2;
        if (S[q + 96] == ip) dm += d3;
    }
    for (; q < end; q += 32) {
        const double d0 = delta[q];
        a0 = fma((double)kr[q], d0, a0);
        if (S[q] == ip) dm += d0;
    }
    double acc = (a0 + a1) + (a2 + a3);
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        dm += __shfl_xor_sync(0xffffffffu, dm, o);
    }
    if (lane == 0) rho[p] = rhs64[p] - (acc * inv_lambda + mdiag * dm);
}

// Chains longer than one cluster launch takes: blocked forward substitution.
// The chain is cut into diagonal panels of pb blocks; each panel is solved by
// the cluster recurrence (with its own refinement rounds) from right-hand
// sides that already hold every earlier panel's contribution, and after each
// panel one launch moves its contribution into the right-hand sides of all
// later rows:
//   rhs_p (= -g[S_p] for the first panel) -= sum_{q in panel} Kss[p][q] delta_q / lambda
//                                            + mdiag * sum_{q in panel, S_q = S_p} delta_q
// One warp per later row, FP64 sums of the FP32 Gram entries times FP64 delta.
__global__ void bdcd_panel_update_kernel(const float *Kss, int64_t ldk, const int32_t *S, int r0, int rows, int sb,
                                         double inv_lambda, double mdiag, const double *g, const double *delta,
                                         double *rhs, int first)
{
    const int lane = threadIdx.x & 31;
    const int64_t p = r0 + rows + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (p >= sb) return;
    const float *kr = Kss + p * ldk + r0;
    const int32_t ip = S[p];
    // four independent FP64 chains per lane; the (rare) repeat term only when some lane matches
    double a[4] = {0.0, 0.0, 0.0, 0.0}, dm = 0.0;
    for (int q0 = 0; q0 < rows; q0 += 128) {  // warp-uniform bounds
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = q0 + 32 * u + lane;
            const bool in = q < rows;
            const double d = in ? delta[r0 + q] : 0.0;
            a[u] = fma(in ? (double)kr[q] : 0.0, d, a[u]);
            const bool hit = in && S[r0 + q] == ip;
            if (__any_sync(0xffffffffu, hit)) dm += hit ? d : 0.0;
        }
    }
    double acc = (a[0] + a[1]) + (a[2] + a[3]);
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        dm += __shfl_xor_sync(0xffffffffu, dm, o);
    }
    if (lane == 0) rhs[p] = (first ? -g[ip] : rhs[p]) - (acc * inv_lambda + mdiag * dm);
}

// scratch: the cluster scratch of one panel, then sb FP64 right-hand sides
size_t blocked_cluster_scratch_bytes(int64_t nblk, int b)
{
    if (b % 4 != 0 || b > 32) return 0;
    const int64_t q = b >= 32 ? 1 : 32 / b;
    const size_t cl = (recur_cluster_scratch_bytes(std::min<int64_t>(nblk, 32 * q), b) + 255) / 256 * 256;
    return cl + sizeof(double) * (size_t)nblk * b;
}

cudaError_t blocked_cluster(const float *Kss, int64_t ldk, const int32_t *S, int nblk, int b, int pb, double lambda,
                            double mdiag, const double *g, int rounds, char *scratch, double *delta, double *w64,
                            float *w32, int *err, cudaStream_t st)
{
    const int sb = nblk * b;
    const int64_t q = b >= 32 ? 1 : 32 / b;
    double *rhs = (double *)(scratch + (recur_cluster_scratch_bytes(std::min<int64_t>(nblk, 32 * q), b) + 255) / 256 * 256);
    for (int p0 = 0; p0 < nblk; p0 += pb) {
        const int nb = std::min(pb, nblk - p0), r0 = p0 * b, rows = nb * b;
        const int P = recur_cluster_size(nb, b, rounds);
        if (P <= 0) return cudaErrorInvalidValue;
        cudaError_t e = launch_recur_cluster(Kss + (int64_t)r0 * ldk + r0, ldk, S + r0, nb, b, P, lambda, mdiag,
                                             const_cast<double *>(g), rounds, scratch, delta + r0,
                                             w64 ? w64 + r0 : nullptr, w32 ? w32 + r0 : nullptr, nullptr, err, st,
                                             p0 ? rhs + r0 : nullptr);
        if (e != cudaSuccess) return e;
        if (r0 + rows < sb) {
            const int later = sb - r0 - rows;
            bdcd_panel_update_kernel<<<(unsigned)((later + 7) / 8), 256, 0, st>>>(
                Kss, ldk, S, r0, rows, sb, 1.0 / lambda, mdiag, g, delta, rhs, p0 == 0);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

template <typename KT, int BT, int NT>
cudaError_t refined_bdcd(const KT *Kss, int64_t ldk, const int32_t *S, int nblk, int b, double lambda, double mdiag,
                         const double *g, int refinements, char *scratch, double *delta, double *w64, float *w32,
                         FusedUpdate *upd, int *err, cudaStream_t st)
{
    const int sb = nblk * b;
    float *W32 = (float *)scratch;
    double *rhs64 = (double *)(scratch + (((size_t)sb * b * 4 + 255) / 256) * 256);
    double *rho = rhs64 + sb;
    const ChainLayout L = chain_layout(sb, b, (int)sizeof(KT), ldk);
    auto kfn = bdcd_chain_kernel<KT, BT, NT>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CHAIN_SMEM_MAX);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (sizeof(KT) == 4) {  // fp32 Gram: the cluster recurrence when it applies
        const int P = recur_cluster_size(nblk, b, refinements + 1);
        if (P > 0) {
            // the cluster kernel also applies the a6 update (alpha and g are the solver's, writable)
            const cudaError_t e =
                launch_recur_cluster((const float *)Kss, ldk, S, nblk, b, P, lambda, mdiag, const_cast<double *>(g),
                                     refinements + 1, scratch, delta, w64, w32, upd, err, st);
            if (e == cudaSuccess && upd) upd->done = true;
            return e;
        }
        const int pb = recur_cluster_panel_blocks(b, refinements + 1);
        if (pb > 0 && pb < nblk && blocked_cluster_scratch_bytes(nblk, b) <= recur_bdcd_scratch_bytes(nblk, b))
            return blocked_cluster((const float *)Kss, ldk, S, nblk, b, pb, lambda, mdiag, g, refinements + 1,
                                   scratch, delta, w64, w32, err, st);
    }
    if (L.total > CHAIN_SMEM_MAX) return cudaErrorInvalidValue;
    // FP64 Gram (the FP64 form): refinement rounds decided on the device, with the FP64
    // factor / forward kernels as the fallback (see RefineState); other forms: fixed rounds
    RefineState *rs = nullptr;
    size_t smf = 0, smw = 0;
    if (sizeof(KT) == 8) {
        smf = sizeof(double) * (size_t)b * b;
        smw = sizeof(double) * ((size_t)sb + b) + sizeof(int32_t) * (size_t)sb;
        if (smf <= DCD_SMEM_LIMIT && smw <= DCD_SMEM_LIMIT) {
            rs = (RefineState *)(scratch + recur_bdcd_scratch_bytes(nblk, b) - REFINE_STATE_BYTES);
            static bool fb_attr = false;
            if (!fb_attr) {
                for (auto fn : {(const void *)bdcd_factor_kernel<KT>, (const void *)bdcd_forward_kernel<KT>}) {
                    const cudaError_t e =
                        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DCD_SMEM_LIMIT);
                    if (e != cudaSuccess) return e;
                }
                fb_attr = true;
            }
        }
    }
    const int rounds = rs ? REFINE_MAX : refinements;
    bdcd_inverse_kernel<KT, BT><<<(unsigned)((nblk + 3) / 4), 128, 0, st>>>(Kss, ldk, nblk, b, (float)(1.0 / lambda),
                                                                            (float)mdiag, W32, err, rs);
    kfn<<<1, NT, L.total, st>>>(Kss, ldk, S, nblk, b, lambda, mdiag, g, nullptr, W32, rhs64, delta, 0,
                                rounds == 0, w64, w32, err, rs);
    for (int r = 1; r <= rounds; ++r) {
        bdcd_residual_kernel<KT><<<(unsigned)((sb + 7) / 8), 256, 0, st>>>(Kss, ldk, S, nblk, b, 1.0 / lambda, mdiag,
                                                                          rhs64, delta, rho, rs);
        kfn<<<1, NT, L.total, st>>>(Kss, ldk, S, nblk, b, lambda, mdiag, g, rho, W32, rhs64, delta, r,
                                    r == rounds, w64, w32, err, rs);
    }
    if (rs) {  // the fallback overwrites the chain's scratch (its Cholesky factors), never the state
        double *Lbuf = (double *)scratch;
        bdcd_factor_kernel<KT><<<(unsigned)nblk, FAC_THREADS, smf, st>>>(Kss, ldk, b, lambda, mdiag, Lbuf, err, rs);
        bdcd_forward_kernel<KT><<<1, FWD_THREADS, smw, st>>>(Kss, ldk, S, nblk, b, lambda, mdiag, g, Lbuf, delta, w64,
                                                             w32, rs);
    }
    return cudaGetLastError();
}

template <typename KT>
cudaError_t refined_bdcd_b(const KT *Kss, int64_t ldk, const int32_t *S, int nblk, int b, double lambda,
                           double mdiag, const double *g, int refinements, char *scratch, double *delta, double *w64,
                           float *w32, FusedUpdate *upd, int *err, cudaStream_t st)
{
    if (b <= 4)
        return refined_bdcd<KT, 4, 1024>(Kss, ldk, S, nblk, b, lambda, mdiag, g, refinements, scratch, delta, w64,
                                         w32, upd, err, st);
    if (b <= 8)
        return refined_bdcd<KT, 8, 1024>(Kss, ldk, S, nblk, b, lambda, mdiag, g, refinements, scratch, delta, w64,
                                         w32, upd, err, st);
    if (b <= 16)
        return refined_bdcd<KT, 16, 1024>(Kss, ldk, S, nblk, b, lambda, mdiag, g, refinements, scratch, delta, w64,
                                          w32, upd, err, st);
    return refined_bdcd<KT, 32, 512>(Kss, ldk, S, nblk, b, lambda, mdiag, g, refinements, scratch, delta, w64, w32,
                                     upd, err, st);
}

}  // namespace

// The same chain for cnt <= DCD_FAST_MAX with its state in registers: the
// whole CTA first forms the coupling coefficients C[j][t] = y_t y_j K_tj
// (+ omega when S_t = S_j, the repeat term of the unrolled update) in shared
// memory; then one warp runs the chain with lane l holding, for t = l, l+32,
// ..., alpha_t, g_t, 1/eta_t and the pending corrections of g_t and rho_t in
// registers (the gradient correction starts at g_t, so the step's gradient
// is read, not formed).  A step is the owner lane's clipped Newton step
// (Algorithm 2, the arithmetic of recur_dcd_kernel), a broadcast, and one FMA
// per later coordinate.  GB300's FP64 compare-and-select costs ~110 cycles
// of latency against 25 for min/max and 65 for add/FMA (measured), so the
// zero tests on the chain are integer tests of the bit patterns.
constexpr int DCD_FAST_MAX = 128;
constexpr int DCD_FAST_K = DCD_FAST_MAX / 32;

template <typename KT>
// pend (optional): alpha and g at the step's coordinates are pend[0][t] + pend[1][t] and
// pend[2][t] + pend[3][t] (a snapshot and the parts not yet in it) instead of alpha[S[t]], g[S[t]]
__global__ void __launch_bounds__(DCD_THREADS) recur_dcd_fast_kernel(const KT *Kss, int64_t ldk, const int32_t *S,
                                                                     int cnt, const double *y, const double *alpha,
                                                                     const double *g, double omega, double nu,
                                                                     double *delta, double *w64, float *w32,
                                                                     DcdPending pend)
{
    extern __shared__ double fsm[];
    double *C = fsm;                                   // C[j * cnt + t]
    double *yS = C + (size_t)cnt * cnt;
    int32_t *sI = (int32_t *)(yS + cnt);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const int32_t i = S[t];
        sI[t] = i;
        yS[t] = y[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    double a[DCD_FAST_K], gg[DCD_FAST_K], ie[DCD_FAST_K], corr[DCD_FAST_K], rc[DCD_FAST_K], th[DCD_FAST_K];
    auto nonzero = [](double x) { return (__double_as_longlong(x) << 1) != 0; };  // x != 0 (+-0 are zero)
    int32_t id[DCD_FAST_K];
    if (threadIdx.x < 32) {  // the chain warp's state (loads in flight while C is formed)
#pragma unroll
        for (int k = 0; k < DCD_FAST_K; ++k) {
            const int t = 32 * k + lane;
            const bool v = t < cnt;
            const int32_t i = v ? sI[t] : -1;
            id[k] = i;
            if (pend.alpha_snap) {
                a[k] = v ? pend.alpha_snap[t] + pend.alpha_add[t] : 0.0;
                gg[k] = v ? pend.g_snap[t] + pend.g_add[t] : 0.0;
            } else {
                a[k] = v ? alpha[i] : 0.0;
                gg[k] = v ? g[i] : 0.0;
            }
            const double eta = v ? kval(Kss, ldk, t, t) + omega : 0.0;  // G_k = V^T U_k + omega I, y_t^2 = 1
            ie[k] = eta > 0.0 ? 1.0 / eta : 0.0;
            corr[k] = gg[k];  // the gradient of coordinate t as the corrections arrive
            rc[k] = 0.0;
            th[k] = 0.0;
        }
    }
    for (int e = threadIdx.x; e < cnt * cnt; e += blockDim.x) {
        const int j = e / cnt, t = e - j * cnt;
        C[e] = yS[t] * yS[j] * kval(Kss, ldk, t, j) + (sI[t] == sI[j] ? omega : 0.0);
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    double rh[DCD_FAST_K];  // rho_t = alpha_t plus the steps of earlier repeats of its index
#pragma unroll
    for (int k = 0; k < DCD_FAST_K; ++k) rh[k] = a[k] + rc[k];
    const bool clipnu = nu <= 1.7976931348623157e308;  // L1: the box's upper bound; L2: none
#pragma unroll
    for (int k = 0; k < DCD_FAST_K; ++k) {
        if (32 * k >= cnt) break;
        for (int jj = 0; jj < 32 && 32 * k + jj < cnt; ++jj) {
            const int j = 32 * k + jj;
            // every lane forms its coordinate's candidate step (convergent code: GB300's FP64 pipe
            // charges a warp instruction the same with one lane or 32); lane jj's is the step
            double t_j;
            {
                const double rho = rh[k], gj = corr[k];
                double c1 = fmax(rho - gj, 0.0), c2 = fmax(rho - gj * ie[k], 0.0);
                if (clipnu) {
                    c1 = fmin(c1, nu);
                    c2 = fmin(c2, nu);
                }
                // the projected gradient clip(rho - g) - rho is nonzero iff the clip moved rho
                const long long b1 = __double_as_longlong(c1), b0 = __double_as_longlong(rho);
                const bool moved = b1 != b0 && ((b1 | b0) << 1) != 0;  // +0 and -0 are the same value
                t_j = moved && nonzero(ie[k]) ? c2 - rho : 0.0;
                if (lane == jj) th[k] = t_j;
            }
            t_j = __shfl_sync(0xffffffffu, t_j, jj);
            if (nonzero(t_j)) {
                const int32_t ij = __shfl_sync(0xffffffffu, id[k], jj);
                const double *Cj = C + (size_t)j * cnt;
#pragma unroll
                for (int kk = k; kk < DCD_FAST_K; ++kk) {
                    if (32 * kk >= cnt) break;  // warp-uniform
                    const int t = 32 * kk + lane;
                    const bool later = t > j && t < cnt;
                    corr[kk] = fma(later ? Cj[t] : 0.0, t_j, corr[kk]);
                    const bool rep = later && id[kk] == ij;
                    if (__any_sync(0xffffffffu, rep) && rep) rh[kk] += t_j;  // repeats are rare
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < DCD_FAST_K; ++k) {
        const int t = 32 * k + lane;
        if (t < cnt) {
            delta[t] = th[k];
            const double wv = yS[t] * th[k];
            if (w64) w64[t] = wv;
            if (w32) w32[t] = (float)wv;
        }
    }
}

cudaError_t launch_recur_dcd(const void *Kss, int kss_f64, int64_t ldk, const int32_t *S, int64_t cnt,
                             const double *y, const double *alpha, const double *g, double omega, double nu,
                             double *delta, double *w64, float *w32, int *err, cudaStream_t st,
                             const DcdPending *pend)
{
    if (cnt <= 0) return cudaSuccess;
    const DcdPending pd = pend ? *pend : DcdPending{};
    if (pend && cnt > DCD_FAST_MAX) return cudaErrorInvalidValue;
    if (cnt <= DCD_FAST_MAX) {
        const size_t fsm = sizeof(double) * (size_t)(cnt * cnt + cnt) + sizeof(int32_t) * cnt;
        static bool fattr[2] = {false, false};
        if (kss_f64) {
            if (!fattr[1]) {
                cudaError_t e = cudaFuncSetAttribute(recur_dcd_fast_kernel<double>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DCD_SMEM_LIMIT);
                if (e != cudaSuccess) return e;
                fattr[1] = true;
            }
            recur_dcd_fast_kernel<double><<<1, DCD_THREADS, fsm, st>>>((const double *)Kss, ldk, S, (int)cnt, y, alpha,
                                                                       g, omega, nu, delta, w64, w32, pd);
        } else {
            if (!fattr[0]) {
                cudaError_t e = cudaFuncSetAttribute(recur_dcd_fast_kernel<float>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DCD_SMEM_LIMIT);
                if (e != cudaSuccess) return e;
                fattr[0] = true;
            }
            recur_dcd_fast_kernel<float><<<1, DCD_THREADS, fsm, st>>>((const float *)Kss, ldk, S, (int)cnt, y, alpha,
                                                                      g, omega, nu, delta, w64, w32, pd);
        }
        return cudaGetLastError();
    }
    size_t sm = sizeof(double) * 7 * cnt + sizeof(int32_t) * ((cnt + 1) & ~1);
    if (cnt <= DCD_SMEM_GRAM_MAX) sm += sizeof(double) * cnt * cnt;
    if (sm > DCD_SMEM_LIMIT) return cudaErrorInvalidValue;
    static bool attr[2] = {false, false};  // set once per instantiation (also keeps graph capture free of it)
    cudaError_t e;
    if (kss_f64) {
        if (!attr[1]) {
            e = cudaFuncSetAttribute(recur_dcd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)DCD_SMEM_LIMIT);
            if (e != cudaSuccess) return e;
            attr[1] = true;
        }
        recur_dcd_kernel<double><<<1, DCD_THREADS, sm, st>>>((const double *)Kss, ldk, S, (int)cnt, y, alpha, g,
                                                             omega, nu, delta, w64, w32, err);
    } else {
        if (!attr[0]) {
            e = cudaFuncSetAttribute(recur_dcd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)DCD_SMEM_LIMIT);
            if (e != cudaSuccess) return e;
            attr[0] = true;
        }
        recur_dcd_kernel<float><<<1, DCD_THREADS, sm, st>>>((const float *)Kss, ldk, S, (int)cnt, y, alpha, g, omega,
                                                            nu, delta, w64, w32, err);
    }
    return cudaGetLastError();
}

size_t recur_bdcd_scratch_bytes(int64_t nblk, int b)
{
    const size_t sb = (size_t)nblk * b;
    size_t refined = ((sb * b * 4 + 255) / 256) * 256 + 2 * sb * 8;
    size_t generic = sizeof(double) * (size_t)nblk * b * (b + 1);
    const size_t cluster = recur_cluster_scratch_bytes(nblk, b);
    if (cluster > refined) refined = cluster;
    const size_t blocked = blocked_cluster_scratch_bytes(nblk, b);
    if (blocked > refined) refined = blocked;
    // the refinement state of the FP64 form sits past everything a step uses
    return ((refined > generic ? refined : generic) + 255) / 256 * 256 + REFINE_STATE_BYTES;
}

// Refined FP32 chain for b <= 32 and sb <= 8192 (the shared-memory limit of
// one CTA: 12 bytes per sampled row); the plain FP64 kernels otherwise.
bool recur_bdcd_lower_gram(int64_t nblk, int b, int refinements, int64_t ldk)
{
    if (!(b <= 32 && nblk >= 1 && nblk * b <= 8192 && refinements >= 0 &&
          chain_layout((int)(nblk * b), b, 4, ldk).total <= CHAIN_SMEM_MAX))
        return false;
    if (recur_cluster_size((int)nblk, b, refinements + 1) > 0) return true;
    const int pb = recur_cluster_panel_blocks(b, refinements + 1);
    return pb > 0 && pb < nblk && blocked_cluster_scratch_bytes(nblk, b) <= recur_bdcd_scratch_bytes(nblk, b);
}

cudaError_t launch_recur_bdcd(const void *Kss, int kss_f64, int64_t ldk, const int32_t *S, int64_t nblk, int b,
                              double lambda, double mdiag, const double *g, int refinements, void *scratch,
                              double *delta, double *w64, float *w32, FusedUpdate *upd, int *err, cudaStream_t st)
{
    if (upd) upd->done = false;
    if (nblk <= 0) return cudaSuccess;
    if (b <= 32 && nblk * b <= 8192 && refinements >= 0 &&
        chain_layout((int)(nblk * b), b, kss_f64 ? 8 : 4, ldk).total <= CHAIN_SMEM_MAX) {
        if (kss_f64)
            return refined_bdcd_b<double>((const double *)Kss, ldk, S, (int)nblk, b, lambda, mdiag, g, refinements,
                                          (char *)scratch, delta, w64, w32, upd, err, st);
        return refined_bdcd_b<float>((const float *)Kss, ldk, S, (int)nblk, b, lambda, mdiag, g, refinements,
                                     (char *)scratch, delta, w64, w32, upd, err, st);
    }
    double *Lbuf = (double *)scratch;
    size_t smf = sizeof(double) * (size_t)b * b;
    size_t smw = sizeof(double) * ((size_t)nblk * b + b) + sizeof(int32_t) * (size_t)nblk * b;
    if (smf > DCD_SMEM_LIMIT || smw > DCD_SMEM_LIMIT) return cudaErrorInvalidValue;
    static bool attr_set = false;
    cudaError_t e;
    if (!attr_set) {
        for (auto fn : {(const void *)bdcd_factor_kernel<double>, (const void *)bdcd_forward_kernel<double>,
                        (const void *)bdcd_factor_kernel<float>, (const void *)bdcd_forward_kernel<float>}) {
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DCD_SMEM_LIMIT);
            if (e != cudaSuccess) return e;
        }
        attr_set = true;
    }
    if (kss_f64) {
        bdcd_factor_kernel<double><<<(unsigned)nblk, FAC_THREADS, smf, st>>>((const double *)Kss, ldk, b, lambda,
                                                                             mdiag, Lbuf, err);
        bdcd_forward_kernel<double><<<1, FWD_THREADS, smw, st>>>((const double *)Kss, ldk, S, (int)nblk, b, lambda,
                                                                 mdiag, g, Lbuf, delta, w64, w32);
    } else {
        bdcd_factor_kernel<float><<<(unsigned)nblk, FAC_THREADS, smf, st>>>((const float *)Kss, ldk, b, lambda, mdiag,
                                                                            Lbuf, err);
        bdcd_forward_kernel<float><<<1, FWD_THREADS, smw, st>>>((const float *)Kss, ldk, S, (int)nblk, b, lambda,
                                                                mdiag, g, Lbuf, delta, w64, w32);
    }
    return cudaGetLastError();
}

}  // namespace dcd
