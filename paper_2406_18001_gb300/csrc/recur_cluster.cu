// recur_cluster.cu -- the BDCD s-step recurrence (eq. bdcd-sstep, Algorithm 4)
// spread over one thread-block cluster.
//
// The inner system is L Delta = -g_S with L the block lower triangle of G
// (G_jt = Kss_jt / lambda + m [S_j = S_t]).  It is solved in FP32 and refined
// with a residual formed in double-single arithmetic (FP32 pairs, ~2^-44
// relative), which makes the result FP64-accurate for the well-conditioned
// blocks of K-RR while avoiding GB300's slow FP64 pipe.
//
// A single SM cannot stream the sb^2/2 Gram entries fast enough (one SM reads
// L2 at ~40-60 B/clock), so the blocks are dealt block-cyclically to the P
// CTAs of a cluster: CTA c owns blocks j = c, c+P, ...  At start every CTA
// copies its blocks' rows of the lower triangle (and diagonal block) into its
// own shared memory, transposed so that lane p (row p) reads consecutive
// addresses.  Then, for t = 0..nblk-1, the owner of block t forms
// delta_t = W_t r_t (W_t = G_tt^-1 from bdcd_inverse_kernel) and sends delta_t
// and delta_t / lambda to every CTA with st.async stores that complete the
// receiving CTA's per-step mbarrier; every CTA waits for step t's values and
// subtracts G_jt delta_t from the right-hand sides of its later blocks.  Only
// 2b floats cross the cluster per step.  All waits are bounded.
#include "dcd_internal.cuh"
#include "ptx.cuh"

namespace dcd {
namespace {

constexpr int CL_THREADS = 128;
constexpr int CL_KMAX = 8;     // blocks owned per CTA
constexpr int CL_RMAX = 3;     // chain rounds (1 + refinements)
constexpr int CL_PMAX = 16;    // CTAs per cluster
constexpr size_t CL_SMEM_MAX = 224 * 1024;
constexpr unsigned long long CL_WAIT_NS = 2000000000ull;

struct ClLayout {
    size_t recv, sI, prev, rhs, rho, wsm, bars, gdata, total;
    int T, nown;
};

__host__ __device__ inline size_t al16(size_t v) { return (v + 15) & ~(size_t)15; }

// Own block j's Gram rows are stored densely, row p at p * gstride(j) with
// gstride(j) = (j+1) b (16-byte aligned rows for the bulk copies).  Lane p
// reads its row's columns in the rotated order (q + p) mod b, which keeps the
// b lanes of a warp on distinct banks.
__host__ __device__ __forceinline__ int gstride(int j, int b) { return (j + 1) * b; }

// float offset of own block k's Gram rows in CTA c (blocks j = c + k'P hold
// (j+1) b^2 floats each)
__host__ __device__ __forceinline__ size_t goff_f(int k, int c, int P, int b)
{
    return (size_t)b * b * ((size_t)k * (c + 1) + (size_t)P * k * (k - 1) / 2);
}

// Layout of CTA c (the arrays that other CTAs write sit at the same offsets in
// every CTA; the per-CTA Gram part is last).
__host__ __device__ inline ClLayout cl_layout(int nblk, int b, int P, int rounds, int c)
{
    ClLayout L;
    const size_t sb = (size_t)nblk * b;
    size_t cur = 0;
    L.recv = cur;
    cur = al16(cur + (size_t)rounds * sb * 4);
    L.sI = cur;
    cur = al16(cur + sb * 4);
    L.prev = cur;
    cur = al16(cur + sb * 4);
    L.rhs = cur;
    cur = al16(cur + (size_t)CL_KMAX * 32 * 8);
    L.rho = cur;
    cur = al16(cur + (size_t)CL_KMAX * 32 * 8);
    L.wsm = cur;
    cur = al16(cur + (size_t)CL_KMAX * b * b * 4);
    L.bars = cur;
    cur = al16(cur + (size_t)rounds * nblk * 8 + 8);  // + the Gram-load barrier
    L.gdata = cur;
    int T = 2;
    while ((size_t)T < 2 * sb) T <<= 1;
    L.T = T;
    size_t gmax = 0;
    L.nown = 0;
    for (int cc = 0; cc < P; ++cc) {
        size_t gs = 0;
        int k = 0;
        for (int j = cc; j < nblk; j += P, ++k) gs += (size_t)b * gstride(j, b) * 4;
        if (cc == c) L.nown = k;
        if (gs > gmax) gmax = gs;
    }
    const size_t hash = 16 * (size_t)T;  // keys, counts, first and last position per slot
    L.total = L.gdata + (gmax > hash ? gmax : hash);
    return L;
}

// double-single accumulation of an exact product (p, e) into (hi, lo)
__device__ __forceinline__ void ds_add(float &hi, float &lo, float p, float e)
{
    const float s = hi + p;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (p - bp);
    hi = s;
    lo += err + e;
}

template <int BT>
__global__ void __launch_bounds__(CL_THREADS, 1)
    bdcd_cluster_kernel(const float *Kss, int64_t ldk, const int32_t *S, int nblk, int b, double lambda, double mdiag,
                        const double *g, const float *W32, int rounds, double *delta, double *w64, float *w32,
                        int *err)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int P = (int)gridDim.x;  // the grid is one cluster
    const uint32_t c = ptx::cluster_ctarank();
    const int sb = nblk * b;
    const ClLayout L = cl_layout(nblk, b, P, rounds, (int)c);
    float *recv = (float *)(sm + L.recv);  // [round][sb]: delta_t as received
    int32_t *sI = (int32_t *)(sm + L.sI);
    int32_t *prev = (int32_t *)(sm + L.prev);
    double *rhs = (double *)(sm + L.rhs);  // own rows: -g_S
    double *rho = (double *)(sm + L.rho);  // own rows: residual of the last round
    float *wsm = (float *)(sm + L.wsm);    // own blocks: W transposed, [k][q][p]
    uint64_t *bars = (uint64_t *)(sm + L.bars);
    float *gd = (float *)(sm + L.gdata);
    __shared__ int abort_flag;
    constexpr int NWARP = CL_THREADS / 32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float inv_lam = (float)(1.0 / lambda);
    const float mf = (float)mdiag;
    const int nown = L.nown;

    // ---- set-up: barriers, indices, repeated-index chains ----
    // Each index gets its own hash slot (linear probing); a slot counts its
    // occurrences and records the first and last position, which gives the
    // previous occurrence directly when an index occurs at most twice (the
    // rare rows of indices seen three times or more scan back).
    int32_t *hkey = (int32_t *)gd;
    int32_t *hcnt = hkey + L.T;
    int32_t *hmin = hcnt + L.T;
    int32_t *hmax = hmin + L.T;
    uint64_t *lbar = bars + rounds * nblk;
    if (tid == 0) {
        for (int i = 0; i <= rounds * nblk; ++i) ptx::mbar_init(&bars[i], 1);
        ptx::mbar_init_fence();
        abort_flag = 0;
    }
    for (int e = tid; e < L.T; e += CL_THREADS) {
        hkey[e] = -1;
        hcnt[e] = 0;
        hmin[e] = INT32_MAX;
        hmax[e] = -1;
    }
    for (int p = tid; p < sb; p += CL_THREADS) sI[p] = S[p];
    __syncthreads();
    for (int p = tid; p < sb; p += CL_THREADS) {
        const int32_t key = sI[p];
        int h = (int)(((uint32_t)key * 2654435761u) & (uint32_t)(L.T - 1));
        for (int probe = 0; probe < L.T; ++probe) {
            const int32_t old = atomicCAS(&hkey[h], -1, key);
            if (old == -1 || old == key) break;
            h = (h + 1) & (L.T - 1);
        }
        prev[p] = h;
        atomicAdd(&hcnt[h], 1);
        atomicMin(&hmin[h], p);
        atomicMax(&hmax[h], p);
    }
    __syncthreads();
    for (int p = tid; p < sb; p += CL_THREADS) {
        const int h = prev[p];
        int pv = -1;
        if (hcnt[h] == 2) {
            pv = (p == hmax[h]) ? hmin[h] : -1;
        } else if (hcnt[h] > 2) {
            const int32_t key = sI[p];
            for (int q = p - 1; q >= 0; --q)
                if (sI[q] == key) {
                    pv = q;
                    break;
                }
        }
        prev[p] = pv;
    }
    __syncthreads();
    // every step of every round expects delta_t (b floats)
    if (tid == 0)
        for (int i = 0; i < rounds * nblk; ++i) ptx::mbar_expect_tx(&bars[i], (uint32_t)(b * 4));
    // own blocks: Gram rows p of block j up to its diagonal block, by bulk
    // copies (one per row, ncol * 4 bytes, 16-byte aligned: b % 4 == 0,
    // ldk % 4 == 0); W transposed and the right-hand sides by plain loads
    if (warp == 0) {
        uint32_t total = 0;
        for (int k = 0; k < nown; ++k) total += (uint32_t)(((int)c + k * P + 1) * b * b * 4);
        if (lane == 0) ptx::mbar_expect_tx(lbar, total);
        __syncwarp();
        for (int k = 0; k < nown; ++k) {
            const int j = (int)c + k * P, jb = j * b, ncol = (j + 1) * b;
            float *gt = gd + goff_f(k, (int)c, P, b);
            for (int p = lane; p < b; p += 32)
                ptx::bulk_g2s(gt + (size_t)p * ncol, Kss + (int64_t)(jb + p) * ldk, (uint32_t)ncol * 4u, lbar);
        }
    }
    for (int k = 0; k < nown; ++k) {
        const int jb = ((int)c + k * P) * b;
        for (int e = tid; e < b * b; e += CL_THREADS) {
            const int p = e / b, q = e - p * b;  // W32 row-major [p][q]
            wsm[(k * b + q) * b + p] = W32[((int64_t)jb + p) * b + q];
        }
        for (int p = tid; p < b; p += CL_THREADS) rhs[k * 32 + p] = -g[sI[jb + p]];
    }
    if (nown > 0 && !ptx::mbar_wait_bounded(lbar, 0, CL_WAIT_NS)) {
        abort_flag = 1;
        set_error(err, DEV_TIMEOUT);
    }
    __syncthreads();
    ptx::cluster_sync();  // every CTA's barriers exist before any remote store

    for (int r = 0; r < rounds; ++r) {
        float *rv = recv + (size_t)r * sb;
        // Warp w runs the chain for own blocks k = w, w + NWARP, ...: it waits
        // for each delta_t itself, updates its blocks, and when it owns block
        // t it forms and sends delta_t.  No CTA-wide barrier per step.
        float rr[CL_KMAX / NWARP];
#pragma unroll
        for (int i = 0; i < CL_KMAX / NWARP; ++i) {
            const int k = warp + i * NWARP;
            rr[i] = (k < nown && lane < b) ? (float)(r == 0 ? rhs[k * 32 + lane] : rho[k * 32 + lane]) : 0.f;
        }
        const bool has_blocks = warp < nown;
        for (int t = 0; t < nblk && has_blocks; ++t) {
            const int tb = t * b;
            const int kt = t / P;
            if (t % P == (int)c && kt % NWARP == warp) {
                float rk = 0.f;
#pragma unroll
                for (int i = 0; i < CL_KMAX / NWARP; ++i)
                    if (warp + i * NWARP == kt) rk = rr[i];
                const float *wt = wsm + (size_t)kt * b * b;
                float d0 = 0.f, d1 = 0.f;
#pragma unroll
                for (int q = 0; q < BT; q += 2) {
                    const float r0 = __shfl_sync(0xffffffffu, rk, q);
                    const float r1 = __shfl_sync(0xffffffffu, rk, q + 1);
                    if (q < b && lane < b) d0 = fmaf(wt[q * b + lane], r0, d0);
                    if (q + 1 < b && lane < b) d1 = fmaf(wt[(q + 1) * b + lane], r1, d1);
                }
                const float d = d0 + d1;
                float dq[BT];
#pragma unroll
                for (int q = 0; q < BT; ++q) dq[q] = __shfl_sync(0xffffffffu, d, q);
                if (lane < P) {
                    const uint32_t rbar = ptx::mapa(ptx::su32(&bars[r * nblk + t]), (uint32_t)lane);
#pragma unroll
                    for (int v = 0; v < BT / 4; ++v)
                        if (4 * v < b)
                            ptx::st_async_v4(ptx::mapa(ptx::su32(rv + tb + 4 * v), (uint32_t)lane),
                                             make_float4(dq[4 * v], dq[4 * v + 1], dq[4 * v + 2], dq[4 * v + 3]), rbar);
                }
            }
            const bool seen = *(volatile int *)&abort_flag
                                  ? false
                                  : ptx::mbar_wait_cluster_bounded(&bars[r * nblk + t], 0, CL_WAIT_NS);
            if (!__all_sync(0xffffffffu, seen)) {
                if (lane == 0) {
                    *(volatile int *)&abort_flag = 1;
                    set_error(err, DEV_TIMEOUT);
                }
                continue;  // keep walking the steps; every later wait is skipped
            }
            // subtract G_jt delta_t = (K_jt delta_t) / lambda + m [S = S] delta_t
#pragma unroll
            for (int i = 0; i < CL_KMAX / NWARP; ++i) {
                const int k = warp + i * NWARP;
                const int j = (int)c + k * P;
                if (k < nown && j > t && lane < b) {
                    const float *gt = gd + goff_f(k, (int)c, P, b) + (size_t)lane * gstride(j, b) + tb;
                    const float *dt = rv + tb;
                    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
                    int qr = lane;  // rotated column (q + lane) mod b
#pragma unroll
                    for (int q = 0; q < BT; q += 4) {
                        if (q < b) s0 = fmaf(gt[qr], dt[qr], s0);
                        if (++qr == b) qr = 0;
                        if (q + 1 < b) s1 = fmaf(gt[qr], dt[qr], s1);
                        if (++qr == b) qr = 0;
                        if (q + 2 < b) s2 = fmaf(gt[qr], dt[qr], s2);
                        if (++qr == b) qr = 0;
                        if (q + 3 < b) s3 = fmaf(gt[qr], dt[qr], s3);
                        if (++qr == b) qr = 0;
                    }
                    float sm_dup = 0.f;
                    for (int qq = prev[j * b + lane]; qq >= tb; qq = prev[qq])
                        if (qq < tb + b) sm_dup += rv[qq];
                    rr[i] -= ((s0 + s1) + (s2 + s3)) * inv_lam + mf * sm_dup;
                }
            }
        }
        __syncthreads();
        if (r + 1 < rounds && !abort_flag) {
            // residual of own rows p (block j): rho = rhs - (1/lambda) sum_q K_pq Delta_q - m sum_{S_q = S_p} Delta_q,
            // Delta_q = sum_{r' <= r} recv[r'][q] (FP32 values, exact in double); products are split exactly
            // (TwoProd) and summed in double-single; one warp per own block, the columns split across lanes.
            for (int k = warp; k < nown; k += NWARP) {
                const int j = (int)c + k * P, jb = j * b, ncol = (j + 1) * b, ld = gstride(j, b);
                const float *gt = gd + goff_f(k, (int)c, P, b);
                const int half = 32 / b > 0 ? 32 / b : 1;  // lanes per row
                const int p = lane % b, part = lane / b;
                // this lane's columns q = part + half * h, h < nq, visited from h = p mod nq
                const int nq = part < half ? (ncol - part + half - 1) / half : 0;
                const int h0 = nq > 0 ? p % nq : 0;
                float hi = 0.f, lo = 0.f;
                double dm = 0.0;
                if (part < half) {
                    for (int h = 0; h < nq; ++h) {
                        int hq = h + h0;
                        if (hq >= nq) hq -= nq;
                        const int q = part + half * hq;
                        const float kv = gt[p * ld + q];
                        for (int rr2 = 0; rr2 <= r; ++rr2) {
                            const float dvv = recv[(size_t)rr2 * sb + q];
                            const float pr = kv * dvv;
                            ds_add(hi, lo, pr, fmaf(kv, dvv, -pr));
                        }
                    }
                    if (part == 0)  // m [S_q = S_p] over q <= p: the diagonal and earlier repeats
                        for (int qq = jb + p; qq >= 0; qq = (qq == jb + p) ? prev[jb + p] : prev[qq])
                            for (int rr2 = 0; rr2 <= r; ++rr2) dm += (double)recv[(size_t)rr2 * sb + qq];
                }
                const double acc = (double)hi + (double)lo;
                // part 0 adds the partial sums of lanes p + b, p + 2b, ... of the same row
                double tot = acc;
                for (int h = 1; h < half; ++h) tot += __shfl_sync(0xffffffffu, acc, (p + h * b) & 31);
                if (part == 0) rho[k * 32 + p] = rhs[k * 32 + p] - (tot / lambda + mdiag * dm);
            }
            __syncthreads();
        }
    }
    if (abort_flag && tid == 0)  // let remote stores still addressed to this CTA land (short bound)
        for (int i = 0; i < rounds * nblk; ++i) ptx::mbar_wait_cluster_bounded(&bars[i], 0, 10000000ull);
    __syncthreads();
    // own rows: Delta = sum over rounds
    for (int k = 0; k < nown; ++k) {
        const int jb = ((int)c + k * P) * b;
        for (int p = tid; p < b; p += CL_THREADS) {
            double d = 0.0;
            for (int r = 0; r < rounds; ++r) d += (double)recv[(size_t)r * sb + jb + p];
            delta[jb + p] = d;
            if (w64) w64[jb + p] = d / lambda;
            if (w32) w32[jb + p] = (float)(d / lambda);
        }
    }
    __syncthreads();
    ptx::cluster_sync();  // no CTA leaves while another may still address it
}

struct ClusterCache {
    int P = 0, nblk = 0, b = 0, rounds = 0, ok = -1;
};

template <int BT>
cudaError_t launch_cluster(const float *Kss, int64_t ldk, const int32_t *S, int nblk, int b, int P, double lambda,
                           double mdiag, const double *g, const float *W32, int rounds, size_t smem, double *delta,
                           double *w64, float *w32, int *err, cudaStream_t st)
{
    auto kfn = bdcd_cluster_kernel<BT>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CL_SMEM_MAX);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)P, 1, 1);
    cfg.blockDim = dim3(CL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)P;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kfn, Kss, ldk, S, nblk, b, lambda, mdiag, g, W32, rounds, delta, w64, w32, err);
}

template <int BT>
bool cluster_fits(int P, size_t smem)
{
    auto kfn = bdcd_cluster_kernel<BT>;
    if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CL_SMEM_MAX) != cudaSuccess)
        return false;
    if (cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)P, 1, 1);
    cfg.blockDim = dim3(CL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)P;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kfn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n >= 1;
}

}  // namespace

// Cluster size for nblk blocks of size b (0: the cluster path does not apply).
int recur_cluster_size(int nblk, int b, int rounds)
{
    if (b % 4 != 0 || b > 32 || rounds < 1 || rounds > CL_RMAX || nblk < 8) return 0;
    const int P = nblk < CL_PMAX ? nblk : CL_PMAX;
    size_t smem = 0;
    for (int c = 0; c < P; ++c) {
        const ClLayout L = cl_layout(nblk, b, P, rounds, c);
        if (L.nown > CL_KMAX) return 0;
        if (L.total > smem) smem = L.total;
    }
    if (smem > CL_SMEM_MAX) return 0;
    static int cache_P = -1, cache_key[3] = {0, 0, 0};
    if (cache_key[0] == nblk && cache_key[1] == b && cache_key[2] == rounds) return cache_P;
    bool ok = b <= 4 ? cluster_fits<4>(P, smem) : b <= 8 ? cluster_fits<8>(P, smem)
                                                        : b <= 16 ? cluster_fits<16>(P, smem) : cluster_fits<32>(P, smem);
    cache_key[0] = nblk;
    cache_key[1] = b;
    cache_key[2] = rounds;
    cache_P = ok ? P : 0;
    return cache_P;
}

cudaError_t launch_recur_cluster(const float *Kss, int64_t ldk, const int32_t *S, int nblk, int b, int P,
                                 double lambda, double mdiag, const double *g, const float *W32, int rounds,
                                 double *delta, double *w64, float *w32, int *err, cudaStream_t st)
{
    size_t smem = 0;
    for (int c = 0; c < P; ++c) {
        const ClLayout L = cl_layout(nblk, b, P, rounds, c);
        if (L.total > smem) smem = L.total;
    }
    if (b <= 4)
        return launch_cluster<4>(Kss, ldk, S, nblk, b, P, lambda, mdiag, g, W32, rounds, smem, delta, w64, w32, err, st);
    if (b <= 8)
        return launch_cluster<8>(Kss, ldk, S, nblk, b, P, lambda, mdiag, g, W32, rounds, smem, delta, w64, w32, err, st);
    if (b <= 16)
        return launch_cluster<16>(Kss, ldk, S, nblk, b, P, lambda, mdiag, g, W32, rounds, smem, delta, w64, w32, err,
                                  st);
    return launch_cluster<32>(Kss, ldk, S, nblk, b, P, lambda, mdiag, g, W32, rounds, smem, delta, w64, w32, err, st);
}

}  // namespace dcd
