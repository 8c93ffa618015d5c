// recur_cluster.cu -- the BDCD s-step recurrence (eq. bdcd-sstep, Algorithm 4)
// on one thread-block cluster, in super-blocks of up to 32 rows.
//
// The inner system is L Delta = -g_S with L the block lower triangle of G
// (G_jt = Kss_jt / lambda + m [S_j = S_t]).  It is solved in FP32 and refined
// once: Delta0 from an FP32 block forward substitution, the residual
// rho = -g_S - L Delta0 with every product split exactly (TwoProd) and summed
// in double-single arithmetic (~2^-44 relative), Delta1 from a second FP32
// substitution on rho, Delta = Delta0 + Delta1.  That is FP64-accurate for the
// well-conditioned blocks of K-RR while avoiding GB300's slow FP64 pipe.
//
// Consecutive blocks are grouped into super-blocks of q = 32 / b blocks
// (Bs = q b <= 32 rows, one row per lane).  bdcd_prep_kernel inverts the
// diagonal part L_JJ of every super-block at once (Gauss-Jordan with one
// thread per entry; L_JJ is block lower triangular with SPD diagonal blocks,
// so no pivoting; one CTA per super-block) while a second set of CTAs marks
// repeated indices and links their occurrences, so a chain step is
// Delta_J = L_JJ^-1 r_J after r_J -= L_JT Delta_T for every earlier T: the
// block forward substitution with the steps inside a super-block regrouped
// into one matrix-vector product.
//
// The sb^2/2 Gram entries do not fit one SM's shared memory and one SM reads
// L2 at only ~40-60 B/clock, so the super-blocks are dealt to the P CTAs of a
// cluster, two per CTA, folded (CTA c owns J = c and 2P-1-c, which balances
// the triangle); each CTA copies its rows' Gram panels (Bs x Bs, row-major)
// once by 2-D TMA.  Per own super-block a CTA runs two warps:
//   round-0 warp: applies Delta0_T as it arrives (T < J), forms Delta0_J
//                 and sends it to every CTA (st.async, completing the
//                 receiver's per-step mbarrier); it accumulates the
//                 double-single residual of its rows panel by panel while it
//                 waits, so rho_J is ready just after Delta0_J;
//   round-1 warp: applies Delta1_T as it arrives and once rho_J is ready
//                 forms Delta1_J, sends it and writes Delta = Delta0 + Delta1.
// The refinement chain thus runs a little behind the first one instead of
// after it.  Panel rows are read as float4 chunks in a lane-rotated order
// (conflict-free).  Every wait is bounded; on expiry the kernel records
// DEV_TIMEOUT, skips its remaining waits and still lets every store
// addressed to it land (bounded) before it leaves.
#include "dcd_internal.cuh"
#include "ptx.cuh"

#include <map>
#include <mutex>

namespace dcd {
namespace {

constexpr int CL_THREADS = 128;  // warps: slot 0 round 0, slot 1 round 0, slot 0 round 1, slot 1 round 1
constexpr int CL_SLOTS = 2;      // own super-blocks per CTA
constexpr int CL_PMAX = 16;      // CTAs per cluster (non-portable size)
constexpr int CL_NSUP_MAX = 2 * CL_PMAX;
constexpr size_t CL_SMEM_MAX = 224 * 1024;
constexpr unsigned long long CL_WAIT_NS = 2000000000ull;
constexpr int NLOCAL = 3 * CL_SLOTS;  // per slot: diagonal panel, other panels, rho ready
constexpr int PREP_THREADS = 256;

struct ClGeom {
    int q, Bs, nsup;
};

__host__ __device__ inline ClGeom cl_geom(int nblk, int b)
{
    ClGeom G;
    G.q = b >= 32 ? 1 : 32 / b;
    G.Bs = G.q * b;
    G.nsup = (nblk + G.q - 1) / G.q;
    return G;
}

// super-block of own slot k of CTA c (folded over 2P)
__host__ __device__ inline int cl_own(int k, int c, int P) { return k == 0 ? c : 2 * P - 1 - c; }

// rows of super-block J
__host__ __device__ inline int cl_rows(int J, int Bs, int sb)
{
    const int r = sb - J * Bs;
    return r < Bs ? r : Bs;
}

struct ClLayout {
    size_t recv, xs, ns, dmask, dsend, rbuf, rho, bars, gdata, ps, total;
    int nown;
};

__host__ __device__ inline size_t al16(size_t v) { return (v + 15) & ~(size_t)15; }

// Layout of CTA c.  Everything other CTAs address (recv, bars) sits at the
// same offset in every CTA; the per-CTA Gram panels are last, from the first
// 128-byte boundary at or after gdata (TMA destinations).  Own slot k keeps
// its J+1 panels (T = 0..J) in order.
__host__ __device__ inline ClLayout cl_layout(int nblk, int b, int P, int c)
{
    const ClGeom G = cl_geom(nblk, b);
    const size_t sb = (size_t)nblk * b;
    ClLayout L;
    size_t cur = 0;
    L.recv = cur;
    cur = al16(cur + 2 * sb * 4);
    L.xs = cur;
    cur = al16(cur + (size_t)CL_SLOTS * 32 * 32 * 4);
    L.ns = cur;
    cur = al16(cur + (size_t)CL_SLOTS * 32 * 32 * 4);
    L.dmask = cur;
    cur = al16(cur + (size_t)CL_SLOTS * CL_NSUP_MAX * 32 * 4);
    L.dsend = cur;
    cur = al16(cur + (size_t)2 * CL_SLOTS * 32 * 4);
    L.rbuf = cur;
    cur = al16(cur + (size_t)2 * CL_SLOTS * 32 * 4);
    L.rho = cur;
    cur = al16(cur + (size_t)CL_SLOTS * 32 * 8);
    L.bars = cur;
    cur = al16(cur + ((size_t)2 * G.nsup + NLOCAL) * 8);
    L.gdata = cur;
    L.ps = ((size_t)G.Bs * G.Bs * 4 + 127) & ~(size_t)127;
    size_t panels = 0;
    L.nown = 0;
    for (int k = 0; k < CL_SLOTS; ++k) {
        const int J = cl_own(k, c, P);
        if (J >= G.nsup || (k == 1 && J == cl_own(0, c, P))) break;
        panels += (size_t)J + 1;
        L.nown = k + 1;
    }
    L.total = L.gdata + 128 + panels * L.ps;
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

__device__ __forceinline__ void ds_prod(float &hi, float &lo, float kv, float dv)
{
    const float pp = kv * dv;
    ds_add(hi, lo, pp, fmaf(kv, dv, -pp));
}

// Row `lane` of a panel (ncol columns, a multiple of 4) times v, FP32: float4
// chunks visited from chunk `lane` onwards (mod ncol / 4), so the lanes of a
// quarter-warp read distinct banks.
__device__ __forceinline__ float panel_dot(const float *pr, const float *v, int lane, int ncol)
{
    const int nc = ncol >> 2;
    const int m0 = nc == 8 ? (lane & 7) : lane % nc;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j < nc) {
            int m = m0 + j;
            m -= m >= nc ? nc : 0;
            const float4 a = *(const float4 *)(pr + 4 * m), x = *(const float4 *)(v + 4 * m);
            s0 = fmaf(a.x, x.x, s0);
            s1 = fmaf(a.y, x.y, s1);
            s2 = fmaf(a.z, x.z, s2);
            s3 = fmaf(a.w, x.w, s3);
        }
    }
    return (s0 + s1) + (s2 + s3);
}

// The same dot product as a double-single pair, each product exact (TwoProd).
__device__ __forceinline__ void panel_dot_ds(const float *pr, const float *v, int lane, int ncol, float &hi, float &lo)
{
    const int nc = ncol >> 2;
    const int m0 = nc == 8 ? (lane & 7) : lane % nc;
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f, h3 = 0.f, l3 = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j < nc) {
            int m = m0 + j;
            m -= m >= nc ? nc : 0;
            const float4 a = *(const float4 *)(pr + 4 * m), x = *(const float4 *)(v + 4 * m);
            ds_prod(h0, l0, a.x, x.x);
            ds_prod(h1, l1, a.y, x.y);
            ds_prod(h2, l2, a.z, x.z);
            ds_prod(h3, l3, a.w, x.w);
        }
    }
    ds_add(h0, l0, h1, l1);
    ds_add(h2, l2, h3, l3);
    ds_add(h0, l0, h2, l2);
    hi = h0;
    lo = l0;
}

// sum of v over the set bits of mask
__device__ __forceinline__ float mask_sum(uint32_t mask, const float *v)
{
    float s = 0.f;
    while (mask) {
        s += v[__ffs(mask) - 1];
        mask &= mask - 1;
    }
    return s;
}

__device__ __forceinline__ bool wait_local(uint64_t *bar, volatile int *abort_flag, int *err)
{
    const bool ok = !*abort_flag && ptx::mbar_wait_bounded(bar, 0, CL_WAIT_NS);
    if (!__all_sync(0xffffffffu, ok)) {
        if ((threadIdx.x & 31) == 0 && !*abort_flag) {
            *abort_flag = 1;
            set_error(err, DEV_TIMEOUT);
        }
        return false;
    }
    return true;
}

__device__ __forceinline__ bool wait_remote(uint64_t *bar, volatile int *abort_flag, int *err)
{
    const bool ok = !*abort_flag && ptx::mbar_wait_cluster_bounded(bar, 0, CL_WAIT_NS);
    if (!__all_sync(0xffffffffu, ok)) {
        if ((threadIdx.x & 31) == 0 && !*abort_flag) {
            *abort_flag = 1;
            set_error(err, DEV_TIMEOUT);
        }
        return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Per super-block J (one CTA of 8 warps; lane j, rows i0 + 8 r):
//   M[J][T][p]: bit q set when position T*Bs + q precedes row J*Bs + p and
//          holds the same index (T <= J): the repeats that the m I term of
//          G couples across overlapping blocks;
//   X[J] = L_JJ^-1 (32 x 32 row-major, FP32; rows and columns past the
//          super-block's rows hold the identity), by Gauss-Jordan on
//          [L_JJ | I] (a thread owns columns j and j+32 of its rows; the
//          matrix is double-buffered so a pivot step needs one barrier); a
//          pivot that is not positive and finite records DEV_NOT_SPD;
//   N[J] = X_J L_{J,J-1} (J >= 1) with L_{J,J-1} = K_{J,J-1} / lambda + m D,
//          D the repeat pattern between J and J-1: the whole coupling of
//          super-block J to its predecessor in one matrix, so that a chain
//          step is Delta_J = X_J r'_J - N_J Delta_{J-1}.
__global__ void __launch_bounds__(PREP_THREADS)
    bdcd_prep_kernel(const float *Kss, int64_t ldk, const int32_t *S, int nblk, int b, float inv_lam, float mf,
                     float *X, float *N, uint32_t *M, int32_t *next, int *err)
{
    constexpr int RPT = 32 / (PREP_THREADS / 32);  // rows per thread
    __shared__ float a[2][32][65];
    __shared__ int sIJ[32], sIT[CL_NSUP_MAX * 32];
    __shared__ int bad, nxt[32];
    const ClGeom G = cl_geom(nblk, b);
    const int Bs = G.Bs, sb = nblk * b;
    const bool links = (int)blockIdx.x >= G.nsup;  // the second half of the grid: masks and links
    const int J = links ? (int)blockIdx.x - G.nsup : (int)blockIdx.x;
    const int base = J * Bs, rows = cl_rows(J, Bs, sb);
    const int i0 = threadIdx.x >> 5, j = threadIdx.x & 31;  // rows i0 + 8 r
    if (threadIdx.x == 0) bad = 0;
    if (threadIdx.x < 32) nxt[threadIdx.x] = INT32_MAX;
    for (int e = threadIdx.x; e < sb; e += PREP_THREADS) sIT[e] = S[e];
    __syncthreads();
    if (links) {
        // next[row]: the next position holding the same index (-1: none); warp i0 scans the
        // positions row + 1 + i0, row + 9 + i0, ... up to its first match, the minimum wins
        if (j < rows) {
            const int row = base + j, key = sIT[row];
            for (int q = row + 1 + i0; q < sb; q += PREP_THREADS / 32)
                if (sIT[q] == key) {
                    atomicMin(&nxt[j], q);
                    break;
                }
        }
        // repeat masks: (T, p = j) for T = i0 + 8 r <= J
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int T = i0 + 8 * r;
            if (T <= J) {
                const int key = j < rows ? sIT[base + j] : -1, row = base + j, tb = T * Bs, tr = cl_rows(T, Bs, sb);
                uint32_t mask = 0;
                for (int q = 0; q < tr; ++q)
                    if (sIT[tb + q] == key && tb + q < row) mask |= 1u << q;
                M[((size_t)J * CL_NSUP_MAX + T) * 32 + j] = mask;
            }
        }
        __syncthreads();
        if (threadIdx.x < rows) next[base + threadIdx.x] = nxt[threadIdx.x] == INT32_MAX ? -1 : nxt[threadIdx.x];
        return;
    }
    if (threadIdx.x < 32) sIJ[threadIdx.x] = threadIdx.x < rows ? sIT[base + threadIdx.x] : -1;
    // [L_JJ | I]
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int i = i0 + 8 * r;
        float v = (i == j) ? 1.f : 0.f;
        if (i < rows && j < rows) {
            v = 0.f;
            if (j / b <= i / b)
                v = Kss[(int64_t)(base + i) * ldk + base + j] * inv_lam + (sIT[base + i] == sIT[base + j] ? mf : 0.f);
        }
        a[0][i][j] = v;
        a[0][i][j + 32] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();
    int cur = 0;
    for (int k = 0; k < 32; ++k) {
        const float piv = a[cur][k][k];
        if (!(piv > 0.f) || !(piv < INFINITY)) {  // the same value in every thread
            if (threadIdx.x == 0) bad = 1;
            break;
        }
        const float ip = __frcp_rn(piv);  // = 1.f / piv (both correctly rounded)
        const float p0 = a[cur][k][j] * ip, p1 = a[cur][k][j + 32] * ip;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int i = i0 + 8 * r;
            const float f = a[cur][i][k];
            a[cur ^ 1][i][j] = (i == k) ? p0 : fmaf(-f, p0, a[cur][i][j]);
            a[cur ^ 1][i][j + 32] = (i == k) ? p1 : fmaf(-f, p1, a[cur][i][j + 32]);
        }
        cur ^= 1;
        __syncthreads();
    }
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) set_error(err, DEV_NOT_SPD);
        return;
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) X[(size_t)J * 1024 + (i0 + 8 * r) * 32 + j] = a[cur][i0 + 8 * r][j + 32];
    if (J == 0) return;
    // N_J = X_J (K_{J,J-1} / lambda + m D): B[t][c] in the other buffer, then row i of X times column j of B
    const int pb = (J - 1) * Bs;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int t = i0 + 8 * r;
        float v = 0.f;
        if (t < rows && j < Bs)
            v = Kss[(int64_t)(base + t) * ldk + pb + j] * inv_lam + (sIJ[t] == sIT[pb + j] ? mf : 0.f);
        a[cur ^ 1][t][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int i = i0 + 8 * r;
        float n = 0.f;
#pragma unroll 8
        for (int t = 0; t < 32; ++t) n = fmaf(a[cur][i][32 + t], a[cur ^ 1][t][j], n);
        N[(size_t)J * 1024 + i * 32 + j] = n;
    }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CL_THREADS, 1)
    bdcd_cluster_kernel(const __grid_constant__ CUtensorMap kmap, const int32_t *S, const float *X,
                        const float *Ng, const uint32_t *Mg, const int32_t *nextg, int nblk, int b, double lambda,
                        double mdiag, double *g, int rounds, double *delta, double *w64, float *w32, double *alpha,
                        uint64_t *ctr, uint64_t ctr_advance, const double *rhs_in, int rhs_add_g, int trig_sup,
                        int *err)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int P = (int)gridDim.x;  // the grid is one cluster
    const int c = (int)ptx::cluster_ctarank();
    const ClGeom G = cl_geom(nblk, b);
    const int Bs = G.Bs, nsup = G.nsup, sb = nblk * b;
    const ClLayout L = cl_layout(nblk, b, P, c);
    float *recv = (float *)(sm + L.recv);          // [round][sb]: Delta_round as received
    float *xsa = (float *)(sm + L.xs);             // [slot][32][32]: L_JJ^-1, row-major
    float *nsa = (float *)(sm + L.ns);             // [slot][32][32]: L_JJ^-1 L_{J,J-1}, row-major
    uint32_t *dmask = (uint32_t *)(sm + L.dmask);  // [slot][T][lane]
    float *dsend = (float *)(sm + L.dsend);        // [round][slot][32]: own Delta_J
    float *rbufa = (float *)(sm + L.rbuf);         // [round][slot][32]: r_J before the product
    double *rhoa = (double *)(sm + L.rho);         // [slot][32]
    uint64_t *bars = (uint64_t *)(sm + L.bars);    // [round][J], then the local barriers
    uint64_t *lb = bars + 2 * nsup;
    const uint32_t goff = ptx::su32(sm + L.gdata);
    unsigned char *gd = sm + L.gdata + ((128u - (goff & 127u)) & 127u);
    __shared__ int abort_flag_s;
    volatile int *abort_flag = &abort_flag_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int slot = warp & 1, role = warp >> 1;
    const int nown = L.nown;
    // A kernel launched after this one as a programmatic dependent (the fused block, on the SMs
    // this cluster leaves free) may start its set-up and tensor-core products once every CTA has
    // signalled; it waits for this grid to finish before it reads the coefficients or the
    // gradient.  The CTA owning super-block trig_sup signals when its round-0 Delta is out (the
    // kernels forked beside the chain have the other SMs until then); every other CTA at once.
    const bool trig_own = trig_sup >= 0 && (trig_sup == cl_own(0, c, P) || (nown > 1 && trig_sup == cl_own(1, c, P)));
    // -(g_S + rhs_in) is read before this CTA signals: a dependent may write g once every CTA has
    __shared__ double rhs_pre[CL_SLOTS * 32];
    if (rhs_in && rhs_add_g) {
        for (int e = tid; e < nown * 32; e += CL_THREADS) {
            const int k = e >> 5, i = e & 31, J = cl_own(k, c, P);
            if (i < cl_rows(J, Bs, sb)) rhs_pre[e] = -(g[S[J * Bs + i]] + rhs_in[J * Bs + i]);
        }
        __syncthreads();
    }
    if (tid == 0 && !trig_own) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const float inv_lam = (float)(1.0 / lambda);
    const float mf = (float)mdiag;

    // ---- set-up: barriers, Gram panels, inverses, repeat masks ----
    if (tid == 0) {
        for (int i = 0; i < 2 * nsup + NLOCAL; ++i) ptx::mbar_init(&bars[i], 1);
        ptx::mbar_init_fence();
        abort_flag_s = 0;
    }
    __syncthreads();
    if (tid == 0) {
        for (int r = 0; r < rounds; ++r)
            for (int J = 0; J < nsup; ++J) ptx::mbar_expect_tx(&bars[r * nsup + J], (uint32_t)(cl_rows(J, Bs, sb) * 4));
        // the panels the chain needs (T < J) first, the diagonal ones (residual only) last
        size_t base = 0;
        for (int k = 0; k < nown; ++k) {
            const int J = cl_own(k, c, P);
            if (J > 0) {
                ptx::mbar_expect_tx(&lb[3 * k + 1], (uint32_t)(J * Bs * Bs * 4));
                for (int T = 0; T < J; ++T)
                    ptx::tma_load_2d(gd + (base + T) * L.ps, &kmap, &lb[3 * k + 1], T * Bs, J * Bs);
            }
            base += (size_t)J + 1;
        }
        base = 0;
        for (int k = 0; k < nown; ++k) {
            const int J = cl_own(k, c, P);
            ptx::mbar_expect_tx(&lb[3 * k + 0], (uint32_t)(Bs * Bs * 4));
            ptx::tma_load_2d(gd + (base + J) * L.ps, &kmap, &lb[3 * k + 0], J * Bs, J * Bs);
            base += (size_t)J + 1;
        }
    }
    for (int k = 0; k < nown; ++k) {
        const int J = cl_own(k, c, P);
        const float4 *xg = (const float4 *)(X + (size_t)J * 1024), *ng = (const float4 *)(Ng + (size_t)J * 1024);
        float4 *xd = (float4 *)(xsa + k * 1024), *nd = (float4 *)(nsa + k * 1024);
        for (int e = tid; e < 256; e += CL_THREADS) {
            xd[e] = xg[e];
            if (J > 0) nd[e] = ng[e];
        }
        for (int e = tid; e < (J + 1) * 32; e += CL_THREADS)
            dmask[k * CL_NSUP_MAX * 32 + e] = Mg[(size_t)J * CL_NSUP_MAX * 32 + e];
    }
    __syncthreads();
    ptx::cluster_sync();  // every CTA's barriers exist and expect their bytes before any remote store

    const int J = slot < nown ? cl_own(slot, c, P) : -1;
    if (J >= 0 && role < rounds) {
        const int rows = cl_rows(J, Bs, sb);
        const int row = J * Bs + lane;  // this lane's position in S (used for lane < rows)
        const float *pan = (const float *)(gd + (slot == 0 ? 0 : (size_t)cl_own(0, c, P) + 1) * L.ps);
        const size_t pstride = L.ps / 4;
        const float *xs = xsa + slot * 1024, *ns = nsa + slot * 1024;
        const uint32_t *dm = dmask + slot * CL_NSUP_MAX * 32;
        uint64_t *dbar = &lb[3 * slot + 0], *pbar = &lb[3 * slot + 1], *rbar = &lb[3 * slot + 2];
        const int r = role;  // the round this warp runs
        float *rv = recv + (size_t)r * sb;
        float *ds = dsend + (r * CL_SLOTS + slot) * 32;
        float *rb = rbufa + (r * CL_SLOTS + slot) * 32;
        // remote addresses of this warp's sends (Delta_J, rows/4 float4 parts, to every CTA)
        const int nparts = rows / 4, nsend = P * nparts;
        uint32_t raddr[4], rbarr[4];
        int soff[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int i = lane + 32 * t;
            const int dest = i < nsend ? i / nparts : 0, pt = i < nsend ? i - dest * nparts : 0;
            raddr[t] = ptx::mapa(ptx::su32(rv + J * Bs + 4 * pt), (uint32_t)dest);
            rbarr[t] = ptx::mapa(ptx::su32(&bars[r * nsup + J]), (uint32_t)dest);
            soff[t] = 4 * pt;
        }

        // ---- the chain of round r ----
        // r'_J: all updates but the one from J-1, which N_J = X_J L_{J,J-1} applies after the product:
        // Delta_J = X_J r'_J - N_J Delta_{J-1}.  X_J r'_J is formed while Delta_{J-1} is on its way.
        // the right-hand side: -g_S; or given (rhs_in); or -(g_S + rhs_in), a part of the gradient
        // not yet in g added first (rhs_add_g; read at the start)
        const double rhs = lane >= rows ? 0.0
                           : !rhs_in    ? -g[S[row]]
                           : rhs_add_g  ? rhs_pre[slot * 32 + lane]
                                        : rhs_in[row];
        float rr = r == 0 ? (float)rhs : 0.f;  // round 0: -g_S minus updates; round 1: sum of updates
        float hi = 0.f, lo = 0.f;              // round 0: double-single sum of L_{row, T<J} Delta0_T
        bool alive = J == 0 || wait_local(pbar, abort_flag, err);
        for (int T = 0; T + 1 < J && alive; ++T) {
            if (!wait_remote(&bars[r * nsup + T], abort_flag, err)) {
                alive = false;
                break;
            }
            if (lane < rows) {
                const float *pr = pan + (size_t)T * pstride + lane * Bs;
                const float *dt = rv + T * Bs;
                const uint32_t mk = dm[T * 32 + lane];
                const float sd = mk ? mask_sum(mk, dt) : 0.f;
                if (r == 0) {  // exact sum, also for the residual
                    float h, l;
                    panel_dot_ds(pr, dt, lane, Bs, h, l);
                    ds_add(hi, lo, h, l);
                    rr -= h * inv_lam + mf * sd;
                } else {
                    rr += panel_dot(pr, dt, lane, Bs) * inv_lam + mf * sd;
                }
            }
        }
        if (r == 1 && alive) {
            alive = wait_local(rbar, abort_flag, err);  // rho_J from the round-0 warp
            rr = lane < rows ? (float)rhoa[slot * 32 + lane] - rr : 0.f;
        }
        float d = 0.f;
        if (alive) {
            rb[lane] = lane < rows ? rr : 0.f;
            __syncwarp();
            d = panel_dot(xs + lane * 32, rb, lane, 32);  // X_J r'_J (X row `lane` in rotated float4 chunks)
        }
        if (alive && J > 0) {
            if (wait_remote(&bars[r * nsup + J - 1], abort_flag, err))
                d -= panel_dot(ns + lane * 32, rv + (J - 1) * Bs, lane, Bs);
            else
                alive = false;
        }
        if (alive) {
            // Delta_J to every CTA of the cluster (this one included)
            ds[lane] = lane < rows ? d : 0.f;
            __syncwarp();
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (lane + 32 * t < nsend) ptx::st_async_v4(raddr[t], *(const float4 *)(ds + soff[t]), rbarr[t]);
            if (r == 0 && rounds > 1) {
                // residual rho_J = -g_J - L_{J, T<=J} Delta0 (double-single products; FP64 repeat term)
                const bool okd = wait_local(dbar, abort_flag, err);
                if (okd && lane < rows) {
                    if (J > 0) {
                        float h, l;
                        panel_dot_ds(pan + (size_t)(J - 1) * pstride + lane * Bs, rv + (J - 1) * Bs, lane, Bs, h, l);
                        ds_add(hi, lo, h, l);
                    }
                    float h, l;  // the diagonal panel: the blocks up to this row's block
                    panel_dot_ds(pan + (size_t)J * pstride + lane * Bs, ds, lane, (lane / b + 1) * b, h, l);
                    ds_add(hi, lo, h, l);
                    double dmv = (double)ds[lane];
                    for (int T = 0; T <= J; ++T) {
                        uint32_t mask = dm[T * 32 + lane];
                        const float *v = T < J ? rv + T * Bs : ds;
                        while (mask) {
                            dmv += (double)v[__ffs(mask) - 1];
                            mask &= mask - 1;
                        }
                    }
                    rhoa[slot * 32 + lane] = rhs - (((double)hi + (double)lo) / lambda + mdiag * dmv);
                }
            } else if (lane < rows) {
                // Delta = sum over rounds
                const double dd = (rounds > 1 ? (double)dsend[(0 * CL_SLOTS + slot) * 32 + lane] : 0.0) + (double)d;
                delta[row] = dd;
                if (w64) w64[row] = dd / lambda;
                if (w32) w32[row] = (float)(dd / lambda);
            }
        }
        if (r == 0 && J == trig_sup && lane == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        if (r == 0 && rounds > 1) {  // always release the round-1 warp (it gives up if this one did)
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(rbar);
        }
    }
    // every Delta addressed to this CTA, and every panel copy, lands before it leaves
    if (tid == 0) {
        for (int k = 0; k < nown; ++k) {
            const unsigned long long lim = *abort_flag ? 10000000ull : CL_WAIT_NS;
            bool ok = ptx::mbar_wait_bounded(&lb[3 * k + 0], 0, lim);
            if (cl_own(k, c, P) > 0) ok = ptx::mbar_wait_bounded(&lb[3 * k + 1], 0, lim) && ok;
            if (!ok && !*abort_flag) {
                *abort_flag = 1;
                set_error(err, DEV_TIMEOUT);
            }
        }
        for (int i = 0; i < rounds * nsup; ++i) {
            const unsigned long long lim = *abort_flag ? 10000000ull : CL_WAIT_NS;
            if (!ptx::mbar_wait_cluster_bounded(&bars[i], 0, lim) && !*abort_flag) {
                *abort_flag = 1;
                set_error(err, DEV_TIMEOUT);
            }
        }
    }
    __syncthreads();
    // a6 for the own rows, now that every Delta has landed here: a row holding the first occurrence
    // of its index adds Delta (over the rounds) of all occurrences, in position order, to alpha and
    // mdiag times that to g (the same sums, in the same order, as the sorted update)
    if (alpha && !*abort_flag && J >= 0 && role == 0 && lane < cl_rows(J, Bs, sb)) {
        const int row = J * Bs + lane;
        bool head = true;
        for (int T = 0; T <= J; ++T) head = head && dmask[slot * CL_NSUP_MAX * 32 + T * 32 + lane] == 0;
        if (head) {
            auto dsum = [&](int q) {
                double d = 0.0;
                for (int r = 0; r < rounds; ++r) d += (double)recv[(size_t)r * sb + q];
                return d;
            };
            double sum = dsum(row);
            for (int q = nextg[row]; q > row; q = nextg[q]) sum += dsum(q);
            const int32_t i = S[row];
            alpha[i] += sum;
            g[i] += mdiag * sum;
        }
    }
    if (alpha && tid == 0 && c == 0 && ctr) *ctr += ctr_advance;
    ptx::cluster_sync();  // no CTA leaves while another may still address it
}

bool cluster_fits(int P, size_t smem)
{
    auto kfn = bdcd_cluster_kernel;
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

// two super-blocks per CTA
int cluster_ctas(int nsup) { return (nsup + 1) / 2; }

size_t cluster_smem(int nblk, int b, int P)
{
    size_t smem = 0;
    for (int c = 0; c < P; ++c) {
        const ClLayout L = cl_layout(nblk, b, P, c);
        if (L.total > smem) smem = L.total;
    }
    return smem;
}

}  // namespace

// Cluster size for nblk blocks of size b (0: the cluster path does not apply).
int recur_cluster_size(int nblk, int b, int rounds)
{
    if (b % 4 != 0 || b > 32 || rounds < 1 || rounds > 2 || nblk < 1) return 0;
    const ClGeom G = cl_geom(nblk, b);
    if (G.nsup > CL_NSUP_MAX) return 0;
    // one occupancy query per shape (a map: batched solves mix shapes)
    static std::mutex mu;
    static std::map<long long, int> cache;
    const long long key = ((long long)nblk << 20) | ((long long)b << 4) | rounds;
    std::lock_guard<std::mutex> lock(mu);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const int P = cluster_ctas(G.nsup);
    const size_t smem = cluster_smem(nblk, b, P);
    const bool ok = smem <= CL_SMEM_MAX && cluster_fits(P, smem);
    cache[key] = ok ? P : 0;
    return ok ? P : 0;
}

size_t recur_cluster_scratch_bytes(int64_t nblk, int b)
{
    if (b % 4 != 0 || b > 32) return 0;
    const ClGeom G = cl_geom((int)nblk, b);
    if (G.nsup > CL_NSUP_MAX) return 0;
    return 2 * (size_t)G.nsup * 1024 * 4 + (size_t)G.nsup * CL_NSUP_MAX * 32 * 4 + (size_t)nblk * b * 4;
}

// The two halves of launch_recur_cluster: the prep kernel (inverses,
// couplings, repeat masks, links; it needs only Kss and S, so a step's prep
// may run ahead of the previous step's chain) and the chain.
cudaError_t launch_recur_cluster_prep(const float *Kss, int64_t ldk, const int32_t *S, int nblk, int b, double lambda,
                                      double mdiag, void *scratch, int *err, cudaStream_t st)
{
    const ClGeom G = cl_geom(nblk, b);
    if (((uintptr_t)scratch & 15) != 0) return cudaErrorInvalidValue;
    float *X = (float *)scratch;
    float *N = X + (size_t)G.nsup * 1024;
    uint32_t *M = (uint32_t *)(N + (size_t)G.nsup * 1024);
    int32_t *next = (int32_t *)(M + (size_t)G.nsup * CL_NSUP_MAX * 32);
    bdcd_prep_kernel<<<(unsigned)(2 * G.nsup), PREP_THREADS, 0, st>>>(Kss, ldk, S, nblk, b, (float)(1.0 / lambda),
                                                                     (float)mdiag, X, N, M, next, err);
    return cudaGetLastError();
}

cudaError_t launch_recur_cluster_chain(const float *Kss, int64_t ldk, const int32_t *S, int nblk, int b, int P,
                                       double lambda, double mdiag, double *g, int rounds, void *scratch,
                                       double *delta, double *w64, float *w32, const FusedUpdate *upd, int *err,
                                       cudaStream_t st, const double *rhs, int trig_sup, bool rhs_add_g, int prio)
{
    const ClGeom G = cl_geom(nblk, b);
    const int sb = nblk * b;
    if ((ldk * 4) % 16 != 0 || ((uintptr_t)Kss & 15) != 0 || ((uintptr_t)scratch & 15) != 0)
        return cudaErrorInvalidValue;
    float *X = (float *)scratch;
    float *N = X + (size_t)G.nsup * 1024;
    uint32_t *M = (uint32_t *)(N + (size_t)G.nsup * 1024);
    int32_t *next = (int32_t *)(M + (size_t)G.nsup * CL_NSUP_MAX * 32);
    CUtensorMap kmap;
    if (!make_map_f32_2d(&kmap, Kss, sb, sb, ldk, G.Bs, G.Bs)) return cudaErrorInvalidValue;
    auto kfn = bdcd_cluster_kernel;
    static bool attr = false;
    cudaError_t e;
    if (!attr) {
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CL_SMEM_MAX);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)P, 1, 1);
    cfg.blockDim = dim3(CL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = cluster_smem(nblk, b, P);
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)P;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributePriority;
    at[1].val.priority = prio;
    cfg.attrs = at;
    cfg.numAttrs = prio ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, kfn, kmap, S, (const float *)X, (const float *)N, (const uint32_t *)M,
                              (const int32_t *)next, nblk, b, lambda, mdiag, g, rounds, delta, w64, w32,
                              upd ? upd->alpha : (double *)nullptr, upd ? upd->ctr : (uint64_t *)nullptr,
                              upd ? upd->ctr_advance : (uint64_t)0, rhs, rhs_add_g ? 1 : 0, trig_sup, err);
}

cudaError_t launch_recur_cluster(const float *Kss, int64_t ldk, const int32_t *S, int nblk, int b, int P,
                                 double lambda, double mdiag, double *g, int rounds, void *scratch, double *delta,
                                 double *w64, float *w32, const FusedUpdate *upd, int *err, cudaStream_t st,
                                 const double *rhs)
{
    cudaError_t e = launch_recur_cluster_prep(Kss, ldk, S, nblk, b, lambda, mdiag, scratch, err, st);
    if (e != cudaSuccess) return e;
    return launch_recur_cluster_chain(Kss, ldk, S, nblk, b, P, lambda, mdiag, g, rounds, scratch, delta, w64, w32, upd,
                                      err, st, rhs);
}

// The largest diagonal panel (in blocks) one cluster launch solves: the
// blocked recurrence for longer chains runs panels of this size.
int recur_cluster_panel_blocks(int b, int rounds)
{
    if (b % 4 != 0 || b > 32) return 0;
    const int q = cl_geom(1, b).q;
    for (int nsup = CL_NSUP_MAX; nsup >= 2; nsup -= 2)
        if (recur_cluster_size(nsup * q, b, rounds) > 0) return nsup * q;
    return 0;
}

}  // namespace dcd
