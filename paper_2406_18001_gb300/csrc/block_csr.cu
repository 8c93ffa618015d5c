// block_csr.cu -- the sampled kernel block for a CSR data matrix.
//
// With A sparse (config: 50 nonzeros in 50000 columns per row), the block
// K(A, A_S) is an SpMM: a_i . a_j for every row i and every sampled row j,
// then the kernel function (Table 1; RBF via ||a||^2 + ||b||^2 - 2 a.b with
// precomputed squared row norms).  The work is bound by streaming A's CSR
// arrays from HBM once per outer step, not by arithmetic, so it runs on the
// CUDA cores (no tensor-core reshaping):
//
//   colmap   once per step, one CTA: the columns touched by the sampled rows
//            as a bitmap over [0, n) with per-word popcount prefixes (rank of
//            a column = its slot), and per slot the (j, value) entries of the
//            sampled rows holding that column.
//   block    one warp per tile of 32 rows: the tile's column indices are
//            read once, coalesced (values only for hits); an index whose
//            column is in the bitmap (rare) is a hit, appended in element order
//            to a per-warp list; then lane r adds value * entry for its row's
//            hits into a per-row row of accumulators (so the partial dots are
//            summed in a fixed order) and marks the touched sampled columns;
//            apply: g_i += rs_i (base_i + sum over touched j of w_j (K_ij -
//            K0_ij)), FP64 add (see csr_block_kernel); store: K_ij.
//
// Sampled columns are processed in chunks of CSR_JC per launch (a tile
// re-reads its nonzeros per chunk); the K-SVM configuration has s*b <= 32.
#include "dcd_internal.cuh"

namespace dcd {

namespace {

constexpr int CSR_JC = 32;        // sampled columns per apply pass
constexpr int CSR_WARPS = 8;      // warps per CTA
constexpr int CSR_GJ = 256;       // sampled columns per Gram pass
constexpr int MAP_THREADS = 1024;

// A product rounded on its own (never contracted into an FMA with the sum it
// joins), so that every route to a dot product adds the same rounded terms.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <typename T>
__device__ __forceinline__ T kfun_t(const KernelParams &kp, T dot, T na, T nb, bool same)
{
    if (kp.kind == DCD_LINEAR) return dot;
    if (kp.kind == DCD_POLY) {
        T t = (T)kp.coef0 + dot, r = t;
        for (int e = 1; e < kp.degree; ++e) r *= t;
        return r;
    }
    T d2 = same ? (T)0 : na + nb - (T)2 * dot;  // the sample's own row: distance exactly 0
    d2 = d2 > (T)0 ? d2 : (T)0;
    return exp(-(T)kp.gamma * d2);
}

// Apply: the block is never formed.  For row i, K(a_i, a_{S_j}) differs from
// its value at a_i . a_{S_j} = 0 only for the sampled rows j sharing a column
// with a_i ("hits", a few per row), so
//   sum_j w_j K_ij = base_i + sum_{j touched by i} w_j (K_ij - K0_ij),
// with K0_ij the kernel at a zero dot: c^d for the polynomial (base_i =
// c^d sum_j w_j), 0 for the linear kernel, exp(-gamma ||a_i||^2) exp(-gamma
// ||a_j||^2) for the RBF (base_i = exp(-gamma ||a_i||^2) sum_j w_j
// exp(-gamma ||a_j||^2)).  The stream over A is therefore its column indices
// only; a nonzero's value is read when its column is in the map.
constexpr int CSR_AW = 8;      // warps per CTA (apply)
constexpr int CSR_HL = 128;    // hit-list capacity per warp (applied when it could overflow)
constexpr int CSR_PF = 4;      // 128-index chunks per prefetch group (two groups in flight)

template <typename T>
struct alignas(16) WarpSmem {
    T acc[32][CSR_JC + 1];
    int32_t hoff[CSR_HL];  // element offset from the tile's first nonzero, ascending
    int32_t hcol[CSR_HL];  // its column
    int32_t hj[CSR_HL];    // resolved: the slot's entry column j - j0 (single entry), -1 (outside
                           // this column chunk), or -2 - slot (several entries)
    T hprod[CSR_HL];       // resolved: value * entry value (single entry) or the value
    int32_t rp[33];        // row offsets relative to the tile's first nonzero
};

constexpr int CSR_SMEM_BITS = 4096;  // bitmap words kept in shared memory (n <= 131072)

template <typename T>
struct alignas(16) CtaSmem {
    T nb[CSR_JC], w[CSR_JC], k0[CSR_JC];  // k0: RBF exp(-gamma ||a_j||^2)
    int32_t sj[CSR_JC];
    T base;                               // poly: c^d sum w; RBF: sum w_j k0_j
    uint32_t bits[CSR_SMEM_BITS];
};

__device__ __forceinline__ bool col_hit(const uint32_t *bits, int32_t c)
{
    return (__ldg(bits + (c >> 5)) >> (c & 31)) & 1u;
}

__device__ __forceinline__ int32_t col_slot(const uint32_t *bits, const int32_t *wprefix, int32_t c)
{
    const uint32_t w = __ldg(bits + (c >> 5));
    return __ldg(wprefix + (c >> 5)) + __popc(w & ((1u << (c & 31)) - 1u));
}

// Applies the warp's listed hits.  First the lanes resolve the hits in
// parallel (value, slot, and for a slot with one entry -- nearly all -- the
// product with that entry); then lane r adds its row's hits (offsets in
// [rp[r], rp[r+1]), a contiguous run of the ascending list found by binary
// search) into acc[r][.] in list order and marks the touched columns.
template <typename T>
__device__ __forceinline__ void flush_hits(WarpSmem<T> &ws, int nh, const CsrColMap &M, const uint32_t *bits,
                                           const T *vals, int64_t e0, int j0, int jc, int lane, int nr,
                                           uint32_t &touched)
{
    __syncwarp();
    for (int h = lane; h < nh; h += 32) {
        const int32_t c = ws.hcol[h];
        const T v = vals[e0 + ws.hoff[h]];
        const int slot = __ldg(M.wprefix + (c >> 5)) + __popc(bits[c >> 5] & ((1u << (c & 31)) - 1u));
        const int q0 = M.slot_off[slot], q1 = M.slot_off[slot + 1];
        if (q1 - q0 == 1) {
            const int j = M.ent_j[q0] - j0;
            ws.hj[h] = j >= 0 && j < jc ? j : -1;
            ws.hprod[h] = mul_rn(v, (T)M.ent_v[q0]);
        } else {
            ws.hj[h] = -2 - slot;
            ws.hprod[h] = v;
        }
    }
    __syncwarp();
    if (lane < nr) {
        const int lo = ws.rp[lane], hi = ws.rp[lane + 1];
        int a = 0, b = nh;
        while (a < b) {
            const int mid = (a + b) >> 1;
            if (ws.hoff[mid] < lo) a = mid + 1;
            else b = mid;
        }
        for (int h = a; h < nh && ws.hoff[h] < hi; ++h) {
            const int jj = ws.hj[h];
            if (jj >= 0) {
                ws.acc[lane][jj] += ws.hprod[h];
                touched |= 1u << jj;
            } else if (jj <= -2) {
                const int slot = -2 - jj;
                const T v = ws.hprod[h];
                for (int q = M.slot_off[slot]; q < M.slot_off[slot + 1]; ++q) {
                    const int j = M.ent_j[q] - j0;
                    if (j >= 0 && j < jc) {
                        ws.acc[lane][j] += mul_rn(v, (T)M.ent_v[q]);
                        touched |= 1u << j;
                    }
                }
            }
        }
    }
    __syncwarp();
}

// four consecutive column indices from element e (-1 past the array): one
// vector load when the quad lies inside the array and it is 16-byte aligned
__device__ __forceinline__ int4 load_cols(const CsrOperand &A, int64_t e)
{
    if (A.vec && e >= 0 && e + 4 <= A.nnz) return __ldg((const int4 *)(A.col_idx + e));
    int4 c;
    c.x = e >= 0 && e < A.nnz ? __ldg(A.col_idx + e) : -1;
    c.y = e + 1 >= 0 && e + 1 < A.nnz ? __ldg(A.col_idx + e + 1) : -1;
    c.z = e + 2 >= 0 && e + 2 < A.nnz ? __ldg(A.col_idx + e + 2) : -1;
    c.w = e + 3 >= 0 && e + 3 < A.nnz ? __ldg(A.col_idx + e + 3) : -1;
    return c;
}

// Kernel function of Table 1, the kind fixed at compile time.
template <typename T, int KIND>
__device__ __forceinline__ T kfun_k(T dot, T na, T nb, bool same, T gamma, T coef0, int degree)
{
    if (KIND == DCD_LINEAR) return dot;
    if (KIND == DCD_POLY) {
        const T t = coef0 + dot;
        T r = t;
        for (int e = 1; e < degree; ++e) r *= t;
        return r;
    }
    T d2 = same ? (T)0 : na + nb - (T)2 * dot;  // the sample's own row: distance exactly 0
    d2 = d2 > (T)0 ? d2 : (T)0;
    return exp(-gamma * d2);
}

// CTA set-up of an apply launch (every thread): the chunk's sampled ids,
// norms, RBF factors and coefficients, the bitmap (shared memory when it
// fits), zeroed accumulators and the base term's column sum (thread 0, in
// column order).
template <typename T, int KIND, bool SBITS>
__device__ __forceinline__ void csr_cta_setup(CtaSmem<T> &cs, WarpSmem<T> &ws, const CsrOperand &A,
                                              const CsrColMap &M, const int32_t *S, int j0, int jc,
                                              const KernelParams &kp, const float *w32, const double *w64)
{
    const int lane = threadIdx.x & 31;
    const T *norm = (const T *)(sizeof(T) == 8 ? (const void *)A.norm64 : (const void *)A.norm32);
    const T gamma = (T)kp.gamma, coef0 = (T)kp.coef0;
    for (int j = threadIdx.x; j < jc; j += blockDim.x) {
        const int32_t sj = S[j0 + j];
        cs.sj[j] = sj;
        cs.nb[j] = KIND == DCD_RBF ? norm[sj] : (T)0;
        cs.k0[j] = KIND == DCD_RBF ? exp(-gamma * cs.nb[j]) : (T)0;
        cs.w[j] = sizeof(T) == 8 ? (T)w64[j0 + j] : (T)w32[j0 + j];
    }
    if (SBITS)
        for (int w = threadIdx.x; w < M.nw; w += blockDim.x) cs.bits[w] = M.bits[w];
    for (int j = 0; j < CSR_JC; ++j) ws.acc[lane][j] = (T)0;
    __syncthreads();
    if (threadIdx.x == 0) {  // the base term's column sum, in column order
        T sw = (T)0;
        for (int j = 0; j < jc; ++j) sw += KIND == DCD_RBF ? cs.w[j] * cs.k0[j] : cs.w[j];
        if (KIND == DCD_POLY) {
            T cd = coef0;
            for (int e = 1; e < kp.degree; ++e) cd *= coef0;
            sw *= cd;
        }
        cs.base = KIND == DCD_LINEAR ? (T)0 : sw;
    }
    __syncthreads();
}

// The full pass over one tile of 32 rows starting at element e0 (n_e
// elements): the tile's column indices are streamed as int4 quads (lane l:
// indices 4 l .. 4 l + 3 of a 128-index chunk), the next group of CSR_PF
// chunks loaded while the current one is tested against the column bitmap;
// hits are listed in element order (warp prefix sum of the per-lane counts)
// as offsets and columns, and flush_hits adds them into the row accumulators.
template <typename T, bool SBITS>
__device__ __forceinline__ void csr_tile_stream(const CsrOperand &A, const CsrColMap &M, WarpSmem<T> &ws,
                                                const uint32_t *bits, const T *vals, int64_t e0, int n_e, int j0,
                                                int jc, int lane, int nr, uint32_t &touched)
{
    const int lead = (int)(e0 & 3);  // quad-aligned start; offsets -3 .. -1 lie before the tile
    int nh = 0;
    int4 cur[CSR_PF], nxt[CSR_PF];
#pragma unroll
    for (int b = 0; b < CSR_PF; ++b)
        cur[b] = -lead + 128 * b < n_e ? load_cols(A, e0 - lead + 128 * b + 4 * lane) : make_int4(-1, -1, -1, -1);
    for (int ob = -lead; ob < n_e; ob += 128 * CSR_PF) {
        const int obn = ob + 128 * CSR_PF;
#pragma unroll
        for (int b = 0; b < CSR_PF; ++b)  // the next group, in flight while this one is tested
            nxt[b] = obn + 128 * b < n_e ? load_cols(A, e0 + obn + 128 * b + 4 * lane) : make_int4(-1, -1, -1, -1);
#pragma unroll
        for (int b = 0; b < CSR_PF; ++b) {
            const int oq = ob + 128 * b + 4 * lane;  // offset of this lane's quad
            const int32_t cc[4] = {cur[b].x, cur[b].y, cur[b].z, cur[b].w};
            unsigned mk = 0;
            if (ob + 128 * b >= 0 && ob + 128 * b + 128 <= n_e) {  // warp-uniform: the chunk lies in the tile
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t wd = SBITS ? bits[cc[q] >> 5] : __ldg(bits + (cc[q] >> 5));
                    mk |= ((wd >> (cc[q] & 31)) & 1u) << q;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const bool in = oq + q >= 0 && oq + q < n_e && cc[q] >= 0;
                    if (in && ((SBITS ? bits[cc[q] >> 5] : __ldg(bits + (cc[q] >> 5))) >> (cc[q] & 31)) & 1u)
                        mk |= 1u << q;
                }
            }
            if (!__any_sync(0xffffffffu, mk != 0)) continue;
            // exclusive prefix of the per-lane hit counts = element order
            const int cnt = __popc(mk);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            if (nh + total > CSR_HL) {
                flush_hits(ws, nh, M, bits, vals, e0, j0, jc, lane, nr, touched);
                nh = 0;
            }
            int pos = nh + incl - cnt;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if ((mk >> q) & 1u) {
                    ws.hoff[pos] = oq + q;
                    ws.hcol[pos] = cc[q];
                    ++pos;
                }
            nh += total;
        }
#pragma unroll
        for (int b = 0; b < CSR_PF; ++b) cur[b] = nxt[b];
    }
    flush_hits(ws, nh, M, bits, vals, e0, j0, jc, lane, nr, touched);
}

// Lane r's row t0 + r: the base term plus, over the touched columns in
// ascending j, w_j (K_ij - K0_ij) (one FMA each); the accumulators return to
// zero; g += rs * sum in FP64.
template <typename T, int KIND>
__device__ __forceinline__ void csr_row_finish(WarpSmem<T> &ws, const CtaSmem<T> &cs, const CsrOperand &A,
                                               const KernelParams &kp, int64_t t0, int lane, int nr,
                                               uint32_t touched, const double *rs, double *g)
{
    const T *norm = (const T *)(sizeof(T) == 8 ? (const void *)A.norm64 : (const void *)A.norm32);
    const T gamma = (T)kp.gamma, coef0 = (T)kp.coef0;
    const T cd = KIND == DCD_POLY ? kfun_k<T, KIND>((T)0, (T)0, (T)0, false, gamma, coef0, kp.degree) : (T)0;
    const int64_t row = t0 + lane;
    if (lane < nr) {
        const T na = KIND == DCD_RBF ? norm[row] : (T)0;
        const T ea = KIND == DCD_RBF ? exp(-gamma * na) : (T)0;
        T sum = KIND == DCD_RBF ? ea * cs.base : cs.base;
        while (touched) {
            const int j = __ffs(touched) - 1;
            touched &= touched - 1;
            const T kv = kfun_k<T, KIND>(ws.acc[lane][j], na, cs.nb[j], cs.sj[j] == row, gamma, coef0, kp.degree);
            const T k0 = KIND == DCD_RBF ? ea * cs.k0[j] : cd;
            ws.acc[lane][j] = (T)0;
            sum = fma(cs.w[j], kv - k0, sum);
        }
        g[row] += (rs ? rs[row] : 1.0) * (double)sum;
    }
    __syncwarp();
}

// Apply, full pass: one warp per tile of 32 consecutive rows, the tile's row
// offsets for the next tile loaded while this one is streamed.
template <typename T, int KIND, bool SBITS>
__global__ void __launch_bounds__(CSR_AW * 32, 3)
    csr_block_kernel(CsrOperand A, CsrColMap M, int64_t nrows, const int32_t *S, int j0, int jc, KernelParams kp,
                     const float *w32, const double *w64, const double *rs, double *g)
{
    extern __shared__ __align__(16) unsigned char csr_sm[];
    CtaSmem<T> &cs = *(CtaSmem<T> *)csr_sm;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<T> &ws = ((WarpSmem<T> *)(csr_sm + sizeof(CtaSmem<T>)))[warp];
    const T *vals = (const T *)(sizeof(T) == 8 ? (const void *)A.vals64 : (const void *)A.vals32);
    csr_cta_setup<T, KIND, SBITS>(cs, ws, A, M, S, j0, jc, kp, w32, w64);
    const uint32_t *bits = SBITS ? cs.bits : M.bits;
    const int64_t ntiles = (nrows + 31) / 32;
    const int64_t tstride = (int64_t)gridDim.x * CSR_AW;
    // row offsets of a tile: lane r holds row_ptr[t0 + r], every lane row_ptr[t0 + nr]; the next
    // tile's are loaded while this one is streamed
    auto load_rp = [&](int64_t tl, int64_t &rv, int64_t &re) {
        if (tl < ntiles) {
            const int64_t t0 = tl * 32;
            const int nr = (int)min((int64_t)32, nrows - t0);
            rv = lane < nr ? A.row_ptr[t0 + lane] : 0;
            re = A.row_ptr[t0 + nr];
        }
    };
    int64_t rpv_n = 0, rend_n = 0;
    load_rp((int64_t)blockIdx.x * CSR_AW + warp, rpv_n, rend_n);
    for (int64_t tile = (int64_t)blockIdx.x * CSR_AW + warp; tile < ntiles; tile += tstride) {
        const int64_t t0 = tile * 32;
        const int nr = (int)min((int64_t)32, nrows - t0);
        const int64_t rpv = rpv_n, rend = rend_n;
        load_rp(tile + tstride, rpv_n, rend_n);
        const int64_t e0 = __shfl_sync(0xffffffffu, rpv, 0);
        if (lane < nr) ws.rp[lane] = (int32_t)(rpv - e0);
        if (lane == 0) ws.rp[nr] = (int32_t)(rend - e0);
        uint32_t touched = 0;
        csr_tile_stream<T, SBITS>(A, M, ws, bits, vals, e0, (int)(rend - e0), j0, jc, lane, nr, touched);
        csr_row_finish<T, KIND>(ws, cs, A, kp, t0, lane, nr, touched, rs, g);
    }
}

// ---------------------------------------------------------------------------
// Apply through the transposed matrix.  With a CSC copy of A, the nonzeros a
// step's kernel block actually needs -- a_ic with column c held by a sampled
// row j -- are found by walking the sampled rows' columns: about
// sum_j sum_{c in S_j} nnz(column c) "incidences" (i, element e, j), against
// every nonzero of A for the full pass.  Per 32-column chunk:
//   scatter  a CTA per (sampled row j, group of CSC_G of its nonzeros): the
//            group's columns, values and column ranges go to shared memory
//            with their prefix sums, then the CTA's threads sweep the group's
//            incidences as one flat range (CSC_U independent loads and
//            atomics per thread in flight) and append key = (e << 10) | (i mod
//            32) << 5 | j and the product a_ie * a_{S_j},c to the bucket of
//            the incidence's 32-row tile (a fixed capacity per tile; a counter
//            per tile, in arbitrary order);
//   apply    a warp per tile (the next tile's bucket loaded while this one
//            is processed) counting-sorts its incidences by row (shared
//            memory atomics), then lane r insertion-sorts its row's few
//            entries by key -- or, when some row holds more than
//            CSC_SHORT_ROW (a sampled row meets itself in all its columns),
//            the warp ranks every key of the tile jointly -- so the products
//            for each j come in element order, the order of the full pass,
//            and forms the row's sum exactly as the full pass does.  A tile
//            whose bucket overflowed runs the full pass over its rows.
// The result is bit-identical to the full pass.
constexpr int CSC_TILE_CAP = 128;  // incidences per 32-row tile (bucket size, sorted in shared memory)
constexpr int CSC_G = 4;           // sampled-row nonzeros per scatter CTA
constexpr int CSC_U = 4;           // incidences per scatter thread in flight
constexpr int CSC_SCATTER_THREADS = 256;

constexpr int CSC_SHORT_ROW = 8;   // a row with more entries in a tile makes the warp sort the tile jointly

template <typename T>
struct alignas(16) CscWarpSmem {
    int64_t skey[CSC_TILE_CAP], rkey[CSC_TILE_CAP];
    T sprod[CSC_TILE_CAP], rprod[CSC_TILE_CAP];
    int32_t rcnt[32], roff[32];
};

template <typename T>
__global__ void __launch_bounds__(CSC_SCATTER_THREADS)
    csc_scatter_kernel(CscOperand C, CsrColMap M, int j0, CscStep W)
{
    __shared__ int64_t cstart[CSC_G];
    __shared__ int64_t pre[CSC_G + 1];
    __shared__ T aval[CSC_G];
    const int j = blockIdx.x, grp = blockIdx.y;
    const T *cval = (const T *)C.val;
    T *prod = (T *)W.prod;
    if (threadIdx.x < 32) {  // one warp: the group's pairs and the prefix of their column lengths
        const int lane = threadIdx.x;
        const int q = grp * CSC_G + lane;
        int64_t len = 0;
        if (lane < CSC_G && q < M.pmax) {
            const int64_t at = (int64_t)(j0 + j) * M.pmax + q;
            len = M.plen[at];
            cstart[lane] = M.pstart[at];
            aval[lane] = (T)M.pval[at];
        }
        int64_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane < CSC_G) pre[lane + 1] = incl;
        if (lane == 0) pre[0] = 0;
    }
    __syncthreads();
    const int64_t total = pre[CSC_G];
    for (int64_t x0 = threadIdx.x; x0 < total; x0 += (int64_t)blockDim.x * CSC_U) {
        int64_t k[CSC_U];
        int q[CSC_U];
        int32_t row[CSC_U];
        int pos[CSC_U];
#pragma unroll
        for (int u = 0; u < CSC_U; ++u) {  // the pair holding incidence x: pre[q] <= x < pre[q + 1]
            const int64_t x = x0 + (int64_t)u * blockDim.x;
            int qq = 0;
#pragma unroll
            for (int b = CSC_G / 2; b > 0; b >>= 1)
                if (qq + b < CSC_G && pre[qq + b] <= x) qq += b;
            q[u] = qq;
            k[u] = x < total ? cstart[qq] + (x - pre[qq]) : -1;
        }
#pragma unroll
        for (int u = 0; u < CSC_U; ++u) row[u] = k[u] >= 0 ? C.row[k[u]] : -1;
#pragma unroll
        for (int u = 0; u < CSC_U; ++u) pos[u] = row[u] >= 0 ? atomicAdd(W.tile_cnt + (row[u] >> 5), 1) : CSC_TILE_CAP;
#pragma unroll
        for (int u = 0; u < CSC_U; ++u)
            if (pos[u] < CSC_TILE_CAP) {
                const int64_t at = (int64_t)(row[u] >> 5) * CSC_TILE_CAP + pos[u];
                W.key[at] = (C.elem[k[u]] << 10) | ((int64_t)(row[u] & 31) << 5) | j;
                prod[at] = mul_rn(cval[k[u]], aval[q[u]]);  // the full pass's product, rounded in T
            }
    }
}

template <typename T, int KIND>
__global__ void __launch_bounds__(CSR_AW * 32, 2)
    csc_apply_kernel(CsrOperand A, CsrColMap M, CscStep W, int64_t nrows, const int32_t *S, int j0, int jc,
                     KernelParams kp, const float *w32, const double *w64, const double *rs, double *g)
{
    extern __shared__ __align__(16) unsigned char csr_sm[];
    CtaSmem<T> &cs = *(CtaSmem<T> *)csr_sm;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<T> &ws = ((WarpSmem<T> *)(csr_sm + sizeof(CtaSmem<T>)))[warp];
    CscWarpSmem<T> &xs =
        ((CscWarpSmem<T> *)(csr_sm + sizeof(CtaSmem<T>) + sizeof(WarpSmem<T>) * CSR_AW))[warp];
    const T *vals = (const T *)(sizeof(T) == 8 ? (const void *)A.vals64 : (const void *)A.vals32);
    const T *prod = (const T *)W.prod;
    // the bitmap stays in global memory: only tiles that overflowed their bucket test it
    csr_cta_setup<T, KIND, false>(cs, ws, A, M, S, j0, jc, kp, w32, w64);
    const int64_t ntiles = (nrows + 31) / 32;
    const int64_t tstride = (int64_t)gridDim.x * CSR_AW;
    constexpr int PER = CSC_TILE_CAP / 32;
    // a tile's counter, row offsets and whole bucket (entries past the counter are stale and
    // masked later); the next tile's are loaded while this one is processed
    int nt_n = 0;
    int64_t rpv_n = 0, rend_n = 0;
    int64_t kk_n[PER];
    T pp_n[PER];
    auto load_tile = [&](int64_t tl) {
        if (tl >= ntiles) return;
        const int64_t t0 = tl * 32;
        const int nr = (int)min((int64_t)32, nrows - t0);
        nt_n = W.tile_cnt[tl];
        rpv_n = lane < nr ? A.row_ptr[t0 + lane] : 0;
        rend_n = A.row_ptr[t0 + nr];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            kk_n[u] = W.key[tl * CSC_TILE_CAP + lane + 32 * u];
            pp_n[u] = prod[tl * CSC_TILE_CAP + lane + 32 * u];
        }
    };
    load_tile((int64_t)blockIdx.x * CSR_AW + warp);
    for (int64_t tile = (int64_t)blockIdx.x * CSR_AW + warp; tile < ntiles; tile += tstride) {
        const int64_t t0 = tile * 32;
        const int nr = (int)min((int64_t)32, nrows - t0);
        const int nt = nt_n;
        const int64_t rpv = rpv_n, rend = rend_n;
        int64_t kk[PER];
        T pp[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            kk[u] = lane + 32 * u < nt ? kk_n[u] : -1;
            pp[u] = pp_n[u];
        }
        load_tile(tile + tstride);
        const int64_t e0 = __shfl_sync(0xffffffffu, rpv, 0);
        uint32_t touched = 0;
        if (nt > CSC_TILE_CAP) {  // the bucket overflowed: the full pass over this tile
            if (lane < nr) ws.rp[lane] = (int32_t)(rpv - e0);
            if (lane == 0) ws.rp[nr] = (int32_t)(rend - e0);
            csr_tile_stream<T, false>(A, M, ws, M.bits, vals, e0, (int)(rend - e0), j0, jc, lane, nr, touched);
        } else if (nt > 0) {
            // counting sort by row (the row's index within the tile is bits 5..9 of the key)
            xs.rcnt[lane] = 0;
            __syncwarp();
#pragma unroll
            for (int u = 0; u < PER; ++u)
                if (kk[u] >= 0) atomicAdd(&xs.rcnt[(int)(kk[u] >> 5) & 31], 1);
            __syncwarp();
            const int rc = xs.rcnt[lane];
            int incl = rc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            xs.roff[lane] = incl - rc;
            xs.rcnt[lane] = 0;
            __syncwarp();
#pragma unroll
            for (int u = 0; u < PER; ++u)
                if (kk[u] >= 0) {
                    const int rl = (int)(kk[u] >> 5) & 31;
                    const int at = xs.roff[rl] + atomicAdd(&xs.rcnt[rl], 1);
                    xs.skey[at] = kk[u];
                    xs.sprod[at] = pp[u];
                }
            __syncwarp();
            const int b0 = incl - rc, b1 = incl;
            const int64_t *sk = xs.skey;
            const T *sp = xs.sprod;
            if (__reduce_max_sync(0xffffffffu, (unsigned)rc) > (unsigned)CSC_SHORT_ROW) {
                // rank every key of the tile (keys are unique; the rank order groups the rows in
                // the order of the counting sort, so the row segments stay where they are)
#pragma unroll
                for (int u = 0; u < PER; ++u)
                    if (kk[u] >= 0) {
                        int r = 0;
                        for (int y = 0; y < nt; ++y) r += xs.skey[y] < kk[u] ? 1 : 0;
                        xs.rkey[r] = kk[u];
                        xs.rprod[r] = pp[u];
                    }
                __syncwarp();
                sk = xs.rkey;
                sp = xs.rprod;
            } else {
                for (int h = b0 + 1; h < b1; ++h) {  // lane r: its row's few entries by key
                    const int64_t kv = xs.skey[h];
                    const T pv = xs.sprod[h];
                    int q = h - 1;
                    while (q >= b0 && xs.skey[q] > kv) {
                        xs.skey[q + 1] = xs.skey[q];
                        xs.sprod[q + 1] = xs.sprod[q];
                        --q;
                    }
                    xs.skey[q + 1] = kv;
                    xs.sprod[q + 1] = pv;
                }
            }
            for (int h = b0; h < b1; ++h) {  // the products per j in element order
                const int j = (int)(sk[h] & 31);
                ws.acc[lane][j] += sp[h];
                touched |= 1u << j;
            }
            __syncwarp();
        }
        csr_row_finish<T, KIND>(ws, cs, A, kp, t0, lane, nr, touched, rs, g);
        if (lane == 0) W.tile_cnt[tile] = 0;  // the counter returns to zero for the next chunk
    }
}

// Store (the sampled Gram and the component block): one warp per listed row
// (rows == nullptr: row r), columns S[j0 .. j0 + jc).  The lanes resolve a
// group of 32 nonzeros' hits in parallel, then the hits are added one at a
// time in element order (a slot with several entries spreads its distinct j
// over the lanes), so every partial dot is summed in a fixed order -- the
// products and order of the apply kernel.
template <typename T>
__global__ void __launch_bounds__(CSR_WARPS * 32)
    csr_gram_kernel(CsrOperand A, CsrColMap M, const int32_t *rows, int64_t nrows, const int32_t *S, int j0, int jc,
                    KernelParams kp, float *out32, double *out64, int64_t ldo)
{
    __shared__ T acc[CSR_WARPS][CSR_GJ];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T *vals = (const T *)(sizeof(T) == 8 ? (const void *)A.vals64 : (const void *)A.vals32);
    const T *norm = (const T *)(sizeof(T) == 8 ? (const void *)A.norm64 : (const void *)A.norm32);
    for (int64_t k = (int64_t)blockIdx.x * CSR_WARPS + warp; k < nrows; k += (int64_t)gridDim.x * CSR_WARPS) {
        for (int j = lane; j < jc; j += 32) acc[warp][j] = (T)0;
        __syncwarp();
        const int64_t r = rows ? (int64_t)rows[k] : k;
        const int64_t e0 = A.row_ptr[r], e1 = A.row_ptr[r + 1];
        for (int64_t eb = e0; eb < e1; eb += 32) {
            // the lanes resolve their hits in parallel: value, slot, and for a slot with one entry
            // (nearly all) its column and the product
            const int64_t e = eb + lane;
            const int32_t c = e < e1 ? __ldg(A.col_idx + e) : -1;
            const bool hit = c >= 0 && col_hit(M.bits, c);
            int jj = -1;
            T prod = (T)0;
            if (hit) {
                const T v = vals[e];
                const int slot = col_slot(M.bits, M.wprefix, c);
                const int q0 = M.slot_off[slot], q1 = M.slot_off[slot + 1];
                if (q1 - q0 == 1) {
                    const int j = M.ent_j[q0] - j0;
                    jj = j >= 0 && j < jc ? j : -1;
                    prod = mul_rn(v, (T)M.ent_v[q0]);
                } else {
                    jj = -2 - slot;
                    prod = v;
                }
            }
            // then add them in element order
            unsigned mk = __ballot_sync(0xffffffffu, hit);
            while (mk) {
                const int src = __ffs(mk) - 1;
                mk &= mk - 1;
                const int js = __shfl_sync(0xffffffffu, jj, src);
                const T ps = __shfl_sync(0xffffffffu, prod, src);
                if (js >= 0) {
                    if (lane == 0) acc[warp][js] += ps;
                } else if (js <= -2) {  // several sampled rows hold this column: distinct j, one per lane
                    const int sl = -2 - js;
                    for (int q = M.slot_off[sl] + lane; q < M.slot_off[sl + 1]; q += 32) {
                        const int j = M.ent_j[q] - j0;
                        if (j >= 0 && j < jc) acc[warp][j] += mul_rn(ps, (T)M.ent_v[q]);
                    }
                }
                __syncwarp();
            }
        }
        const T na = kp.kind == DCD_RBF ? norm[r] : (T)0;
        for (int j = lane; j < jc; j += 32) {
            const int32_t sj = S[j0 + j];
            const T nb = kp.kind == DCD_RBF ? norm[sj] : (T)0;
            const T kv = kfun_t<T>(kp, acc[warp][j], na, nb, sj == r);
            if (sizeof(T) == 8) out64[k * ldo + j0 + j] = (double)kv;
            else out32[k * ldo + j0 + j] = (float)kv;
        }
        __syncwarp();
    }
}

// Exclusive scan of one value per thread over the CTA (warp shuffles, two
// barriers); *total receives the sum.
__device__ __forceinline__ int cta_excl_scan(int v, int *wsum, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int x = lane < nw ? wsum[lane] : 0, xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += t;
        }
        if (lane < nw) wsum[lane] = xi - x;  // exclusive warp offsets
        if (lane == 31) *total = xi;
    }
    __syncthreads();
    return wsum[warp] + incl - v;
}

// Column map of the sampled rows S[0..cnt) (one CTA).  Slots are the ranks of
// the touched columns; entries of a slot are (j, a_{S_j, c}).  The bitmap and
// the word prefixes are built in shared memory when they fit (SMAP) and
// copied out at the end.
constexpr int MAP_SMEM_WORDS = 8192;  // n <= 262144

template <bool SMAP>
__global__ void __launch_bounds__(MAP_THREADS) csr_colmap_kernel(CsrOperand A, const int32_t *S, int cnt, CsrColMap M,
                                                                 int *err)
{
    extern __shared__ uint32_t map_sm[];
    __shared__ int wsum[MAP_THREADS / 32];
    __shared__ int tot_slots, tot_ent;
    __shared__ long long total;
    uint32_t *bits = SMAP ? map_sm : M.bits;
    int32_t *wprefix = SMAP ? (int32_t *)(map_sm + M.nw) : M.wprefix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) total = 0;
    for (int w = tid; w < M.nw; w += MAP_THREADS) bits[w] = 0u;
    __syncthreads();
    // 0. the sampled rows' nonzeros must fit the entry capacity
    for (int j = tid; j < cnt; j += MAP_THREADS) {
        const int64_t r = S[j];
        if (r >= 0 && r < A.m) atomicAdd((unsigned long long *)&total, (unsigned long long)(A.row_ptr[r + 1] - A.row_ptr[r]));
    }
    __syncthreads();
    if (total > M.cap) {  // the same value in every thread
        if (tid == 0) set_error(err, DEV_INTERNAL);
        return;
    }
    // the transposed apply's pair table: per sampled position and nonzero slot, the column's CSC
    // range and the value
    if (M.plen)
        for (int j = warp; j < cnt; j += MAP_THREADS / 32) {
            const int64_t r = S[j];
            const bool ok = r >= 0 && r < A.m;
            const int64_t e0 = ok ? A.row_ptr[r] : 0, len = ok ? A.row_ptr[r + 1] - e0 : 0;
            for (int q = lane; q < M.pmax; q += 32) {
                const int64_t at = (int64_t)j * M.pmax + q;
                if (q < len) {
                    const int32_t c = A.col_idx[e0 + q];
                    const int64_t c0 = M.csc_col_ptr[c];
                    M.pstart[at] = c0;
                    M.plen[at] = (int32_t)(M.csc_col_ptr[c + 1] - c0);
                    M.pval[at] = A.vals64 ? A.vals64[e0 + q] : (double)A.vals32[e0 + q];
                } else {
                    M.plen[at] = 0;
                }
            }
        }
    // 1. mark the columns (warp per sampled row)
    for (int j = warp; j < cnt; j += MAP_THREADS / 32) {
        const int64_t r = S[j];
        if (r < 0 || r >= A.m) {
            if (lane == 0) set_error(err, DEV_BAD_INDEX);
            continue;
        }
        for (int64_t e = A.row_ptr[r] + lane; e < A.row_ptr[r + 1]; e += 32) {
            const int32_t c = A.col_idx[e];
            atomicOr(&bits[c >> 5], 1u << (c & 31));
        }
    }
    __syncthreads();
    // 2. exclusive popcount prefix over the words (contiguous chunk per thread)
    const int per = (M.nw + MAP_THREADS - 1) / MAP_THREADS;
    const int w0 = tid * per, w1 = min(M.nw, w0 + per);
    int s = 0;
    for (int w = w0; w < w1; ++w) s += __popc(bits[w]);
    int run = cta_excl_scan(s, wsum, &tot_slots);
    for (int w = w0; w < w1; ++w) {
        wprefix[w] = run;
        run += __popc(bits[w]);
    }
    __syncthreads();
    const int nslots = tot_slots;
    // 3. entries per slot (counts are zero on entry and return to zero below)
    for (int j = warp; j < cnt; j += MAP_THREADS / 32) {
        const int64_t r = S[j];
        if (r < 0 || r >= A.m) continue;
        for (int64_t e = A.row_ptr[r] + lane; e < A.row_ptr[r + 1]; e += 32) {
            const int32_t c = A.col_idx[e];
            const uint32_t w = bits[c >> 5];
            atomicAdd(&M.counts[wprefix[c >> 5] + __popc(w & ((1u << (c & 31)) - 1u))], 1);
        }
    }
    __syncthreads();
    // 4. slot offsets: exclusive scan of the counts
    const int sper = (nslots + MAP_THREADS - 1) / MAP_THREADS;
    const int s0 = tid * sper, s1 = min(nslots, s0 + sper);
    int cs = 0;
    for (int q = s0; q < s1; ++q) cs += M.counts[q];
    int run2 = cta_excl_scan(cs, wsum, &tot_ent);
    for (int q = s0; q < s1; ++q) {
        M.slot_off[q] = run2;
        run2 += M.counts[q];
    }
    if (tid == 0) M.slot_off[nslots] = tot_ent;
    __syncthreads();
    // 5. fill (taking the counts back to zero); the shared map goes out meanwhile
    if (SMAP)
        for (int w = tid; w < M.nw; w += MAP_THREADS) {
            M.bits[w] = bits[w];
            M.wprefix[w] = wprefix[w];
        }
    for (int j = warp; j < cnt; j += MAP_THREADS / 32) {
        const int64_t r = S[j];
        if (r < 0 || r >= A.m) continue;
        for (int64_t e = A.row_ptr[r] + lane; e < A.row_ptr[r + 1]; e += 32) {
            const int32_t c = A.col_idx[e];
            const uint32_t w = bits[c >> 5];
            const int slot = wprefix[c >> 5] + __popc(w & ((1u << (c & 31)) - 1u));
            const int pos = M.slot_off[slot] + atomicSub(&M.counts[slot], 1) - 1;
            M.ent_j[pos] = j;
            M.ent_v[pos] = A.vals64 ? A.vals64[e] : (double)A.vals32[e];
        }
    }
}

// squared row norms (FP32 and FP64), the longest row, and a validity check
// of the CSR arrays (bad counts the offending rows and entries)
__global__ void csr_prep_kernel(CsrOperand A, int *bad, int *maxlen)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= A.m) return;
    const int64_t e0 = A.row_ptr[r], e1 = A.row_ptr[r + 1];
    if (lane == 0 && (e1 < e0 || e0 < 0 || e1 > A.nnz)) atomicAdd(bad, 1);
    if (lane == 0 && e1 >= e0) atomicMax(maxlen, (int)min(e1 - e0, (int64_t)INT32_MAX));
    double s = 0.0;
    if (e1 >= e0 && e0 >= 0 && e1 <= A.nnz)
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int32_t c = A.col_idx[e];
            if (c < 0 || c >= A.n) atomicAdd(bad, 1);
            const double v = A.vals64 ? A.vals64[e] : (double)A.vals32[e];
            s += v * v;
        }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        if (A.norm64) A.norm64[r] = s;
        if (A.norm32) A.norm32[r] = (float)s;
    }
}

int sm_count()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    return sms;
}

template <typename T, int KIND, bool SBITS>
cudaError_t launch_csr_apply_k(const CsrOperand &A, const CsrColMap &M, int64_t nrows, const int32_t *S,
                               int64_t ncols, const KernelParams &kp, const float *w32, const double *w64,
                               const double *rs, double *g, cudaStream_t st)
{
    auto kfn = csr_block_kernel<T, KIND, SBITS>;
    const size_t smem = sizeof(CtaSmem<T>) + sizeof(WarpSmem<T>) * CSR_AW;
    static int per_sm = 0;  // resident CTAs per SM, queried once per instantiation (before any capture)
    if (!per_sm) {
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, CSR_AW * 32, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    const int64_t tiles = (nrows + 31) / 32;
    int64_t grid = (tiles + CSR_AW - 1) / CSR_AW;
    if (grid > (int64_t)sm_count() * per_sm) grid = (int64_t)sm_count() * per_sm;
    for (int64_t j0 = 0; j0 < ncols; j0 += CSR_JC) {
        const int jc = (int)min((int64_t)CSR_JC, ncols - j0);
        kfn<<<(unsigned)grid, CSR_AW * 32, smem, st>>>(A, M, nrows, S, (int)j0, jc, kp, w32, w64, rs, g);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_csr_apply(const CsrOperand &A, const CsrColMap &M, int64_t nrows, const int32_t *S, int64_t ncols,
                             const KernelParams &kp, const float *w32, const double *w64, const double *rs, double *g,
                             cudaStream_t st)
{
    const bool sb = M.nw <= CSR_SMEM_BITS;
#define CSR_K(KD)                                                                                    \
    return sb ? launch_csr_apply_k<T, KD, true>(A, M, nrows, S, ncols, kp, w32, w64, rs, g, st)     \
              : launch_csr_apply_k<T, KD, false>(A, M, nrows, S, ncols, kp, w32, w64, rs, g, st)
    if (kp.kind == DCD_RBF) CSR_K(DCD_RBF);
    if (kp.kind == DCD_POLY) CSR_K(DCD_POLY);
    CSR_K(DCD_LINEAR);
#undef CSR_K
}

template <typename T>
cudaError_t launch_csr_gram(const CsrOperand &A, const CsrColMap &M, const int32_t *rows, int64_t nrows,
                            const int32_t *S, int64_t ncols, const KernelParams &kp, float *out32, double *out64,
                            int64_t ldo, cudaStream_t st)
{
    int64_t grid = (nrows + CSR_WARPS - 1) / CSR_WARPS;
    if (grid > sm_count() * 8) grid = sm_count() * 8;
    for (int64_t j0 = 0; j0 < ncols; j0 += CSR_GJ) {
        const int jc = (int)min((int64_t)CSR_GJ, ncols - j0);
        csr_gram_kernel<T><<<(unsigned)grid, CSR_WARPS * 32, 0, st>>>(A, M, rows, nrows, S, (int)j0, jc, kp, out32,
                                                                       out64, ldo);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// CSC build (once per operand): entries per column, their exclusive scan, and
// the entries themselves (row, CSR element index, value) in arbitrary order
// within a column -- the apply sorts by element index.
__global__ void csc_colcount_kernel(CsrOperand A, int32_t *cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= A.m) return;
    for (int64_t e = A.row_ptr[r] + lane; e < A.row_ptr[r + 1]; e += 32) atomicAdd(cnt + A.col_idx[e], 1);
}

// One CTA: off[i] = sum_{q < i} cnt[q] for i <= count, *maxv = max cnt.
__global__ void __launch_bounds__(1024) excl_scan_kernel(const int32_t *cnt, int64_t count, int64_t *off, int *maxv)
{
    __shared__ int64_t wsum[32];
    __shared__ int64_t run_base;
    __shared__ int mx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        run_base = 0;
        mx = 0;
    }
    __syncthreads();
    int lmax = 0;
    for (int64_t b0 = 0; b0 < count; b0 += blockDim.x) {
        const int64_t t = b0 + threadIdx.x;
        const int64_t v = t < count ? (int64_t)cnt[t] : 0;
        lmax = max(lmax, (int)v);
        int64_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int64_t x = lane < nw ? wsum[lane] : 0, xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, xi, o);
                if (lane >= o) xi += u;
            }
            if (lane < nw) wsum[lane] = xi - x;
        }
        __syncthreads();
        const int64_t base = run_base;
        if (t < count) off[t] = base + wsum[warp] + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) run_base = base + wsum[warp] + incl;
        __syncthreads();
    }
    atomicMax(&mx, lmax);
    __syncthreads();
    if (threadIdx.x == 0) {
        off[count] = run_base;
        *maxv = mx;
    }
}

template <typename T>
__global__ void csc_fill_kernel(CsrOperand A, const int64_t *col_ptr, int32_t *cur, int32_t *row, int64_t *elem,
                                T *val)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= A.m) return;
    const T *vals = (const T *)(sizeof(T) == 8 ? (const void *)A.vals64 : (const void *)A.vals32);
    for (int64_t e = A.row_ptr[r] + lane; e < A.row_ptr[r + 1]; e += 32) {
        const int32_t c = A.col_idx[e];
        const int64_t pos = col_ptr[c] + atomicAdd(cur + c, 1);
        row[pos] = (int32_t)r;
        elem[pos] = e;
        val[pos] = vals[e];
    }
}

template <typename T>
cudaError_t launch_csc_scatter_chunk(const CsrColMap &M, const CscOperand &C, const CscStep &W, int maxrow,
                                     int64_t j0, int jc, cudaStream_t st)
{
    const unsigned groups = (unsigned)std::max(1, (maxrow + CSC_G - 1) / CSC_G);
    csc_scatter_kernel<T><<<dim3((unsigned)jc, groups), CSC_SCATTER_THREADS, 0, st>>>(C, M, (int)j0, W);
    return cudaGetLastError();
}

template <typename T, int KIND>
cudaError_t launch_csc_apply_k(const CsrOperand &A, const CsrColMap &M, const CscOperand &C, const CscStep &W,
                               int maxrow, const int32_t *S, int64_t ncols, const KernelParams &kp, const float *w32,
                               const double *w64, const double *rs, double *g, bool first_scattered, cudaStream_t st)
{
    auto kfn = csc_apply_kernel<T, KIND>;
    const size_t smem = sizeof(CtaSmem<T>) + (sizeof(WarpSmem<T>) + sizeof(CscWarpSmem<T>)) * CSR_AW;
    static int per_sm = 0;  // resident CTAs per SM, queried once per instantiation (before any capture)
    if (!per_sm) {
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, CSR_AW * 32, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    const int64_t ntiles = (A.m + 31) / 32;
    int64_t grid = (ntiles + CSR_AW - 1) / CSR_AW;
    if (grid > (int64_t)sm_count() * per_sm) grid = (int64_t)sm_count() * per_sm;
    for (int64_t j0 = 0; j0 < ncols; j0 += CSR_JC) {
        const int jc = (int)min((int64_t)CSR_JC, ncols - j0);
        if (j0 > 0 || !first_scattered) {
            const cudaError_t e = launch_csc_scatter_chunk<T>(M, C, W, maxrow, j0, jc, st);
            if (e != cudaSuccess) return e;
        }
        kfn<<<(unsigned)grid, CSR_AW * 32, smem, st>>>(A, M, W, A.m, S, (int)j0, jc, kp, w32, w64, rs, g);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_csc_apply(const CsrOperand &A, const CsrColMap &M, const CscOperand &C, const CscStep &W,
                             int maxrow, const int32_t *S, int64_t ncols, const KernelParams &kp, const float *w32,
                             const double *w64, const double *rs, double *g, bool first, cudaStream_t st)
{
    if (kp.kind == DCD_RBF)
        return launch_csc_apply_k<T, DCD_RBF>(A, M, C, W, maxrow, S, ncols, kp, w32, w64, rs, g, first, st);
    if (kp.kind == DCD_POLY)
        return launch_csc_apply_k<T, DCD_POLY>(A, M, C, W, maxrow, S, ncols, kp, w32, w64, rs, g, first, st);
    return launch_csc_apply_k<T, DCD_LINEAR>(A, M, C, W, maxrow, S, ncols, kp, w32, w64, rs, g, first, st);
}

}  // namespace

size_t csr_colmap_bytes(int64_t n, int64_t cap)
{
    const int64_t nw = (n + 31) / 32;
    return (size_t)nw * 8 + (size_t)(cap + 1) * 4 * 2 + (size_t)cap * (4 + 8) + 256 * 5;
}

CsrColMap csr_colmap_carve(void *base, int64_t n, int64_t cap)
{
    CsrColMap M;
    char *p = (char *)base;
    auto take = [&](size_t bytes) {
        char *r = p;
        p += (bytes + 255) / 256 * 256;
        return (void *)r;
    };
    M.nw = (int)((n + 31) / 32);
    M.cap = cap;
    M.bits = (uint32_t *)take((size_t)M.nw * 4);
    M.wprefix = (int32_t *)take((size_t)M.nw * 4);
    M.slot_off = (int32_t *)take((size_t)(cap + 1) * 4);
    M.counts = (int32_t *)take((size_t)(cap + 1) * 4);
    M.ent_j = (int32_t *)take((size_t)cap * 4);
    M.ent_v = (double *)take((size_t)cap * 8);
    return M;
}

cudaError_t launch_csr_prep(const CsrOperand &A, int *bad, int *maxlen, cudaStream_t st)
{
    if (A.m <= 0) return cudaSuccess;
    const int64_t blocks = (A.m * 32 + 255) / 256;
    csr_prep_kernel<<<(unsigned)blocks, 256, 0, st>>>(A, bad, maxlen);
    return cudaGetLastError();
}

cudaError_t launch_csr_colmap(const CsrOperand &A, const int32_t *S, int64_t cnt, const CsrColMap &M, int *err,
                              cudaStream_t st)
{
    if (cnt <= 0) return cudaSuccess;
    if (M.nw <= MAP_SMEM_WORDS) {
        const size_t smem = (size_t)M.nw * 8;
        static bool attr = false;
        if (!attr) {
            const cudaError_t e = cudaFuncSetAttribute(csr_colmap_kernel<true>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, MAP_SMEM_WORDS * 8);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        csr_colmap_kernel<true><<<1, MAP_THREADS, smem, st>>>(A, S, (int)cnt, M, err);
    } else {
        csr_colmap_kernel<false><<<1, MAP_THREADS, 0, st>>>(A, S, (int)cnt, M, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_csr_block(const CsrOperand &A, const CsrColMap &M, bool fp64, const KernelParams &kp,
                             const int32_t *rows, int64_t nrows, const int32_t *S, int64_t ncols, const float *w32,
                             const double *w64, const double *rs, double *g, void *out, int64_t ldo, cudaStream_t st)
{
    if (nrows <= 0 || ncols <= 0) return cudaSuccess;
    if (out) {
        return fp64 ? launch_csr_gram<double>(A, M, rows, nrows, S, ncols, kp, nullptr, (double *)out, ldo, st)
                    : launch_csr_gram<float>(A, M, rows, nrows, S, ncols, kp, (float *)out, nullptr, ldo, st);
    }
    if (rows) return cudaErrorInvalidValue;  // apply runs over rows 0 .. nrows-1
    CsrOperand Av = A;
    const void *vp = fp64 ? (const void *)A.vals64 : (const void *)A.vals32;
    Av.vec = ((uintptr_t)A.col_idx & 15) == 0 && ((uintptr_t)vp & 15) == 0;
    return fp64 ? launch_csr_apply<double>(Av, M, nrows, S, ncols, kp, w32, w64, rs, g, st)
                : launch_csr_apply<float>(Av, M, nrows, S, ncols, kp, w32, w64, rs, g, st);
}

namespace {
size_t take_bytes(char *&p, size_t bytes)
{
    const size_t a = (bytes + 255) / 256 * 256;
    p += a;
    return a;
}
}  // namespace

size_t csc_bytes(int64_t n, int64_t nnz, bool fp64)
{
    return (size_t)(n + 1) * 8 + (size_t)n * 4 + (size_t)nnz * (4 + 8 + (fp64 ? 8 : 4)) + 256 * 5;
}

cudaError_t launch_csc_build(const CsrOperand &A, bool fp64, void *base, CscOperand *C, int *maxcol_dev,
                             cudaStream_t st)
{
    char *p = (char *)base;
    int64_t *col_ptr = (int64_t *)p;
    take_bytes(p, (size_t)(A.n + 1) * 8);
    int32_t *cnt = (int32_t *)p;
    take_bytes(p, (size_t)A.n * 4);
    int32_t *row = (int32_t *)p;
    take_bytes(p, (size_t)A.nnz * 4);
    int64_t *elem = (int64_t *)p;
    take_bytes(p, (size_t)A.nnz * 8);
    void *val = p;
    C->col_ptr = col_ptr;
    C->row = row;
    C->elem = elem;
    C->val = val;
    C->n = A.n;
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)A.n * 4, st);
    if (e != cudaSuccess) return e;
    if (A.m > 0) {
        const unsigned blocks = (unsigned)((A.m * 32 + 255) / 256);
        csc_colcount_kernel<<<blocks, 256, 0, st>>>(A, cnt);
    }
    excl_scan_kernel<<<1, 1024, 0, st>>>(cnt, A.n, col_ptr, maxcol_dev);
    if ((e = cudaMemsetAsync(cnt, 0, (size_t)A.n * 4, st)) != cudaSuccess) return e;
    if (A.m > 0) {
        const unsigned blocks = (unsigned)((A.m * 32 + 255) / 256);
        if (fp64) csc_fill_kernel<double><<<blocks, 256, 0, st>>>(A, col_ptr, cnt, row, elem, (double *)val);
        else csc_fill_kernel<float><<<blocks, 256, 0, st>>>(A, col_ptr, cnt, row, elem, (float *)val);
    }
    return cudaGetLastError();
}

size_t csc_step_bytes(int64_t m, int64_t cnt, int maxrow, bool fp64)
{
    const int64_t ntiles = (m + 31) / 32, pairs = cnt * (int64_t)std::max(maxrow, 1);
    return (size_t)ntiles * 4 + (size_t)ntiles * CSC_TILE_CAP * (8 + (fp64 ? 8 : 4)) + (size_t)pairs * (8 + 4 + 8) +
           256 * 6;
}

CscStep csc_step_carve(void *base, int64_t m, int64_t cnt, int maxrow, const CscOperand &C, CsrColMap *M)
{
    const int64_t ntiles = (m + 31) / 32, pairs = cnt * (int64_t)std::max(maxrow, 1);
    char *p = (char *)base;
    CscStep W;
    W.tile_cnt = (int32_t *)p;
    take_bytes(p, (size_t)ntiles * 4);
    W.key = (int64_t *)p;
    take_bytes(p, (size_t)ntiles * CSC_TILE_CAP * 8);
    M->pstart = (int64_t *)p;
    take_bytes(p, (size_t)pairs * 8);
    M->pval = (double *)p;
    take_bytes(p, (size_t)pairs * 8);
    M->plen = (int32_t *)p;
    take_bytes(p, (size_t)pairs * 4);
    M->pmax = std::max(maxrow, 1);
    M->csc_col_ptr = C.col_ptr;
    W.prod = p;
    return W;
}

cudaError_t launch_csr_apply_csc(const CsrOperand &A, const CsrColMap &M, const CscOperand &C, const CscStep &W,
                                 bool fp64, int maxrow, const KernelParams &kp, const int32_t *S, int64_t ncols,
                                 const float *w32, const double *w64, const double *rs, double *g, cudaStream_t st,
                                 bool first_scattered)
{
    if (ncols <= 0 || A.m <= 0) return cudaSuccess;
    CsrOperand Av = A;
    const void *vp = fp64 ? (const void *)A.vals64 : (const void *)A.vals32;
    Av.vec = ((uintptr_t)A.col_idx & 15) == 0 && ((uintptr_t)vp & 15) == 0;
    return fp64 ? launch_csc_apply<double>(Av, M, C, W, maxrow, S, ncols, kp, w32, w64, rs, g, first_scattered, st)
                : launch_csc_apply<float>(Av, M, C, W, maxrow, S, ncols, kp, w32, w64, rs, g, first_scattered, st);
}

cudaError_t launch_csr_csc_scatter_first(const CsrColMap &M, const CscOperand &C, const CscStep &W, bool fp64,
                                         int maxrow, int64_t ncols, cudaStream_t st)
{
    if (ncols <= 0) return cudaSuccess;
    const int jc = (int)min((int64_t)CSR_JC, ncols);
    return fp64 ? launch_csc_scatter_chunk<double>(M, C, W, maxrow, 0, jc, st)
                : launch_csc_scatter_chunk<float>(M, C, W, maxrow, 0, jc, st);
}

}  // namespace dcd
