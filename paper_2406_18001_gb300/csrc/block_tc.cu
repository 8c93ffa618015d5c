// block_tc.cu -- the sampled kernel block on the sm_103a tensor cores.
//
// C[i, j] = a_i . b_j for a packed, zero-padded operand A (rows of the data
// matrix) and B (the s*b sampled rows), both K-major, is formed by
// tcgen05.mma (kind::f16 with bf16 inputs, kind::tf32 on fp32 inputs, or
// kind::f8f6f4 on per-row-scaled e4m3 codes) with FP32 accumulators in tensor
// memory.  The epilogue maps C through the kernel
// function of Table 1 -- the RBF via the expansion ||a||^2 + ||b||^2 - 2 a.b
// of Section 5.2 -- and either
//   apply: contracts each row with the column coefficients w and adds
//          rs[i] * sum_j K_ij w_j to the FP64 gradient g[i] (the m x sb block
//          is never written to memory), or
//   store: writes K_ij (FP32) -- used for the sampled Gram, so that the
//          recurrence sees exactly the values the apply pass uses.
// The apply form has a third, accurate epilogue (MODE_ACC, on the split-tf32
// operand) for recomputing the gradient from alpha: the RBF exponent in
// double-single arithmetic, exp2 by reduction to the nearest integer and a
// degree-7 Taylor polynomial, and the contraction with FP64 coefficients in
// double-single.  On the sliced operand (exact products) its kernel values
// are within ~1e-8 of the exact kernel of the data; the fast epilogue's carry
// the FP32-accumulated dot's ~1e-7 and the FP32 exponent's ~2.5e-7.
//
// Two kernels, both persistent with one CTA per SM and 320 threads:
//   block_tc_kernel  (store) over 128-row tiles x N-chunks of 64 columns
//                    (up to 256 when held to a few CTAs);
//   block_tc2_kernel (apply) on CTA pairs (tcgen05 cta_group::2) over
//                    (256-row tile, N-chunk) units, each CTA staging half of
//                    an N-chunk of B; the pairs take contiguous ranges of the
//                    units, a tile split between two pairs summed by the one
//                    that finishes it last (see pair_units).
// Warp roles in both:
//   warp 0      TMA producer: 128-byte-swizzled k-blocks of A and B into a
//               shared-memory ring (mbarrier complete_tx)
//   warp 1      TMEM allocator and MMA issuer (one thread); accumulators are
//               double-buffered (2 x BN columns) so the epilogue of one
//               N-chunk overlaps the MMAs of the next
//   warps 2..9  epilogue: tcgen05.ld 32 lanes x 32 columns per load, one
//               thread per row; warp w reads TMEM lanes 32 (w % 4)..+31, warps
//               2..5 take the first half of each N-chunk's columns and warps
//               6..9 the second half (two warps per scheduler hide the load and
//               MUFU latency); in the apply form the second half's row sums
//               reach the first half through shared memory once per tile, in a
//               fixed order; the apply's epilogue waits (griddepcontrol.wait)
//               for the grid before it, so that it may run as a programmatic
//               dependent whose products start early
// Every mbarrier wait is bounded; on timeout the CTA records DEV_TIMEOUT,
// drains its in-flight copies and MMAs (bounded), frees TMEM and returns.
#include "dcd_internal.cuh"
#include "ptx.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

namespace dcd {

namespace {

constexpr int BM = 128;                 // rows per tile = TMEM lanes
constexpr int BN_MAX = 256;             // columns per N-chunk (max)
constexpr int ROW_BYTES = 128;          // one swizzled k-block row
constexpr int A_STAGE = BM * ROW_BYTES;          // 16 KB
constexpr int B_STAGE = BN_MAX * ROW_BYTES;      // 32 KB
constexpr int RING_BYTES = 4 * (A_STAGE + B_STAGE);  // 4 single stages or 2 split stages

// Operand modes: bf16 (kind::f16), tf32 (kind::tf32 on fp32 storage), and
// split bf16 ("bf16x3": a = hi + lo with hi = bf16(a), lo = bf16(a - hi);
// a.b ~ hi.hi + hi.lo + lo.hi, three MMAs per k-step into one accumulator,
// dropping only lo.lo, about 2^-16 relative).
// Split tf32 ("tf32x3") is the same with kind::tf32 and tf32 planes (~22
// significant bits, at half the bf16 MMA rate).
// fp16: kind::f16 on fp16 operands q, the matrix scaled by one power of two
// (a ~ s q, |q| < 2^15; 11 significant bits against bf16's 8), one MMA per
// k-step; the epilogue folds s^2 into its per-row factor (row_s[i] col_s[0]:
// every scale of an fp16 operand is the same number).
// fp8: e4m3 codes q with per-row scales (a_i ~ s_i q_i), kind::f8f6f4 with 32
// codes per MMA (so a 128-byte k-block is again 4 MMAs); the products
// q_i q_j are exact and the epilogue restores a_i.a_j = s_i s_j (q_i.q_j).
// MODE_ACC: the split-tf32 products with the accurate apply epilogue (pairs only).
// MODE_SLICED: sliced operands (4 planes of small integers, per-row powers of
// two); the 10 plane products with p + q <= 3 go into 4 accumulators by
// p + q, whose FP32 sums are exact integers; accurate epilogue (pairs only).
constexpr int MODE_BF16 = 0, MODE_TF32 = 1, MODE_BF16X3 = 2, MODE_TF32X3 = 3, MODE_FP8 = 4, MODE_ACC = 5,
              MODE_SLICED = 6, MODE_FP16 = 7;
constexpr int SLICED_BN = 128;  // N-chunk of the sliced apply: 4 accumulators fill the 512 TMEM columns
// The apply's fast RBF epilogue factors K_ij w_j = 2^(rf c - h_i) (w_j 2^(-h_j)) when every row and
// column term h = gamma log2(e) ||x||^2 of the launch's warp is at most this (both factors then stay
// well inside the FP32 range); otherwise it evaluates 2^(min(0, rf c - h_i - h_j)) w_j.
constexpr float RBF_FACTOR_HMAX = 64.f;
constexpr int XCH_BYTES = 2 * BM * 8;  // apply: row sums of the second epilogue half, double-buffered
// single-CTA kernel, per epilogue warp: the column terms of its half of an N-chunk (RBF term,
// id, fp8 scale: 3 x 128 words) and a 32 x 16 transpose tile (row stride 17) for the store form
constexpr int STG_WORDS = 3 * 128 + 32 * 17;
constexpr int SMEM_BYTES = RING_BYTES + 1024 /*alignment slack*/ + 256 /*barriers*/ + 8 * STG_WORDS * 4;
constexpr int NTHREADS = 320;
constexpr uint32_t TMEM_COLS = 512;
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s bound on any single wait

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity.  Returns false if the
// CTA is aborting (another role timed out) or this wait timed out.
// The bound counts SM clock cycles (clock64 is cheap; %globaltimer reads are
// not): WAIT_NS at an assumed 2.1 GHz.
constexpr long long WAIT_CYCLES = (long long)(WAIT_NS * 21 / 10);

__device__ __noinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *err)
{
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t spin = 1;; ++spin) {
        if (mbar_test(bar, parity)) return true;
        if ((spin & 15) == 0) {
            if (*abort_flag) return false;
            if (clock64() - t0 > WAIT_CYCLES) {
                *abort_flag = 1;
                set_error(err, DEV_TIMEOUT);
                return false;
            }
        }
    }
}

// Wait without the abort shortcut (drain path), still bounded.
__device__ __noinline__ void mbar_drain(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > WAIT_CYCLES) return;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            su32(dst)),
        "l"((uint64_t)map), "r"(su32(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), descriptor
// version 1, layout type 2 (SWIZZLE_128B).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: D = F32, A/B format (kind::f16: bf16 = 1;
// kind::tf32: tf32 = 2; kind::f8f6f4: e4m3 = 0), both K-major, N >> 3 at bit
// 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(int fmt, int n, int m)
{
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

// MK: 0 kind::f16, 1 kind::tf32, 2 kind::f8f6f4
template <int MK>
__device__ __forceinline__ void mma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    if (MK == 1)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtm),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    else if (MK == 2)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtm),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtm),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

// tcgen05.ld of 32 lanes x 32 columns, issued and waited for separately (the
// next group's load overlaps this group's arithmetic); the wait names the
// destination registers, so that no use of them is scheduled before it.
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// tcgen05.ld of 32 lanes x 16 columns, waited for at once
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    tmem_ld_wait(r);
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct TcArgs {
    int lo_off;           // split mode: column offset of the lo halves (= n_pad)
    const float *row_h;   // per-row RBF term gamma*log2(e)*||a_i||^2 (nrows_out entries)
    const float *col_h;   // per-column term, padded with zeros to nchunks*BN
    const float *col_w;   // apply: coefficients, padded with zeros
    const double *rs;     // apply: per-row scale or null
    const float *row_s;   // fp8, fp16: per-row scales of the A operand (nrows_out entries)
    const float *col_s;   // fp8, fp16: per-column scales, padded with zeros like col_h
    double *g;            // apply: gradient (nrows_out)
    float *out;           // store: output, row-major with ldo
    int64_t ldo;
    int64_t nrows_out;
    int64_t ncols;
    int num_tiles, nchunks, kblocks, bn;
    int store;            // 1: store epilogue, 0: apply
    int lower;            // store: skip the N-chunks above the diagonal
    int items;            // apply: num_tiles; store: num_tiles * nchunks
    int degree;
    float two_gl;         // 2 * gamma * log2(e)
    float coef0;
    int *err;
    double *part;         // apply on pairs: per-chunk row sums of the row tiles two pairs share (or null)
    unsigned *cnt;        // apply on pairs: arrivals per shared tile and CTA rank
    int late_pairs;       // apply on pairs: the last late_pairs pairs take late_units units fewer
    int late_units;
    // MODE_ACC: low parts of the RBF terms (h + h_lo), FP64 coefficients, 2 gamma log2(e) as hi + lo
    const float *row_hl;
    const float *col_hl;
    const double *col_w64;
    float two_gl_lo;
    // data-matrix row of each block row / column (null: the row / column number); RBF: K = 1
    // where they are equal (d^2 = 0 on a row's own sample)
    const int32_t *row_id;
    const int32_t *col_id;
    int dep_wait;         // apply: the epilogue waits for the grid before this one (griddepcontrol.wait)
};

// ------------------------------------------------- double-single helpers --
// Error-free transformations (Knuth's TwoSum, Dekker's Fast2Sum and the
// FMA product): s + e equals a + b (a * b) exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)  // |a| >= |b|
{
    s = a + b;
    e = b - (s - a);
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = a * b;
    e = fmaf(a, b, -p);
}

// 2^x for x <= 0 given as x_hi + x_lo (|x_lo| <= ulp(x_hi)), as a
// double-single kh + kl: x = k + f with k = rint(x_hi), |f| <= 1/2, and
// u = f ln 2 (double-single, ln 2 as hi + lo); e^u = 1 + u + u^2 T(u) with T
// the Taylor polynomial of degree 5 of (e^u - 1 - u) / u^2 (truncation below
// 5.3e-9 relative for |u| <= 0.35), the small u^2 T(u) in FP32 from u's high
// part, 1 + u + u^2 T(u) summed in double-single; then 2^k applied to the
// exponent fields.  Results below 2^-125 are returned as 0.
__device__ __forceinline__ void exp2_ds(float xh, float xl, float &kh, float &kl)
{
    if (xh < -125.f) {
        kh = 0.f;
        kl = 0.f;
        return;
    }
    const float k = rintf(xh);
    const float fh = xh - k;  // exact
    float uh, ul;
    two_prod(fh, 0x1.62e430p-1f, uh, ul);
    ul = fmaf(fh, 0x1.fdf474p-26f, fmaf(xl, 0x1.62e430p-1f, ul));
    float t = 1.f / 5040.f;
    t = fmaf(t, uh, 1.f / 720.f);
    t = fmaf(t, uh, 1.f / 120.f);
    t = fmaf(t, uh, 1.f / 24.f);
    t = fmaf(t, uh, 1.f / 6.f);
    t = fmaf(t, uh, 0.5f);
    const float tail = t * uh * uh;
    float sh, sl;
    fast_two_sum(1.f, uh, sh, sl);  // |uh| < 1
    sl += ul + tail;
    fast_two_sum(sh, sl, sh, sl);
    const float sc = __int_as_float(((int)k + 127) << 23);
    kh = sh * sc;
    kl = sl * sc;
}

// K(a_i, b_j) from the accumulator c; rf is the per-row factor: 2 gamma
// log2(e) (RBF) or 1 (poly, linear), times the row scale in the fp8 and fp16
// modes (where c already carries the column scale).
template <int KIND>
__device__ __forceinline__ float kf32(float c, float hr, float hc, float rf, const TcArgs &a)
{
    if (KIND == DCD_RBF) {
        float t = fmaf(c, rf, -(hr + hc));
        return ex2f(fminf(t, 0.f));
    } else if (KIND == DCD_LINEAR) {
        return c * rf;
    } else {
        float t = fmaf(c, rf, a.coef0), r = t;
        for (int e = 1; e < a.degree; ++e) r *= t;
        return r;
    }
}

// The accurate epilogue's kernel value (kh + kl) from a dot product given as
// dh + dl (double-single): the RBF exponent x = 2 gamma log2(e) (a.b) - (h_i
// + h_j) = -gamma log2(e) d^2 in double-single, clamped at 0, then exp2_ds;
// the polynomial by repeated double-single products; linear as it is.
template <int KIND>
__device__ __forceinline__ void k_accurate(float dh, float dl, float hr, float hrl, float hc, float hcl,
                                           const TcArgs &a, float &kh, float &kl)
{
    kl = 0.f;
    if (KIND == DCD_RBF) {
        float sh, sl, ph, pl, xh, xl;
        two_sum(hr, hc, sh, sl);
        sl += hrl + hcl;
        two_prod(a.two_gl, dh, ph, pl);
        pl = fmaf(a.two_gl, dl, fmaf(a.two_gl_lo, dh, pl));
        two_sum(ph, -sh, xh, xl);
        xl += pl - sl;
        fast_two_sum(xh, xl, xh, xl);
        if (xh > 0.f) {  // d^2 >= 0
            xh = 0.f;
            xl = 0.f;
        }
        exp2_ds(xh, xl, kh, kl);
    } else if (KIND == DCD_LINEAR) {
        kh = dh;
        kl = dl;
    } else {
        float th, tl;
        two_sum(a.coef0, dh, th, tl);
        tl += dl;
        fast_two_sum(th, tl, th, tl);
        float rh = th, rl = tl;
        for (int e = 1; e < a.degree; ++e) {
            float pp, pe;
            two_prod(rh, th, pp, pe);
            pe = fmaf(rh, tl, fmaf(rl, th, pe));
            fast_two_sum(pp, pe, rh, rl);
        }
        kh = rh;
        kl = rl;
    }
}

// store form: one item = one (row tile, N-chunk) pair; with `lower`, the
// chunks that start past the tile's last row are empty items (every role
// skips them alike)
// N-chunks of row tile t that reach the lower triangle (the store form's lower option)
__host__ __device__ __forceinline__ int lower_chunks(int t, int bn, int nchunks)
{
    const int64_t n = ((int64_t)t * BM + BM - 1) / bn + 1;
    return n < nchunks ? (int)n : nchunks;
}

// The single-CTA kernel's work item: one (row tile, N-chunk); with lower, only the chunks that
// reach the lower triangle are items, numbered tile by tile
__device__ __forceinline__ void item_range(const TcArgs &a, int item, int &tile, int &c0, int &c1)
{
    if (a.lower) {
        int t = 0, rem = item;
        for (int n = lower_chunks(0, a.bn, a.nchunks); rem >= n && t + 1 < a.num_tiles;
             n = lower_chunks(++t, a.bn, a.nchunks))
            rem -= n;
        tile = t;
        c0 = rem;
        c1 = c0 + 1;
        return;
    }
    tile = item / a.nchunks;
    c0 = item % a.nchunks;
    c1 = c0 + 1;
}

template <int MODE, int KIND>
__global__ void __launch_bounds__(NTHREADS, 1)
    block_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs a)
{
    constexpr bool TF32 = MODE == MODE_TF32 || MODE == MODE_TF32X3;
    constexpr bool FP8 = MODE == MODE_FP8;
    constexpr bool FP16 = MODE == MODE_FP16;
    constexpr bool SCALED = FP8 || FP16;  // operand scales restored in the epilogue
    constexpr int MK = TF32 ? 1 : FP8 ? 2 : 0;
    constexpr bool SPLIT = MODE == MODE_BF16X3 || MODE == MODE_TF32X3;
    constexpr int STAGES = SPLIT ? 2 : 4;
    constexpr int A_ST = SPLIT ? 2 * A_STAGE : A_STAGE;  // hi then lo
    constexpr int B_ST = SPLIT ? 2 * B_STAGE : B_STAGE;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * A_ST;
    uint64_t *bars = (uint64_t *)(smem + RING_BYTES);
    uint64_t *full = bars;                 // STAGES
    uint64_t *empty = bars + STAGES;       // STAGES
    uint64_t *tfull = bars + 2 * STAGES;   // 2
    uint64_t *tempty = tfull + 2;          // 2
    uint64_t *drain = tempty + 2;          // 1
    uint32_t *tmem_holder = (uint32_t *)(drain + 1);
    volatile int *abort_flag = (volatile int *)(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 8);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem_base = *tmem_holder;
    const int bn = a.bn;
    const int kb_elems = TF32 ? 32 : FP8 ? 128 : 64;  // elements per 128-byte k-block

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------- producer --
            uint32_t it = 0;
            bool ok = true;
            const uint32_t bytes = (uint32_t)((SPLIT ? 2 : 1) * (A_STAGE + bn * ROW_BYTES));
            for (int item = blockIdx.x; ok && item < a.items; item += gridDim.x) {
                int tile, c0, c1;
                item_range(a, item, tile, c0, c1);
                for (int nc = c0; ok && nc < c1; ++nc)
                    for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
                        const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
                        if (!mbar_wait(&empty[s], ph ^ 1, abort_flag, a.err)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(&full[s], bytes);
                        tma_load_2d(sA + s * A_ST, &tmA, &full[s], kb * kb_elems, tile * BM);
                        tma_load_2d(sB + s * B_ST, &tmB, &full[s], kb * kb_elems, nc * bn);
                        if (SPLIT) {
                            tma_load_2d(sA + s * A_ST + A_STAGE, &tmA, &full[s], a.lo_off + kb * kb_elems, tile * BM);
                            tma_load_2d(sB + s * B_ST + B_STAGE, &tmB, &full[s], a.lo_off + kb * kb_elems, nc * bn);
                        }
                    }
            }
            if (!ok) {  // let every issued copy land before the CTA exits
                uint32_t first = it > STAGES ? it - STAGES : 0;
                for (uint32_t j = first; j < it; ++j) mbar_drain(&full[j % STAGES], (j / STAGES) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // --------------------------------------------------------- MMA --
            const uint32_t idesc = make_idesc(TF32 ? 2 : SCALED ? 0 : 1, bn, BM);  // tf32, e4m3 / f16, bf16
            uint32_t it = 0, acc_it = 0;
            bool ok = true, issued = false;
            for (int item = blockIdx.x; ok && item < a.items; item += gridDim.x) {
                int tile, c0, c1;
                item_range(a, item, tile, c0, c1);
                for (int nc = c0; ok && nc < c1; ++nc, ++acc_it) {
                    const uint32_t buf = acc_it & 1, aph = (acc_it >> 1) & 1;
                    if (!mbar_wait(&tempty[buf], aph ^ 1, abort_flag, a.err)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t dtm = tmem_base + buf * (uint32_t)bn;
                    for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
                        const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
                        if (!mbar_wait(&full[s], ph, abort_flag, a.err)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint32_t ab = su32(sA + s * A_ST), bb = su32(sB + s * B_ST);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            mma<MK>(dtm, sw128_desc(ab + 32 * k), sw128_desc(bb + 32 * k), idesc,
                                    (kb > 0 || k > 0) ? 1u : 0u);
                            if (SPLIT) {
                                mma<MK>(dtm, sw128_desc(ab + 32 * k), sw128_desc(bb + B_STAGE + 32 * k), idesc, 1u);
                                mma<MK>(dtm, sw128_desc(ab + A_STAGE + 32 * k), sw128_desc(bb + 32 * k), idesc, 1u);
                            }
                        }
                        issued = true;
                        mma_commit(&empty[s]);
                    }
                    if (!ok) break;
                    mma_commit(&tfull[buf]);
                }
            }
            if (!ok && issued) {  // wait (bounded) for the MMAs already issued
                mma_commit(drain);
                mbar_drain(drain, 0);
            }
        }
    } else {
        // ------------------------------------------------------ epilogue --
        const int quarter = warp & 3;  // warps 2..9 -> TMEM lanes 64,96,0,32,64,96,0,32
        const int half = (warp - 2) >> 2;
        const int row_in_tile = quarter * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        const int ngrp = bn / 32, cg0 = half ? ngrp / 2 : 0, cg1 = half ? ngrp : ngrp / 2;
        // this warp's column terms of the current chunk (staged once per chunk) and transpose tile
        float *sh = (float *)(smem + RING_BYTES + 256) + (warp - 2) * STG_WORDS;
        int *sid = (int *)(sh + 128);
        float *ssc = sh + 256;
        float *xt = sh + 384;
        uint32_t acc_it = 0;
        bool ok = true;
        for (int item = blockIdx.x; ok && item < a.items; item += gridDim.x) {
            int tile, c0, c1;
            item_range(a, item, tile, c0, c1);
            const int64_t row = (int64_t)tile * BM + row_in_tile;
            const bool row_ok = row < a.nrows_out;
            const float hr = (KIND == DCD_RBF && row_ok) ? a.row_h[row] : 0.f;
            const float rsc = !SCALED ? 1.f : !row_ok ? 0.f : FP8 ? a.row_s[row] : a.row_s[row] * a.col_s[0];
            const float rf = KIND == DCD_RBF ? a.two_gl * rsc : rsc;
            const int rid = !row_ok ? -2 : a.row_id ? a.row_id[row] : (int)row;
            for (int nc = c0; nc < c1; ++nc, ++acc_it) {
                const uint32_t buf = acc_it & 1, aph = (acc_it >> 1) & 1;
                const int64_t cw0 = (int64_t)nc * bn + cg0 * 32;  // this warp's first column
                for (int j = lane; j < (cg1 - cg0) * 32; j += 32) {
                    const int64_t c = cw0 + j;
                    const bool in = c < a.ncols;
                    sh[j] = KIND == DCD_RBF && in ? a.col_h[c] : 0.f;
                    sid[j] = !in ? -1 : a.col_id ? a.col_id[c] : (int)c;
                    if (FP8) ssc[j] = in ? a.col_s[c] : 0.f;
                }
                __syncwarp();
                // every lane polls; the warp proceeds only if all lanes saw the
                // phase complete, so the aligned tcgen05.ld never diverges
                const bool seen = mbar_wait(&tfull[buf], aph, abort_flag, a.err);
                if (!__all_sync(0xffffffffu, seen)) {
                    ok = false;
                    break;
                }
                fence_after();
                for (int cg = cg0; cg < cg1; ++cg) {
                    float v[32];
                    tmem_ld32(tmem_base + lane_addr + buf * (uint32_t)bn + (uint32_t)(cg * 32), v);
                    const int j0 = (cg - cg0) * 32;
                    const int64_t colbase = (int64_t)nc * bn + cg * 32;
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const float c = FP8 ? v[q] * ssc[j0 + q] : v[q];
                        // K with the own-sample rule of the RBF (d^2 = 0 where the row and the column
                        // are the same data row)
                        v[q] = KIND == DCD_RBF && rid == sid[j0 + q] ? 1.f : kf32<KIND>(c, hr, sh[j0 + q], rf, a);
                    }
                    // the 32 x 32 group to memory in two 16-column halves through the transpose tile:
                    // lanes 0..15 write columns 0..15 of one row, lanes 16..31 of the next
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) xt[lane * 17 + q] = v[16 * hh + q];
                        __syncwarp();
                        const int cq = lane & 15;
                        const int64_t col = colbase + 16 * hh + cq;
#pragma unroll 4
                        for (int r2 = 0; r2 < 32; r2 += 2) {
                            const int rr = r2 + (lane >> 4);
                            const int64_t orow = (int64_t)tile * BM + quarter * 32 + rr;
                            if (orow < a.nrows_out && col < a.ncols) a.out[orow * a.ldo + col] = xt[rr * 17 + cq];
                        }
                        __syncwarp();
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
            }
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
}

// ------------------------------------------------ two-SM apply kernel --
// The apply form on CTA pairs (clusters of 2, tcgen05 cta_group::2).  The
// pair owns a 256-row tile; the even CTA issues M = 256 MMAs whose A rows come
// 128 from each CTA's shared memory and whose N-chunk of B is split in two
// halves, one per CTA.  A CTA therefore receives 128 + bn/2 rows per k-block
// instead of 128 + bn -- a third less operand traffic per MMA -- and one MMA
// instruction does twice the work.  Each CTA's tensor memory holds its own
// 128 rows x bn accumulator columns, read back by its own 8 epilogue warps
// exactly as in block_tc_kernel.
//   full[s]   (even CTA) its producer arrives expecting the bytes of both
//             CTAs' loads, which complete_tx on it (the odd CTA's may land
//             first: the transaction count may dip below zero meanwhile)
//   empty[s]  (both) the MMA commit, multicast to the pair
//   tfull[b]  (both) the MMA commit of a finished accumulator, multicast
//   tempty[b] (even CTA) all 16 epilogue warps of the pair arrive
// Every wait is bounded as in block_tc_kernel; the pair meets at a cluster
// barrier after set-up and before tensor memory is released.
constexpr int BM2 = 2 * BM;                          // rows per pair tile
constexpr int B2_STAGE = (BN_MAX / 2) * ROW_BYTES;   // 16 KB: half of an N-chunk
constexpr int RING2_BYTES = 6 * (A_STAGE + B2_STAGE);  // 6 single or 3 split stages
constexpr int CST_FLOATS = 6 * 128;                   // staged column terms per epilogue warp
constexpr int SMEM2_BYTES = RING2_BYTES + 1024 + 256 + XCH_BYTES + 8 * CST_FLOATS * 4;

// arrive on an mbarrier of the pair given by its shared::cluster address
__device__ __forceinline__ void arrive_cl(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}

// TMA tile load into this CTA's shared memory, completing on an mbarrier of
// either CTA of the pair (cluster address)
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, uint32_t bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
        "%4}], [%2];" ::"r"(su32(dst)),
        "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

template <int MK>
__device__ __forceinline__ void mma2(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    if (MK == 1)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtm),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    else if (MK == 2)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtm),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtm),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// arrive on `bar` in both CTAs of the pair once the issued MMAs complete
__device__ __forceinline__ void mma_commit_pair(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            su32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

__device__ __forceinline__ void mma_commit_own2(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

// The (row tile, N-chunk) units of a pair.  Ranged: the units, in row-major
// order, are cut into npairs contiguous ranges (each at least one tile long,
// so a tile is shared by at most two pairs) of near-equal length, or, with
// late pairs, the last L pairs' ranges D units shorter than the others'.
// Else each pair takes whole tiles pair, pair + npairs, ...
// (The host keeps items * nchunks below 2^31.)
__device__ __forceinline__ int64_t range_start(int64_t U, int npairs, int L, int D, int p)
{
    // sum of the first p range lengths (times npairs): early ranges s = (U + L D) / npairs, late s - D
    const int64_t late = p > npairs - L ? p - (npairs - L) : 0;
    return ((int64_t)p * (U + (int64_t)L * D) - (int64_t)npairs * D * late) / npairs;
}

__device__ __forceinline__ void pair_units(const TcArgs &a, int pair, int npairs, bool &ranged, int &u0, int &u1,
                                           int &n)
{
    const int64_t U = (int64_t)a.items * a.nchunks;
    ranged = a.part != nullptr && U / npairs >= a.nchunks;
    if (ranged) {
        int L = a.late_pairs, D = a.late_units;
        if (L <= 0 || L >= npairs || D <= 0 || (U + (int64_t)L * D) / npairs - D < a.nchunks) L = D = 0;
        u0 = (int)range_start(U, npairs, L, D, pair);
        u1 = (int)range_start(U, npairs, L, D, pair + 1);
        n = u1 - u0;
    } else {
        u0 = 0;
        u1 = (int)U;
        n = pair < a.items ? (a.items - pair + npairs - 1) / npairs * a.nchunks : 0;
    }
}

// The i-th unit of a pair.  Ranged: even pairs take their tiles first to
// last, odd pairs last to first (the chunks of a tile in order either way),
// so that both pairs that share a tile reach it at about the same time (at
// the start of both ranges, or at the end of both) and its rows of A are
// read from memory once.
__device__ __forceinline__ void pair_unit(const TcArgs &a, int pair, int npairs, bool ranged, int u0, int u1, int i,
                                          int &tile, int &nc)
{
    if (ranged) {
        const int nch = a.nchunks;
        int u = u0 + i;
        if (pair & 1) {
            const int thi = (u1 - 1) / nch, tlo = u0 / nch;
            const int top = u1 - max(u0, thi * nch);  // units of the last tile
            if (i < top) {
                u = u1 - top + i;
            } else {
                const int j = i - top, mid = (thi - 1 - tlo) * nch;  // units of the full tiles between
                u = j < mid ? (thi - 1 - j / nch) * nch + j % nch : u0 + (j - mid);
            }
        }
        tile = u / nch;
        nc = u % nch;
    } else {
        tile = pair + i / a.nchunks * npairs;
        nc = i % a.nchunks;
    }
}

template <int MODE, int KIND>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHREADS, 1)
    block_tc2_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs a)
{
    constexpr bool SL = MODE == MODE_SLICED;
    constexpr bool ACC = MODE == MODE_ACC || SL;  // the accurate epilogue
    constexpr bool TF32 = MODE == MODE_TF32 || MODE == MODE_TF32X3 || MODE == MODE_ACC;
    constexpr bool FP8 = MODE == MODE_FP8;
    constexpr bool FP16 = MODE == MODE_FP16;
    constexpr bool SCALED = FP8 || FP16;  // operand scales restored in the epilogue
    constexpr int MK = TF32 ? 1 : FP8 ? 2 : 0;
    constexpr bool SPLIT = MODE == MODE_BF16X3 || MODE == MODE_TF32X3 || MODE == MODE_ACC;
    constexpr int PLANES = SL ? 4 : SPLIT ? 2 : 1;  // operand planes (hi, lo / the four slices)
    constexpr int STAGES = SL ? 2 : SPLIT ? 3 : 6;
    // a stage holds every plane of one k-block; the sliced form's B planes are SLICED_BN / 2 rows
    constexpr int B_PLANE = SL ? (SLICED_BN / 2) * ROW_BYTES : B2_STAGE;
    constexpr int A_ST = PLANES * A_STAGE;
    constexpr int B_ST = PLANES * B_PLANE;
    constexpr int NACC = SL ? 1 : 2;  // accumulator buffers in tensor memory
    static_assert(STAGES * (A_ST + B_ST) <= RING2_BYTES, "operand ring exceeds its shared memory");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * A_ST;
    uint64_t *bars = (uint64_t *)(smem + RING2_BYTES);
    uint64_t *full = bars;                 // STAGES (even CTA)
    uint64_t *empty = bars + STAGES;       // STAGES
    uint64_t *tfull = bars + 2 * STAGES;   // 2
    uint64_t *tempty = tfull + 2;          // 2 (even CTA)
    uint64_t *drain = tempty + 2;          // 1
    uint64_t *xfull = drain + 1;           // 2
    uint64_t *xfree = xfull + 2;           // 2
    double *xch = (double *)(smem + RING2_BYTES + 256);  // [2][BM]
    uint32_t *tmem_holder = (uint32_t *)(xfree + 2);
    volatile int *abort_flag = (volatile int *)(tmem_holder + 1);

    const uint32_t rank = ptx::cluster_ctarank();
    const int pair = (int)(blockIdx.x >> 1), npairs = (int)(gridDim.x >> 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 16);
            mbar_init(&xfull[b], 4);
            mbar_init(&xfree[b], 4);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    ptx::cluster_sync();  // both CTAs' barriers exist before any cross-CTA arrive
    fence_after();
    const uint32_t tmem_base = *tmem_holder;
    const int bn = a.bn, bh = bn / 2;
    const int kb_elems = TF32 ? 32 : FP8 ? 128 : 64;
    const uint32_t full0 = ptx::mapa(su32(full), 0), tempty0 = ptx::mapa(su32(tempty), 0);
    bool ranged;
    int u0, u1, nunits;
    pair_units(a, pair, npairs, ranged, u0, u1, nunits);

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------- producer --
            uint32_t it = 0;
            bool ok = true;
            const uint32_t bytes = (uint32_t)(2 * PLANES * (A_STAGE + bh * ROW_BYTES));  // both CTAs'
            for (int i = 0; ok && i < nunits; ++i) {
                int item, nc;
                pair_unit(a, pair, npairs, ranged, u0, u1, i, item, nc);
                for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
                        const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
                        if (!mbar_wait(&empty[s], ph ^ 1, abort_flag, a.err)) {
                            ok = false;
                            break;
                        }
                        const uint32_t fb = full0 + 8u * s;
                        const int ya = item * BM2 + (int)rank * BM, yb = nc * bn + (int)rank * bh;
                        if (rank == 0) mbar_expect_tx(&full[s], bytes);
#pragma unroll
                        for (int pl = 0; pl < PLANES; ++pl) {  // plane pl starts at column pl * lo_off
                            tma_load_2d_pair(sA + s * A_ST + pl * A_STAGE, &tmA, fb, pl * a.lo_off + kb * kb_elems, ya);
                            tma_load_2d_pair(sB + s * B_ST + pl * B_PLANE, &tmB, fb, pl * a.lo_off + kb * kb_elems, yb);
                        }
                    }
            }
            // the last stages' empties arrive after the final MMAs: wait for them, so that no
            // commit is still addressed to this CTA when the pair leaves (bounded)
            const uint32_t first = it > STAGES ? it - STAGES : 0;
            for (uint32_t j = first; j < it; ++j) mbar_drain(&empty[j % STAGES], ((j / STAGES) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // --------------------------------------------------------- MMA --
            const uint32_t idesc = make_idesc(TF32 ? 2 : SCALED ? 0 : 1, bn, BM2);  // tf32, e4m3 / f16, bf16
            uint32_t it = 0, acc_it = 0;
            bool ok = true, issued = false;
            for (int i = 0; ok && i < nunits; ++i, ++acc_it) {
                    const uint32_t buf = acc_it % NACC, aph = (acc_it / NACC) & 1;
                    if (!mbar_wait(&tempty[buf], aph ^ 1, abort_flag, a.err)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t dtm = tmem_base + buf * (uint32_t)bn;
                    for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
                        const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
                        if (!mbar_wait(&full[s], ph, abort_flag, a.err)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint32_t ab = su32(sA + s * A_ST), bb = su32(sB + s * B_ST);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (SL) {
                                // accumulator g (columns g * bn..) takes the products of slices p and g - p
#pragma unroll
                                for (int g = 0; g < 4; ++g)
#pragma unroll
                                    for (int p = 0; p <= g; ++p)
                                        mma2<MK>(dtm + (uint32_t)(g * bn), sw128_desc(ab + p * A_STAGE + 32 * k),
                                                 sw128_desc(bb + (g - p) * B_PLANE + 32 * k), idesc,
                                                 (kb > 0 || k > 0 || p > 0) ? 1u : 0u);
                                continue;
                            }
                            mma2<MK>(dtm, sw128_desc(ab + 32 * k), sw128_desc(bb + 32 * k), idesc,
                                     (kb > 0 || k > 0) ? 1u : 0u);
                            if (SPLIT) {
                                mma2<MK>(dtm, sw128_desc(ab + 32 * k), sw128_desc(bb + B2_STAGE + 32 * k), idesc, 1u);
                                mma2<MK>(dtm, sw128_desc(ab + A_STAGE + 32 * k), sw128_desc(bb + 32 * k), idesc, 1u);
                            }
                        }
                        issued = true;
                        mma_commit_pair(&empty[s]);
                    }
                    if (!ok) break;
                    mma_commit_pair(&tfull[buf]);
                }
            if (issued) {  // every MMA (and its commits) done before the pair tears down
                mma_commit_own2(drain);
                mbar_drain(drain, 0);
            }
        }
    } else {
        // ------------------------------------------------------ epilogue --
        // the coefficients and the gradient may come from the grid before this one (a programmatic
        // dependency: the tensor-memory products above start without it); a no-op otherwise.  A
        // launch beside a grid whose results it does not read skips the wait (dep_wait = 0).
        if (a.dep_wait) asm volatile("griddepcontrol.wait;" ::: "memory");
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row_in_tile = quarter * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        const int ngrp = bn / 32, cg0 = half ? ngrp / 2 : 0, cg1 = half ? ngrp : ngrp / 2;
        // this warp's column terms of the current chunk (its half: <= 4 groups): K-term, coefficient, scale
        float *cst = (float *)(smem + RING2_BYTES + 256 + XCH_BYTES) + (warp - 2) * CST_FLOATS;
        uint32_t acc_it = 0, item_it = 0;
        bool ok = true;
        int64_t row = 0;
        bool row_ok = false;
        float hr = 0.f, hrl = 0.f, rf = 0.f, rsl = 0.f;
        int rid = -2;  // data-matrix row of this thread's row (-2: none)
        const int *cid = (const int *)(cst + 512);  // staged column ids (-1 past the block)
        double tacc = 0.0;  // this half's row sum over the tile's chunks so far, in chunk order
        const int nch = a.nchunks;
        bool fast_cols = false, fast_row = false;  // the factored RBF form applies (warp-uniform)
        for (int i = 0; ok && i < nunits; ++i, ++acc_it) {
            int item, nc;
            pair_unit(a, pair, npairs, ranged, u0, u1, i, item, nc);
            const int u = item * nch + nc;
            if (u == u0 || nc == 0) {  // first chunk of a tile in this pair's units
                row = (int64_t)item * BM2 + (int64_t)rank * BM + row_in_tile;
                row_ok = row < a.nrows_out;
                hr = (KIND == DCD_RBF && row_ok) ? a.row_h[row] : 0.f;
                if (ACC) hrl = (KIND == DCD_RBF && row_ok) ? a.row_hl[row] : 0.f;
                if (SL) rsl = row_ok ? a.row_s[row] * 0x1p-12f : 0.f;  // 2^(e_i - 12)
                rid = row_ok ? (a.row_id ? a.row_id[row] : (int)row) : -2;
                const float rsc = !SCALED ? 1.f : !row_ok ? 0.f : FP8 ? a.row_s[row] : a.row_s[row] * a.col_s[0];
                rf = KIND == DCD_RBF ? a.two_gl * rsc : rsc;
                fast_row = __all_sync(0xffffffffu, hr <= RBF_FACTOR_HMAX);
                tacc = 0.0;
            }
            const bool whole = !ranged || (item * nch >= u0 && (item + 1) * nch <= u1);
            const bool last = nc == nch - 1 || u == u1 - 1;  // last chunk of the tile in this pair's units
            // this chunk's part of the row sum (this half's column groups): the fast epilogue adds
            // its groups in double-single FP32 (GB300's FP64 pipe issues ~1.6 operations per clock
            // per SM, too few for per-group FP64 sums at the bf16 MMA rate), the accurate ones in FP64
            double cs = 0.0;
            float cs_h = 0.f, cs_l = 0.f;
            // one 32-column group: terms from the staged columns (4 per shared-memory load), the
            // same sums in the same order as a column-by-column loop
            // the 32 columns' kernel values (`own`: bit q set where column q is this row's own
            // sample, d^2 = 0 there; the checked form runs only for the rare groups that hold one)
            auto group_terms = [&](const uint32_t(&r)[32], int j0, unsigned own, float &p0, float &p1) {
                if (KIND == DCD_RBF && !FP8 && !ACC && !own && fast_cols && fast_row) {
                    // K_ij w_j = 2^(rf c - h_i) (w_j 2^(-h_j)): the exponent's row and column terms split
                    // apart (both <= RBF_FACTOR_HMAX, so neither factor leaves the FP32 range); rf c <=
                    // h_i + h_j by Cauchy-Schwarz, so the first factor is at most 2^(h_j)
                    const float4 *f4 = (const float4 *)(cst + 384 + j0);
                    const float nh = -hr;
#pragma unroll
                    for (int q4 = 0; q4 < 8; ++q4) {
                        const float4 ff = f4[q4];
                        p0 = fmaf(ex2f(fmaf(__uint_as_float(r[4 * q4]), rf, nh)), ff.x, p0);
                        p1 = fmaf(ex2f(fmaf(__uint_as_float(r[4 * q4 + 1]), rf, nh)), ff.y, p1);
                        p0 = fmaf(ex2f(fmaf(__uint_as_float(r[4 * q4 + 2]), rf, nh)), ff.z, p0);
                        p1 = fmaf(ex2f(fmaf(__uint_as_float(r[4 * q4 + 3]), rf, nh)), ff.w, p1);
                    }
                    return;
                }
                const float4 *h4 = (const float4 *)(cst + j0), *w4 = (const float4 *)(cst + 128 + j0),
                             *s4 = (const float4 *)(cst + 256 + j0);
#pragma unroll
                for (int q4 = 0; q4 < 8; ++q4) {
                    const float4 hh = KIND == DCD_RBF ? h4[q4] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 ww = w4[q4];
                    float c0 = __uint_as_float(r[4 * q4]), c1 = __uint_as_float(r[4 * q4 + 1]);
                    float c2 = __uint_as_float(r[4 * q4 + 2]), c3 = __uint_as_float(r[4 * q4 + 3]);
                    if (FP8) {
                        const float4 ss = s4[q4];
                        c0 *= ss.x;
                        c1 *= ss.y;
                        c2 *= ss.z;
                        c3 *= ss.w;
                    }
                    float k0 = kf32<KIND>(c0, hr, hh.x, rf, a), k1 = kf32<KIND>(c1, hr, hh.y, rf, a);
                    float k2 = kf32<KIND>(c2, hr, hh.z, rf, a), k3 = kf32<KIND>(c3, hr, hh.w, rf, a);
                    if (own) {
                        k0 = (own >> (4 * q4)) & 1u ? 1.f : k0;
                        k1 = (own >> (4 * q4 + 1)) & 1u ? 1.f : k1;
                        k2 = (own >> (4 * q4 + 2)) & 1u ? 1.f : k2;
                        k3 = (own >> (4 * q4 + 3)) & 1u ? 1.f : k3;
                    }
                    p0 = fmaf(k0, ww.x, p0);
                    p1 = fmaf(k1, ww.y, p1);
                    p0 = fmaf(k2, ww.z, p0);
                    p1 = fmaf(k3, ww.w, p1);
                }
            };
            // one 32-column group: terms from the staged columns (4 per shared-memory load), the
            // same sums in the same order as a column-by-column loop
            auto group = [&](const uint32_t(&r)[32], int j0) {
                float p0 = 0.f, p1 = 0.f;
                // the own-sample columns of this warp's 32 rows: each lane tests one column id
                unsigned own = 0;
                if (KIND == DCD_RBF && !a.row_id) {
                    const int wr0 = __shfl_sync(0xffffffffu, rid, 0);  // lanes hold consecutive rows
                    const unsigned off = (unsigned)(cid[j0 + lane] - wr0);
                    unsigned hits = __ballot_sync(0xffffffffu, rid >= 0 && off < 32u);
                    while (hits) {
                        const int q = __ffs(hits) - 1;
                        hits &= hits - 1;
                        if (cid[j0 + q] == rid) own |= 1u << q;
                    }
                } else if (KIND == DCD_RBF) {  // rows given by id: every column tested
                    for (int q = 0; q < 32; ++q) own |= (cid[j0 + q] == rid ? 1u : 0u) << q;
                }
                if (own) group_terms(r, j0, own, p0, p1);
                else group_terms(r, j0, 0u, p0, p1);
                float a0, b0, e0;
                two_sum(p0, p1, a0, b0);
                two_sum(cs_h, a0, cs_h, e0);
                cs_l += e0 + b0;
            };
            // the accurate form of one group: staged columns [h | w_hi | w_lo | h_lo]; the exponent
            // x = 2 gamma log2(e) c - (h_i + h_j) = -gamma log2(e) d^2 and the kernel value in
            // double-single, the products with w summed in double-single (two sums, alternate columns)
            auto contract = [&](float kh, float kl, int j, int q, float &ah0, float &al0, float &ah1, float &al1) {
                const float wh = cst[128 + j], wl = cst[256 + j];
                float pp, pe, sm, se;
                two_prod(kh, wh, pp, pe);
                pe = fmaf(kh, wl, fmaf(kl, wh, pe));
                if (q & 1) {
                    two_sum(ah1, pp, sm, se);
                    al1 += se + pe;
                    ah1 = sm;
                } else {
                    two_sum(ah0, pp, sm, se);
                    al0 += se + pe;
                    ah0 = sm;
                }
            };
            auto group_acc = [&](const uint32_t(&r)[32], int j0) {
                float ah0 = 0.f, al0 = 0.f, ah1 = 0.f, al1 = 0.f;
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int j = j0 + q;
                    float kh, kl;
                    if (KIND == DCD_RBF && cid[j] == rid) {  // the own sample: d^2 = 0
                        kh = 1.f;
                        kl = 0.f;
                    } else {
                        k_accurate<KIND>(__uint_as_float(r[q]), 0.f, hr, hrl, cst[j], cst[384 + j], a, kh, kl);
                    }
                    contract(kh, kl, j, q, ah0, al0, ah1, al1);
                }
                cs += ((double)ah0 + (double)al0) + ((double)ah1 + (double)al1);
            };
            // the sliced form of one group: the four accumulators' exact integer sums G_g (plane
            // products with p + q = g) for 16 columns at a time, combined in double-single as
            // a.b = 2^(e_i + e_j - 12) (G0 + 2^-7 G1 + 2^-14 G2 + 2^-21 G3)
            auto group_sl = [&](uint32_t tb, int cg, int j0) {
                float ah0 = 0.f, al0 = 0.f, ah1 = 0.f, al1 = 0.f;
#pragma unroll 1
                for (int hh = 0; hh < 2; ++hh) {
                    float G0[16], G1[16], G2[16], G3[16];
                    const uint32_t ta = tb + (uint32_t)(cg * 32 + hh * 16);
                    tmem_ld16(ta, G0);
                    tmem_ld16(ta + (uint32_t)bn, G1);
                    tmem_ld16(ta + 2u * (uint32_t)bn, G2);
                    tmem_ld16(ta + 3u * (uint32_t)bn, G3);
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int j = j0 + hh * 16 + q;
                        float kh, kl;
                        if (KIND == DCD_RBF && cid[j] == rid) {  // the own sample: d^2 = 0
                            kh = 1.f;
                            kl = 0.f;
                        } else {
                            float th, tl, uh, ul, vh, vl, e1;
                            two_sum(G2[q] * 0x1p-14f, G3[q] * 0x1p-21f, th, tl);
                            two_sum(G1[q] * 0x1p-7f, th, uh, e1);
                            ul = e1 + tl;
                            two_sum(G0[q], uh, vh, e1);
                            vl = e1 + ul;
                            const float scl = rsl * cst[640 + j];  // 2^(e_i + e_j - 12), exact
                            k_accurate<KIND>(vh * scl, vl * scl, hr, hrl, cst[j], cst[384 + j], a, kh, kl);
                        }
                        contract(kh, kl, j, q, ah0, al0, ah1, al1);
                    }
                }
                cs += ((double)ah0 + (double)al0) + ((double)ah1 + (double)al1);
            };
            const uint32_t buf = acc_it % NACC, aph = (acc_it / NACC) & 1;
            // stage this warp's columns while the accumulator is still being formed
            const int64_t cbase = (int64_t)nc * bn + cg0 * 32;
            for (int j = lane; j < (cg1 - cg0) * 32; j += 32) {
                if (KIND == DCD_RBF) {
                    cst[j] = a.col_h[cbase + j];
                    const int64_t c = cbase + j;
                    ((int *)cst)[512 + j] = c < a.ncols ? (a.col_id ? a.col_id[c] : (int)c) : -1;
                }
                if (ACC) {
                    const double wv = cbase + j < a.ncols ? a.col_w64[cbase + j] : 0.0;
                    const float wh = (float)wv;
                    cst[128 + j] = wh;
                    cst[256 + j] = (float)(wv - (double)wh);
                    if (KIND == DCD_RBF) cst[384 + j] = a.col_hl[cbase + j];
                    if (SL) cst[640 + j] = cbase + j < a.ncols ? a.col_s[cbase + j] : 0.f;
                } else {
                    cst[128 + j] = a.col_w[cbase + j];
                    if (FP8) cst[256 + j] = a.col_s[cbase + j];
                    // the RBF's column factor w_j 2^(-h_j) of the factored form below
                    if (KIND == DCD_RBF && !FP8) cst[384 + j] = a.col_w[cbase + j] * ex2f(-a.col_h[cbase + j]);
                }
            }
            if (KIND == DCD_RBF && !ACC && !FP8) {  // the factored form needs every h_j <= RBF_FACTOR_HMAX
                float hm = 0.f;
                for (int j = lane; j < (cg1 - cg0) * 32; j += 32) hm = fmaxf(hm, cst[j]);
                fast_cols = __all_sync(0xffffffffu, hm <= RBF_FACTOR_HMAX);
            }
            __syncwarp();
            const bool seen = mbar_wait(&tfull[buf], aph, abort_flag, a.err);
            if (!__all_sync(0xffffffffu, seen)) {
                ok = false;
                break;
            }
            fence_after();
            const uint32_t tb = tmem_base + lane_addr + buf * (uint32_t)bn;
            if constexpr (SL) {
                for (int cg = cg0; cg < cg1; ++cg) group_sl(tb, cg, (cg - cg0) * 32);
            } else {
                uint32_t ra[32], rb[32];
                if (cg0 < cg1) {
                    tmem_ld32_issue(tb + (uint32_t)(cg0 * 32), ra);
                    tmem_ld_wait(ra);
                }
                auto any_group = [&](const uint32_t(&r)[32], int j0) {
                    if constexpr (ACC) group_acc(r, j0);
                    else group(r, j0);
                };
                for (int cg = cg0; cg < cg1; cg += 2) {  // ra holds group cg
                    if (cg + 1 < cg1) tmem_ld32_issue(tb + (uint32_t)((cg + 1) * 32), rb);
                    any_group(ra, (cg - cg0) * 32);
                    if (cg + 1 < cg1) {
                        tmem_ld_wait(rb);
                        if (cg + 2 < cg1) tmem_ld32_issue(tb + (uint32_t)((cg + 2) * 32), ra);
                        any_group(rb, (cg + 1 - cg0) * 32);
                        if (cg + 2 < cg1) tmem_ld_wait(ra);
                    }
                }
            }
            cs += (double)cs_h + (double)cs_l;
            fence_before();
            __syncwarp();
            if (lane == 0) arrive_cl(tempty0 + 8u * buf);
            if (!whole) {
                // a tile shared with the neighbouring pair: park this chunk's sums in its slot (the
                // index of the pair boundary inside the tile); the last of the 16 epilogue warps of
                // the two pairs (this CTA rank) to arrive adds every chunk's sums in chunk order
                const int slot = item * nch < u0 ? pair : pair + 1;
                double *pt = a.part + (size_t)slot * nch * 2 * BM2 + (size_t)rank * BM;
                pt[((size_t)nc * 2 + half) * BM2 + row_in_tile] = cs;
                if (last) {
                    __threadfence();
                    __syncwarp();
                    unsigned old = 0;
                    if (lane == 0) old = atomicAdd(&a.cnt[2 * slot + (int)rank], 1u);
                    old = __shfl_sync(0xffffffffu, old, 0);
                    if (old == 15u) {
                        __threadfence();
                        for (int r = lane; r < BM; r += 32) {
                            const int64_t grow = (int64_t)item * BM2 + (int64_t)rank * BM + r;
                            if (grow >= a.nrows_out) continue;
                            double t0 = 0.0, t1 = 0.0;
                            for (int k = 0; k < nch; ++k) {
                                t0 += __ldcg(pt + (size_t)k * 2 * BM2 + r);
                                t1 += __ldcg(pt + ((size_t)k * 2 + 1) * BM2 + r);
                            }
                            a.g[grow] += (a.rs ? a.rs[grow] : 1.0) * (t0 + t1);
                        }
                        if (lane == 0) a.cnt[2 * slot + (int)rank] = 0u;
                    }
                }
                continue;
            }
            tacc += cs;
            if (!last) continue;
            const uint32_t xb = item_it & 1, xph = (item_it >> 1) & 1;
            ++item_it;
            double *xc = xch + xb * BM;
            if (half) {
                const bool fr = mbar_wait(&xfree[xb], xph ^ 1, abort_flag, a.err);
                if (!__all_sync(0xffffffffu, fr)) {
                    ok = false;
                    break;
                }
                xc[row_in_tile] = tacc;
                __syncwarp();
                if (lane == 0) mbar_arrive(&xfull[xb]);
            } else {
                const bool fu = mbar_wait(&xfull[xb], xph, abort_flag, a.err);
                if (!__all_sync(0xffffffffu, fu)) {
                    ok = false;
                    break;
                }
                const double tot = tacc + xc[row_in_tile];
                __syncwarp();
                if (lane == 0) mbar_arrive(&xfree[xb]);
                if (row_ok) a.g[row] += (a.rs ? a.rs[row] : 1.0) * tot;
            }
        }
    }
    fence_before();
    __syncthreads();
    ptx::cluster_sync();  // the pair is done with each other's barriers and tensor memory
    fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
}

// ------------------------------------------------------------------ host --
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

bool make_map(CUtensorMap *map, const TcOperand &op, int box_rows)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const bool f32 = op.kind == PACK_TF32 || op.kind == PACK_TF32X3, fp8 = op.kind == PACK_FP8;
    const int esz = f32 ? 4 : fp8 ? 1 : 2;
    const int64_t cols = op.kind == PACK_SLICED                                  ? 4 * op.n_pad
                         : (op.kind == PACK_BF16X3 || op.kind == PACK_TF32X3) ? 2 * op.n_pad
                                                                              : op.n_pad;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)op.nrows};
    cuuint64_t strides[1] = {(cuuint64_t)(cols * esz)};
    cuuint32_t box[2] = {(cuuint32_t)(ROW_BYTES / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                   : op.kind == PACK_FP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                         : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = fn(map, dt, 2,
                    const_cast<void *>(op.rows), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int MODE, int KIND>
cudaError_t launch_kind(int grid, const CUtensorMap &mA, const CUtensorMap &mB, const TcArgs &a, cudaStream_t st)
{
    auto kfn = block_tc_kernel<MODE, KIND>;
    static bool attr_set = false;  // one attribute call per instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    kfn<<<grid, NTHREADS, SMEM_BYTES, st>>>(mA, mB, a);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_mode(int grid, const CUtensorMap &mA, const CUtensorMap &mB, const TcArgs &a, int kind,
                        cudaStream_t st)
{
    if (kind == DCD_RBF) return launch_kind<MODE, DCD_RBF>(grid, mA, mB, a, st);
    if (kind == DCD_POLY) return launch_kind<MODE, DCD_POLY>(grid, mA, mB, a, st);
    return launch_kind<MODE, DCD_LINEAR>(grid, mA, mB, a, st);
}

template <int MODE, int KIND>
cudaError_t launch_kind2(int npairs, const CUtensorMap &mA, const CUtensorMap &mB, const TcArgs &a, cudaStream_t st,
                         bool pdl, int prio)
{
    auto kfn = block_tc2_kernel<MODE, KIND>;
    static int max_pairs = 0;  // co-resident pairs, queried once per instantiation (before any capture)
    if (!max_pairs) {
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM2_BYTES);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2, 1, 1);
        cfg.blockDim = dim3(NTHREADS, 1, 1);
        cfg.dynamicSmemBytes = SMEM2_BYTES;
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, kfn, &cfg);
        if (e != cudaSuccess) return e;
        if (n < 1) return cudaErrorInvalidConfiguration;
        max_pairs = n;
    }
    if (npairs > max_pairs) npairs = max_pairs;
    if (!pdl && !prio) {
        kfn<<<2 * npairs, NTHREADS, SMEM2_BYTES, st>>>(mA, mB, a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * npairs, 1, 1);
    cfg.blockDim = dim3(NTHREADS, 1, 1);
    cfg.dynamicSmemBytes = SMEM2_BYTES;
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
    return cudaLaunchKernelEx(&cfg, kfn, mA, mB, a);
}

template <int MODE>
cudaError_t launch_mode2(int npairs, const CUtensorMap &mA, const CUtensorMap &mB, const TcArgs &a, int kind,
                         cudaStream_t st, bool pdl, int prio)
{
    if (kind == DCD_RBF) return launch_kind2<MODE, DCD_RBF>(npairs, mA, mB, a, st, pdl, prio);
    if (kind == DCD_POLY) return launch_kind2<MODE, DCD_POLY>(npairs, mA, mB, a, st, pdl, prio);
    return launch_kind2<MODE, DCD_LINEAR>(npairs, mA, mB, a, st, pdl, prio);
}

}  // namespace

bool tc_available()
{
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    return major == 10 && minor == 3 && encode_fn() != nullptr;
}

bool make_map_f32_2d(CUtensorMap *map, const float *base, int64_t cols, int64_t rows, int64_t ld, int box_cols,
                     int box_rows)
{
    auto fn = encode_fn();
    if (!fn || cols < 1 || rows < 1 || (ld * 4) % 16 != 0 || ((uintptr_t)base & 15) != 0) return false;
    if (box_cols < 1 || box_cols > 256 || box_rows < 1 || box_rows > 256 || (box_cols * 4) % 16 != 0) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

cudaError_t launch_block_tc(const TcOperand &Aop, const TcOperand &Bop, const KernelParams &kp, const float *row_h,
                            const float *col_h, const float *col_w, const double *rs, double *g, float *out,
                            int64_t ldo, int64_t nrows_out, int64_t ncols, int *err, cudaStream_t st, bool lower,
                            const TcSplit *split, bool pdl, int max_pairs, const TcAccurate *acc, bool pdl_wait,
                            int prio)
{
    if (nrows_out <= 0 || ncols <= 0) return cudaSuccess;
    // the accurate apply epilogue: split-tf32 or sliced operands, FP64 coefficients, RBF terms as hi + lo
    const bool sliced = Aop.kind == PACK_SLICED;
    if (acc && (out != nullptr || (Aop.kind != PACK_TF32X3 && !sliced) || !acc->w64 ||
                (kp.kind == DCD_RBF && (!acc->row_hl || !acc->col_hl))))
        return cudaErrorInvalidValue;
    if (sliced && (!acc || !Aop.scale || !Bop.scale || Aop.n_pad > SLICED_N_MAX)) return cudaErrorInvalidValue;
    if (Aop.kind != Bop.kind || Aop.n_pad != Bop.n_pad) return cudaErrorInvalidValue;
    if (Aop.kind != PACK_BF16 && Aop.kind != PACK_TF32 && Aop.kind != PACK_BF16X3 && Aop.kind != PACK_TF32X3 &&
        Aop.kind != PACK_FP8 && Aop.kind != PACK_SLICED && Aop.kind != PACK_FP16)
        return cudaErrorInvalidValue;
    if ((Aop.kind == PACK_FP8 || Aop.kind == PACK_FP16) && (!Aop.scale || !Bop.scale)) return cudaErrorInvalidValue;
    const int kb_elems = k_block_elems(Aop.kind);
    if (Aop.n_pad % kb_elems) return cudaErrorInvalidValue;
    int bn = (int)((ncols + 31) / 32) * 32;
    if (bn > (sliced ? SLICED_BN : BN_MAX)) bn = sliced ? SLICED_BN : BN_MAX;
    // store mode (the sampled Gram) has few rows: narrower N-chunks give
    // more work items and spread them over more SMs -- unless it is held to a
    // few CTAs (max_pairs), where wide chunks mean fewer, longer items
    if (out != nullptr && max_pairs <= 0) bn = bn > 64 ? 64 : bn;
    // the apply form runs on CTA pairs (each CTA stages half of an N-chunk of B)
    const bool pair = out == nullptr;
    CUtensorMap mA, mB;
    if (!make_map(&mA, Aop, BM) || !make_map(&mB, Bop, pair ? bn / 2 : bn)) return cudaErrorInvalidValue;
    TcArgs a;
    a.lo_off = (int)Aop.n_pad;
    a.row_h = row_h;
    a.col_h = col_h;
    a.col_w = col_w;
    a.rs = rs;
    a.row_s = Aop.scale;
    a.col_s = Bop.scale;
    a.g = g;
    a.out = out;
    a.ldo = ldo;
    a.nrows_out = nrows_out;
    a.ncols = ncols;
    a.num_tiles = (int)((nrows_out + (pair ? 2 * BM : BM) - 1) / (pair ? 2 * BM : BM));
    a.nchunks = (int)((ncols + bn - 1) / bn);
    a.kblocks = (int)(Aop.n_pad / kb_elems);
    a.bn = bn;
    a.store = out != nullptr;
    a.lower = a.store && lower;
    a.items = a.store ? a.num_tiles * a.nchunks : a.num_tiles;
    if (a.lower) {
        a.items = 0;
        for (int t = 0; t < a.num_tiles; ++t) a.items += lower_chunks(t, a.bn, a.nchunks);
    }
    a.degree = kp.degree;
    a.two_gl = (float)(2.0 * kp.gamma * 1.4426950408889634);
    a.coef0 = (float)kp.coef0;
    a.err = err;
    a.part = nullptr;
    a.cnt = nullptr;
    a.late_pairs = 0;
    a.late_units = 0;
    a.row_id = Aop.ids;
    a.col_id = Bop.ids;
    a.dep_wait = pdl_wait ? 1 : 0;
    a.row_hl = acc ? acc->row_hl : nullptr;
    a.col_hl = acc ? acc->col_hl : nullptr;
    a.col_w64 = acc ? acc->w64 : nullptr;
    {
        const double tg = 2.0 * kp.gamma * 1.4426950408889634;
        a.two_gl_lo = (float)(tg - (double)a.two_gl);
    }
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    if (pair) {
        if ((int64_t)a.num_tiles * a.nchunks >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
        int npairs = a.items < sms / 2 ? a.items : sms / 2;
        if (max_pairs > 0 && npairs > max_pairs) npairs = max_pairs;
        if (split && split->part && split->cnt && split->pairs >= npairs && split->chunks >= a.nchunks) {
            a.part = split->part;
            a.cnt = split->cnt;
            a.late_pairs = split->late_pairs;
            a.late_units = split->late_units;
        }
        if (sliced) return launch_mode2<MODE_SLICED>(npairs, mA, mB, a, kp.kind, st, pdl, prio);
        if (acc) return launch_mode2<MODE_ACC>(npairs, mA, mB, a, kp.kind, st, pdl, prio);
        if (Aop.kind == PACK_TF32) return launch_mode2<MODE_TF32>(npairs, mA, mB, a, kp.kind, st, pdl, prio);
        if (Aop.kind == PACK_BF16X3) return launch_mode2<MODE_BF16X3>(npairs, mA, mB, a, kp.kind, st, pdl, prio);
        if (Aop.kind == PACK_TF32X3) return launch_mode2<MODE_TF32X3>(npairs, mA, mB, a, kp.kind, st, pdl, prio);
        if (Aop.kind == PACK_FP8) return launch_mode2<MODE_FP8>(npairs, mA, mB, a, kp.kind, st, pdl, prio);
        if (Aop.kind == PACK_FP16) return launch_mode2<MODE_FP16>(npairs, mA, mB, a, kp.kind, st, pdl, prio);
        return launch_mode2<MODE_BF16>(npairs, mA, mB, a, kp.kind, st, pdl, prio);
    }
    int grid = a.items < sms ? a.items : sms;
    if (max_pairs > 0 && grid > max_pairs) grid = max_pairs;
    if (Aop.kind == PACK_TF32) return launch_mode<MODE_TF32>(grid, mA, mB, a, kp.kind, st);
    if (Aop.kind == PACK_BF16X3) return launch_mode<MODE_BF16X3>(grid, mA, mB, a, kp.kind, st);
    if (Aop.kind == PACK_TF32X3) return launch_mode<MODE_TF32X3>(grid, mA, mB, a, kp.kind, st);
    if (Aop.kind == PACK_FP8) return launch_mode<MODE_FP8>(grid, mA, mB, a, kp.kind, st);
    if (Aop.kind == PACK_FP16) return launch_mode<MODE_FP16>(grid, mA, mB, a, kp.kind, st);
    return launch_mode<MODE_BF16>(grid, mA, mB, a, kp.kind, st);
}

}  // namespace dcd
