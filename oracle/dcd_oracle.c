/*
 * dcd_oracle.c -- plain, slow, FP64 CPU oracle for s-step DCD (K-SVM) and
 * s-step BDCD (K-RR), "Scalable Dual Coordinate Descent for Kernel Methods"
 * (arXiv 2406.18001).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke check
 * and the benchmark's CPU-baseline leg may load or call this library.  The
 * CUDA product path never links, imports or executes it, and it shares no
 * code, header or table with that path.
 *
 * Every routine follows the paper's algorithm in its own order and notation
 * (U_k and Q_k are materialised, corrections are summed as printed) with no
 * blocking or reordering.  All arithmetic is IEEE double; the build uses
 * -ffp-contract=off so x86 and Arm produce the same bits.
 *
 * Threads (OpenMP, when the compiler has it): only loops whose iterations
 * write separate outputs run in parallel -- the rows of U_k / Q_k and of a
 * kernel block, the rows of Q alpha and K alpha -- and each output is formed
 * by the same operations in the same order as with one thread, so every
 * result is bit-identical for any thread count (orc_set_threads).  Sums over
 * rows stay sequential.
 *
 * Readings of points the paper leaves open (each listed in the design notes):
 *  - Q = diag(y) K diag(y), as the dual in Section 3.1 defines it (the
 *    Algorithm 1/2 shorthand K(diag(y)A, .) agrees only for the linear kernel
 *    and odd-degree polynomials with c = 0).
 *  - omega = 1/(2C) for K-SVM-L2, nu = C (L1) or +inf (L2), Algorithm 1.
 *  - H counts inner iterations: H coordinate updates (DCD) or H block updates
 *    (BDCD); outer steps = ceil(H/s), the last one shorter when s does not
 *    divide H.
 *  - eta <= 0 (zero row, linear kernel, L1) gives theta = 0.
 *  - Index stream: a counter-based SplitMix64 (Steele, Lea & Flood, OOPSLA
 *    2014).  DCD draws i.i.d. uniform indices; each BDCD block is a uniform
 *    b-subset drawn by Floyd's algorithm (Bentley & Floyd, CACM 1987).
 *  - K-RR system matrix M = K/lambda + m I (Algorithm 3's G_k, eq. krr-problem).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads used by the parallel row loops (1 without OpenMP); returns the
 * count in effect. */
int orc_set_threads(int32_t threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
    return omp_get_max_threads();
#else
    (void)threads;
    return 1;
#endif
}

#define ORC_LINEAR 0
#define ORC_POLY 1
#define ORC_RBF 2

typedef struct {
    int32_t kind;
    int32_t degree; /* polynomial degree d >= 2 (Table 1) */
    double gamma;   /* RBF: exp(-gamma * ||a - b||^2) (Table 1's sigma) */
    double coef0;   /* polynomial: (coef0 + a.b)^d, coef0 >= 0 (Table 1) */
} orc_kernel;

/* ------------------------------------------------------------------ RNG -- */
/* SplitMix64: state advances by the golden-ratio increment, each output is
 * the 64-bit finaliser of the new state.  draw(seed, stream, c) is output
 * number c+1 of the SplitMix64 sequence whose starting state is output number
 * 2*stream+1 of the sequence seeded with `seed`. */
static const uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ULL;

static uint64_t sm_finalise(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output number k >= 1 of SplitMix64 started from `state`. */
uint64_t orc_splitmix64(uint64_t state, uint64_t k)
{
    return sm_finalise(state + k * SM_GAMMA);
}

uint64_t orc_draw(uint64_t seed, uint64_t stream, uint64_t ctr)
{
    return orc_splitmix64(orc_splitmix64(seed, 2 * stream + 1), ctr + 1);
}

/* uniform integer in [0, range): high 64 bits of the 128-bit product */
static uint64_t below(uint64_t u, uint64_t range)
{
    return (uint64_t)(((unsigned __int128)u * (unsigned __int128)range) >> 64);
}

/* DCD coordinate of global iteration t (Algorithm 1: "choose i_k uniformly"). */
int64_t orc_dcd_index(uint64_t seed, int64_t m, uint64_t t)
{
    return (int64_t)below(orc_draw(seed, 0, t), (uint64_t)m);
}

/* BDCD block number t (global, 0-based): b distinct indices, uniformly chosen
 * without replacement (Algorithm 3), by Floyd's algorithm on stream t+1:
 * for q = 0..b-1, J = m-b+q, r = uniform in [0, J]; take r unless already
 * taken, else take J.  Indices are stored in the order they are taken. */
void orc_bdcd_block(uint64_t seed, int64_t m, int32_t b, uint64_t t, int64_t *out)
{
    for (int32_t q = 0; q < b; ++q) {
        int64_t J = m - b + q;
        int64_t r = (int64_t)below(orc_draw(seed, t + 1, (uint64_t)q), (uint64_t)(J + 1));
        int taken = 0;
        for (int32_t p = 0; p < q; ++p)
            if (out[p] == r) { taken = 1; break; }
        out[q] = taken ? J : r;
    }
}

void orc_sample_dcd(uint64_t seed, int64_t m, uint64_t first, int64_t count, int64_t *out)
{
    for (int64_t c = 0; c < count; ++c) out[c] = orc_dcd_index(seed, m, first + (uint64_t)c);
}

void orc_sample_bdcd(uint64_t seed, int64_t m, int32_t b, uint64_t first_block, int64_t nblocks,
                     int64_t *out)
{
    for (int64_t c = 0; c < nblocks; ++c) orc_bdcd_block(seed, m, b, first_block + (uint64_t)c, out + c * b);
}

/* -------------------------------------------------------------- kernels -- */
/* Table 1, by direct definition; the RBF distance is summed from the
 * coordinate differences, not expanded. */
double orc_kernel_eval(const orc_kernel *k, const double *a, const double *b, int64_t n)
{
    if (k->kind == ORC_RBF) {
        double d2 = 0.0;
        for (int64_t c = 0; c < n; ++c) {
            double d = a[c] - b[c];
            d2 += d * d;
        }
        return exp(-k->gamma * d2);
    }
    double dot = 0.0;
    for (int64_t c = 0; c < n; ++c) dot += a[c] * b[c];
    if (k->kind == ORC_LINEAR) return dot;
    double t = k->coef0 + dot, r = t;
    for (int32_t e = 1; e < k->degree; ++e) r *= t;
    return r;
}

/* out[r*nc + c] = K(a_rows[r], a_cols[c]); rows == NULL means all m rows. */
void orc_kernel_block(const orc_kernel *k, const double *A, int64_t m, int64_t n, int64_t lda,
                      const int64_t *rows, int64_t nr, const int64_t *cols, int64_t nc, double *out)
{
    if (rows == NULL) nr = m;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nr; ++r) {
        const double *ar = A + (rows ? rows[r] : r) * lda;
        for (int64_t c = 0; c < nc; ++c) out[r * nc + c] = orc_kernel_eval(k, ar, A + cols[c] * lda, n);
    }
}

/* --------------------------------------------------- small dense solver -- */
/* Solve G x = r for symmetric positive definite G (b x b, row-major) by a
 * Cholesky factorisation G = L L^T; returns 0, or -1 if G is not SPD. */
static int chol_solve(const double *G, int64_t b, const double *r, double *x, double *L)
{
    for (int64_t i = 0; i < b; ++i) {
        for (int64_t j = 0; j <= i; ++j) {
            double s = G[i * b + j];
            for (int64_t p = 0; p < j; ++p) s -= L[i * b + p] * L[j * b + p];
            if (i == j) {
                if (!(s > 0.0)) return -1;
                L[i * b + i] = sqrt(s);
            } else {
                L[i * b + j] = s / L[j * b + j];
            }
        }
    }
    for (int64_t i = 0; i < b; ++i) { /* L z = r */
        double s = r[i];
        for (int64_t p = 0; p < i; ++p) s -= L[i * b + p] * x[p];
        x[i] = s / L[i * b + i];
    }
    for (int64_t i = b - 1; i >= 0; --i) { /* L^T x = z */
        double s = x[i];
        for (int64_t p = i + 1; p < b; ++p) s -= L[p * b + i] * x[p];
        x[i] = s / L[i * b + i];
    }
    return 0;
}

/* --------------------------------------------------------- Algorithm 1 -- */
static void svm_consts(int32_t loss, double C, double *nu, double *omega)
{
    if (loss == 1) { *nu = C; *omega = 0.0; }
    else { *nu = INFINITY; *omega = 1.0 / (2.0 * C); }
}

/* theta for one coordinate (Algorithm 1, projected-gradient test and clipped
 * Newton step; Algorithm 2 uses the same rule with rho for alpha_i). */
static double dcd_theta(double rho, double g, double eta, double nu)
{
    double gt = fabs(fmin(fmax(rho - g, 0.0), nu) - rho);
    if (gt != 0.0 && eta > 0.0) return fmin(fmax(rho - g / eta, 0.0), nu) - rho;
    return 0.0;
}

/* Algorithm 1: DCD for K-SVM-L1 (loss=1) / K-SVM-L2 (loss=2).  H coordinate
 * updates, global iteration counter starting at `first`; alpha is alpha_0 on
 * entry and alpha_H on exit.  Returns 0. */
int orc_dcd_svm(const double *A, int64_t m, int64_t n, int64_t lda, const double *y,
                const orc_kernel *k, int32_t loss, double C, int64_t H, uint64_t seed,
                uint64_t first, double *alpha)
{
    double nu, omega;
    svm_consts(loss, C, &nu, &omega);
    double *u = (double *)malloc(sizeof(double) * (size_t)m);
    if (!u) return -2;
    for (int64_t it = 0; it < H; ++it) {
        int64_t i = orc_dcd_index(seed, m, first + (uint64_t)it);
        /* u_k = Q e_{i_k}: column i of diag(y) K diag(y) */
#pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < m; ++r)
            u[r] = y[r] * y[i] * orc_kernel_eval(k, A + r * lda, A + i * lda, n);
        double eta = u[i] + omega;
        double dot = 0.0;
        for (int64_t r = 0; r < m; ++r) dot += u[r] * alpha[r];
        double g = dot - 1.0 + omega * alpha[i];
        alpha[i] += dcd_theta(alpha[i], g, eta, nu);
    }
    free(u);
    return 0;
}

/* --------------------------------------------------------- Algorithm 2 -- */
/* s-step DCD: per outer step, U_k = Q V_k (m x s), G_k = V_k^T U_k + omega I,
 * then the s thetas sequentially with the unrolled gradient corrections, and
 * one update of alpha.  Same iteration numbering as orc_dcd_svm. */
int orc_sstep_dcd_svm(const double *A, int64_t m, int64_t n, int64_t lda, const double *y,
                      const orc_kernel *k, int32_t loss, double C, int32_t s, int64_t H,
                      uint64_t seed, uint64_t first, double *alpha)
{
    if (s < 1) return -1;
    double nu, omega;
    svm_consts(loss, C, &nu, &omega);
    double *U = (double *)malloc(sizeof(double) * (size_t)m * (size_t)s);
    double *G = (double *)malloc(sizeof(double) * (size_t)s * (size_t)s);
    double *theta = (double *)malloc(sizeof(double) * (size_t)s);
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)s);
    if (!U || !G || !theta || !idx) { free(U); free(G); free(theta); free(idx); return -2; }
    for (int64_t done = 0; done < H; done += s) {
        int64_t cnt = (H - done < s) ? (H - done) : s;
        for (int64_t j = 0; j < cnt; ++j) idx[j] = orc_dcd_index(seed, m, first + (uint64_t)(done + j));
        /* U_k = K(A~, A~_k) with the y_i y_j reading: U[r][j] = Q(r, i_j) */
#pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < m; ++r)
            for (int64_t j = 0; j < cnt; ++j)
                U[r * cnt + j] = y[r] * y[idx[j]] * orc_kernel_eval(k, A + r * lda, A + idx[j] * lda, n);
        /* G_k = V_k^T U_k + omega I */
        for (int64_t t = 0; t < cnt; ++t)
            for (int64_t j = 0; j < cnt; ++j) G[t * cnt + j] = U[idx[t] * cnt + j] + (t == j ? omega : 0.0);
        for (int64_t j = 0; j < cnt; ++j) {
            double eta = G[j * cnt + j];
            double rho = alpha[idx[j]];
            for (int64_t t = 0; t < j; ++t)
                if (idx[t] == idx[j]) rho += theta[t];
            double dot = 0.0;
            for (int64_t r = 0; r < m; ++r) dot += U[r * cnt + j] * alpha[r];
            double g = dot - 1.0 + omega * alpha[idx[j]];
            for (int64_t t = 0; t < j; ++t) g += U[idx[t] * cnt + j] * theta[t];
            for (int64_t t = 0; t < j; ++t)
                if (idx[t] == idx[j]) g += omega * theta[t];
            theta[j] = dcd_theta(rho, g, eta, nu);
        }
        for (int64_t t = 0; t < cnt; ++t) alpha[idx[t]] += theta[t];
    }
    free(U); free(G); free(theta); free(idx);
    return 0;
}

/* --------------------------------------------------------- Algorithm 3 -- */
/* BDCD for K-RR: H block updates of size b, global block counter from
 * `first_block`.  Returns 0, or -1 if some G_k is not SPD. */
int orc_bdcd_krr(const double *A, int64_t m, int64_t n, int64_t lda, const double *y,
                 const orc_kernel *k, double lambda, int32_t b, int64_t H, uint64_t seed,
                 uint64_t first_block, double *alpha)
{
    if (b < 1 || b > m) return -1;
    double *U = (double *)malloc(sizeof(double) * (size_t)m * (size_t)b);
    double *G = (double *)malloc(sizeof(double) * (size_t)b * (size_t)b);
    double *L = (double *)malloc(sizeof(double) * (size_t)b * (size_t)b);
    double *rhs = (double *)malloc(sizeof(double) * (size_t)b);
    double *d = (double *)malloc(sizeof(double) * (size_t)b);
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)b);
    int rc = 0;
    if (!U || !G || !L || !rhs || !d || !idx) rc = -2;
    for (int64_t it = 0; rc == 0 && it < H; ++it) {
        orc_bdcd_block(seed, m, b, first_block + (uint64_t)it, idx);
#pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < m; ++r) /* U_k = K(A, V_k^T A) */
            for (int32_t p = 0; p < b; ++p)
                U[r * b + p] = orc_kernel_eval(k, A + r * lda, A + idx[p] * lda, n);
        for (int32_t p = 0; p < b; ++p) /* G_k = V_k^T U_k / lambda + m I */
            for (int32_t q = 0; q < b; ++q)
                G[p * b + q] = U[idx[p] * b + q] / lambda + (p == q ? (double)m : 0.0);
        for (int32_t p = 0; p < b; ++p) {
            double ua = 0.0;
            for (int64_t r = 0; r < m; ++r) ua += U[r * b + p] * alpha[r];
            rhs[p] = y[idx[p]] - (double)m * alpha[idx[p]] - ua / lambda;
        }
        if (chol_solve(G, b, rhs, d, L) != 0) { rc = -1; break; }
        for (int32_t p = 0; p < b; ++p) alpha[idx[p]] += d[p];
    }
    free(U); free(G); free(L); free(rhs); free(d); free(idx);
    return rc;
}

/* --------------------------------------------------------- Algorithm 4 -- */
/* s-step BDCD: per outer step Q_k = K(A, Omega_k^T A) (m x sb); for
 * j = 1..s the b x b system of eq. (bdcd-sstep) with the m V^T V and
 * (1/lambda) U^T V correction sums; one alpha update at the end. */
int orc_sstep_bdcd_krr(const double *A, int64_t m, int64_t n, int64_t lda, const double *y,
                       const orc_kernel *k, double lambda, int32_t b, int32_t s, int64_t H,
                       uint64_t seed, uint64_t first_block, double *alpha)
{
    if (b < 1 || b > m || s < 1) return -1;
    int64_t sb = (int64_t)s * b;
    double *Q = (double *)malloc(sizeof(double) * (size_t)m * (size_t)sb);
    double *G = (double *)malloc(sizeof(double) * (size_t)b * (size_t)b);
    double *L = (double *)malloc(sizeof(double) * (size_t)b * (size_t)b);
    double *rhs = (double *)malloc(sizeof(double) * (size_t)b);
    double *D = (double *)malloc(sizeof(double) * (size_t)sb);
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)sb);
    int rc = 0;
    if (!Q || !G || !L || !rhs || !D || !idx) rc = -2;
    for (int64_t done = 0; rc == 0 && done < H; done += s) {
        int64_t cnt = (H - done < s) ? (H - done) : s;
        int64_t w = cnt * b; /* columns of Q_k this outer step */
        for (int64_t j = 0; j < cnt; ++j)
            orc_bdcd_block(seed, m, b, first_block + (uint64_t)(done + j), idx + j * b);
#pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < m; ++r)
            for (int64_t c = 0; c < w; ++c) Q[r * w + c] = orc_kernel_eval(k, A + r * lda, A + idx[c] * lda, n);
        for (int64_t j = 0; j < cnt; ++j) {
            const int64_t *vj = idx + j * b; /* V_{sk+j}; U_{sk+j} = Q_k columns jb..jb+b-1 */
            for (int32_t p = 0; p < b; ++p)
                for (int32_t q = 0; q < b; ++q)
                    G[p * b + q] = Q[vj[p] * w + j * b + q] / lambda + (p == q ? (double)m : 0.0);
            for (int32_t p = 0; p < b; ++p) {
                double v = y[vj[p]] - (double)m * alpha[vj[p]];
                double corr_m = 0.0; /* sum_t V_j^T V_t Delta_t */
                for (int64_t t = 0; t < j; ++t)
                    for (int32_t q = 0; q < b; ++q)
                        if (idx[t * b + q] == vj[p]) corr_m += D[t * b + q];
                v -= (double)m * corr_m;
                double ua = 0.0; /* U_j^T alpha_sk */
                for (int64_t r = 0; r < m; ++r) ua += Q[r * w + j * b + p] * alpha[r];
                v -= ua / lambda;
                double corr_u = 0.0; /* sum_t U_j^T V_t Delta_t */
                for (int64_t t = 0; t < j; ++t)
                    for (int32_t q = 0; q < b; ++q) corr_u += Q[idx[t * b + q] * w + j * b + p] * D[t * b + q];
                v -= corr_u / lambda;
                rhs[p] = v;
            }
            if (chol_solve(G, b, rhs, D + j * b, L) != 0) { rc = -1; break; }
        }
        if (rc != 0) break;
        for (int64_t c = 0; c < w; ++c) alpha[idx[c]] += D[c];
    }
    free(Q); free(G); free(L); free(rhs); free(D); free(idx);
    return rc;
}

/* ------------------------------------------------ objectives and checks -- */
/* (Q alpha)_i = y_i sum_j y_j K(a_i, a_j) alpha_j, by direct summation. */
static void svm_q_alpha(const double *A, int64_t m, int64_t n, int64_t lda, const double *y,
                        const orc_kernel *k, const double *alpha, double *qa)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < m; ++j)
            if (alpha[j] != 0.0) s += y[j] * alpha[j] * orc_kernel_eval(k, A + i * lda, A + j * lda, n);
        qa[i] = y[i] * s;
    }
}

/* K-SVM gradient of the minimisation-form dual, g = Q alpha - 1 + omega alpha. */
int orc_svm_gradient(const double *A, int64_t m, int64_t n, int64_t lda, const double *y,
                     const orc_kernel *k, int32_t loss, double C, const double *alpha, double *g)
{
    double nu, omega;
    svm_consts(loss, C, &nu, &omega);
    svm_q_alpha(A, m, n, lda, y, k, alpha, g);
    for (int64_t i = 0; i < m; ++i) g[i] += -1.0 + omega * alpha[i];
    return 0;
}

/* out[0] = primal P(w(alpha)), out[1] = dual D(alpha) in maximisation form,
 * out[2] = P - D, out[3] = sum of KKT violations.
 *   P = 1/2 a^T Q a + C sum max(0, 1 - (Qa)_i)      (L1, eq. softsvm)
 *   P = 1/2 a^T Q a + C sum max(0, 1 - (Qa)_i)^2    (L2)
 *   D = 1^T a - 1/2 a^T Q a [- ||a||^2/(4C) for L2] (Section 3.1 duals) */
int orc_svm_objectives(const double *A, int64_t m, int64_t n, int64_t lda, const double *y,
                       const orc_kernel *k, int32_t loss, double C, const double *alpha, double *out)
{
    double *qa = (double *)malloc(sizeof(double) * (size_t)m);
    if (!qa) return -2;
    svm_q_alpha(A, m, n, lda, y, k, alpha, qa);
    double aqa = 0.0, sa = 0.0, sa2 = 0.0, hinge = 0.0, kkt = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        aqa += alpha[i] * qa[i];
        sa += alpha[i];
        sa2 += alpha[i] * alpha[i];
        double xi = fmax(0.0, 1.0 - qa[i]);
        hinge += (loss == 1) ? xi : xi * xi;
        if (loss == 1) {
            double viol = 0.0;
            if (alpha[i] <= 0.0) viol = fmax(0.0, 1.0 - qa[i]);
            else if (alpha[i] >= C) viol = fmax(0.0, qa[i] - 1.0);
            else viol = fabs(qa[i] - 1.0);
            kkt += viol;
        } else {
            double gi = qa[i] + alpha[i] / (2.0 * C) - 1.0;
            kkt += (alpha[i] > 0.0) ? fabs(gi) : fmax(0.0, -gi);
        }
    }
    double P = 0.5 * aqa + C * hinge;
    double D = sa - 0.5 * aqa - ((loss == 2) ? sa2 / (4.0 * C) : 0.0);
    out[0] = P;
    out[1] = D;
    out[2] = P - D;
    out[3] = kkt;
    free(qa);
    return 0;
}

/* K-RR gradient of eq. (krr-problem): g = (1/lambda) K alpha + m alpha - y. */
int orc_krr_gradient(const double *A, int64_t m, int64_t n, int64_t lda, const double *y,
                     const orc_kernel *k, double lambda, const double *alpha, double *g)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < m; ++j)
            if (alpha[j] != 0.0) s += orc_kernel_eval(k, A + i * lda, A + j * lda, n) * alpha[j];
        g[i] = s / lambda + (double)m * alpha[i] - y[i];
    }
    return 0;
}

/* K-RR dual objective 1/2 a^T (K/lambda + m I) a - y^T a (eq. krr-problem). */
double orc_krr_objective(const double *A, int64_t m, int64_t n, int64_t lda, const double *y,
                         const orc_kernel *k, double lambda, const double *alpha)
{
    double *ka = (double *)malloc(sizeof(double) * (size_t)m); /* (K alpha)_i */
    if (!ka) return NAN;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < m; ++j)
            if (alpha[j] != 0.0) s += orc_kernel_eval(k, A + i * lda, A + j * lda, n) * alpha[j];
        ka[i] = s;
    }
    double quad = 0.0, lin = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        quad += alpha[i] * (ka[i] / lambda + (double)m * alpha[i]);
        lin += y[i] * alpha[i];
    }
    free(ka);
    return 0.5 * quad - lin;
}

/* Closed form of K-RR (Section 5.1's alpha*): solve (K/lambda + m I) a = y by
 * a dense Cholesky factorisation of the full m x m matrix.  Returns 0, -1 if
 * not SPD, -2 on allocation failure. */
int orc_krr_closed_form(const double *A, int64_t m, int64_t n, int64_t lda, const double *y,
                        const orc_kernel *k, double lambda, double *alpha)
{
    double *M = (double *)malloc(sizeof(double) * (size_t)m * (size_t)m);
    double *L = (double *)malloc(sizeof(double) * (size_t)m * (size_t)m);
    if (!M || !L) { free(M); free(L); return -2; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < m; ++j)
            M[i * m + j] = orc_kernel_eval(k, A + i * lda, A + j * lda, n) / lambda + (i == j ? (double)m : 0.0);
    int rc = chol_solve(M, m, y, alpha, L);
    free(M); free(L);
    return rc;
}
