/*
 * mcinv_oracle.c -- FP64 CPU oracle of the correlated-chains (CC) sampler of
 * Garcia-Cortes & Cabrillo, "A Monte Carlo algorithm for efficient large matrix
 * inversion" (Sec. 2, Eqs. 4, 5, 5a, 5b, Eq. 1/C, Eq. tr, Algorithm 1).
 *
 * TEST INFRASTRUCTURE.  This file is the slow, obviously correct statement of
 * what the CUDA library computes.  Only the tests, the package smoke check and
 * the benchmark's CPU-baseline leg may build, load or call it.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * Arithmetic is C99 double complex throughout; a real matrix is carried with
 * zero imaginary parts (products with exact zeros stay exact).
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *  - Noise: Z2 (+-1) noise, the kind the paper prefers (Sec. 1); it satisfies
 *    Eqs. 5a/5b.  The same phi_i^(k) feeds Eq. 4 and Eq. 5 (Sec. 2).
 *  - phi is drawn from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 *    random numbers: as easy as 1, 2, 3", SC'11) with key (seed lo, seed hi)
 *    and counter (row >> 7, chain, cycle, matrix); the sign is bit (row & 31)
 *    of output word ((row >> 5) & 3): bit 1 -> phi = -1.
 *  - 1/sqrt(c*_ii) in Eq. 5 is read as beta_i = 1/conj(sqrt(c_ii)) with the
 *    principal square root, so that alpha_i * conj(beta_i) = 1/c_ii, which is
 *    what the demonstration (Eqs. Theta, Gamma, series) needs.  For a matrix
 *    given in real storage with c_ii < 0 the real reading alpha = 1/sqrt|c|,
 *    beta = -1/sqrt|c| is used (same product 1/c_ii, real arithmetic).
 *  - Trace: the estimator is read as sum_i q_i z_i conj(w_i) (i.e. w^dagger Q z
 *    for diagonal Q), the reading consistent with Eq. 1/C; Eq. tr prints
 *    z^dagger Q w, which for complex C is its complex conjugate.
 *  - Cycles are counted from 0 in one global counter shared by burn-in and
 *    sampling; samples are the states after cycles N..M-1 (M-N samples, Eq. 1/C).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (SC'11, Sec. 4 of Salmon et al.): a 10-round Feistel-like     */
/* bijection on four 32-bit words built from two 32x32->64 multiplications,    */
/* with a Weyl sequence bumping the two key words between rounds.              */
/* ------------------------------------------------------------------------- */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u /* golden ratio */
#define ORC_PHILOX_W1 0xBB67AE85u /* sqrt(3) - 1 */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* phi_row^(cycle) of chain `chain` of matrix `matrix`: +1 or -1 (Eqs. 5a/5b). */
int orc_phi(uint64_t seed, uint32_t matrix, uint32_t chain, uint32_t cycle, uint32_t row)
{
    uint32_t ctr[4] = {row >> 7, chain, cycle, matrix};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    uint32_t bit = (out[(row >> 5) & 3u] >> (row & 31u)) & 1u;
    return bit ? -1 : 1;
}

/* The noise of every row and of chains chain0 .. chain0+K-1 in one cycle:
 * out[i*K + c] = phi(seed, matrix, chain0 + c, cycle, i). */
void orc_noise_plane(int64_t n, int64_t K, uint64_t seed, uint32_t matrix, uint32_t chain0, uint32_t cycle,
                     int8_t *out)
{
    for (int64_t i = 0; i < n; ++i)
        for (int64_t c = 0; c < K; ++c)
            out[i * K + c] = (int8_t)orc_phi(seed, matrix, chain0 + (uint32_t)c, cycle, (uint32_t)i);
}

/* ------------------------------------------------------------------------- */
/* Problem: a CSR matrix C with its diagonal present.                          */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t n;
    const int64_t *row_ptr; /* [n+1] */
    const int32_t *col;     /* [nnz], strictly increasing within a row */
    const double *val;      /* [nnz] real, or [2*nnz] interleaved re,im */
    int is_complex;
} orc_matrix;

static cplx orc_entry(const orc_matrix *m, int64_t e)
{
    return m->is_complex ? (m->val[2 * e] + I * m->val[2 * e + 1]) : (cplx)m->val[e];
}

/*
 * Per-row constants of Eqs. 4 and 5: inv_d = 1/c_ii, alpha = 1/sqrt(c_ii),
 * beta = 1/sqrt(c*_ii) read as 1/conj(sqrt(c_ii)).  Returns 0, or -1-i when
 * row i has no diagonal, or a zero / non-finite one (D must be non-singular,
 * Sec. 2.2).
 */
int64_t orc_row_constants(int64_t n, const int64_t *row_ptr, const int32_t *col,
                          const double *val, int is_complex,
                          double *alpha, double *beta, double *inv_d /* each [2n] re,im */)
{
    orc_matrix m = {n, row_ptr, col, val, is_complex};
    for (int64_t i = 0; i < n; ++i) {
        int found = 0;
        cplx cii = 0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (col[e] == i) { cii = orc_entry(&m, e); found = 1; }
        if (!found || cii == 0 || !isfinite(creal(cii)) || !isfinite(cimag(cii)))
            return -1 - i;
        cplx a, b;
        if (!is_complex) {
            double r = sqrt(fabs(creal(cii)));
            a = 1.0 / r;
            b = (creal(cii) > 0 ? 1.0 : -1.0) / r;
        } else {
            cplx s = csqrt(cii); /* principal branch */
            a = 1.0 / s;
            b = 1.0 / conj(s);
        }
        cplx d = 1.0 / cii;
        alpha[2 * i] = creal(a); alpha[2 * i + 1] = cimag(a);
        beta[2 * i] = creal(b);  beta[2 * i + 1] = cimag(b);
        inv_d[2 * i] = creal(d); inv_d[2 * i + 1] = cimag(d);
    }
    return 0;
}

/* Column access to C (needed by Eq. 5, which runs down column i of C). */
typedef struct {
    int64_t *col_ptr;  /* [n+1] */
    int64_t *row_idx;  /* [nnz] */
    int64_t *entry;    /* [nnz] index of the entry in the CSR arrays */
} orc_columns;

static int orc_build_columns(const orc_matrix *m, orc_columns *c)
{
    int64_t n = m->n, nnz = m->row_ptr[n];
    c->col_ptr = calloc((size_t)n + 1, sizeof(int64_t));
    c->row_idx = malloc((size_t)(nnz ? nnz : 1) * sizeof(int64_t));
    c->entry = malloc((size_t)(nnz ? nnz : 1) * sizeof(int64_t));
    if (!c->col_ptr || !c->row_idx || !c->entry) return -1;
    for (int64_t e = 0; e < nnz; ++e) c->col_ptr[m->col[e] + 1]++;
    for (int64_t j = 0; j < n; ++j) c->col_ptr[j + 1] += c->col_ptr[j];
    int64_t *fill = malloc((size_t)n * sizeof(int64_t) + 1);
    if (!fill) return -1;
    memcpy(fill, c->col_ptr, (size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) /* rows ascending: each column's rows come out sorted */
        for (int64_t e = m->row_ptr[i]; e < m->row_ptr[i + 1]; ++e) {
            int64_t p = fill[m->col[e]]++;
            c->row_idx[p] = i;
            c->entry[p] = e;
        }
    free(fill);
    return 0;
}

static void orc_free_columns(orc_columns *c)
{
    free(c->col_ptr); free(c->row_idx); free(c->entry);
}

/*
 * One CC cycle (Eqs. 4 and 5) for one chain, in place, rows i = 0..n-1
 * ascending.  z and w are strided views: element i lives at z[i*stride].
 * In-place storage makes z_j (j < i) the cycle-k value and z_j (j > i) the
 * cycle-(k-1) value, exactly as Eq. 4 prescribes; likewise for w in Eq. 5.
 */
static void orc_cycle_one_chain(const orc_matrix *m, const orc_columns *cols,
                                const cplx *alpha, const cplx *beta, const cplx *inv_d,
                                uint64_t seed, uint32_t matrix, uint32_t chain, uint32_t cycle,
                                cplx *z, cplx *w, int64_t stride)
{
    for (int64_t i = 0; i < m->n; ++i) {
        double phi = (double)orc_phi(seed, matrix, chain, cycle, (uint32_t)i);
        /* Eq. 4: z_i = phi_i/sqrt(c_ii) - (1/c_ii) sum_{j<i} c_ij z_j^(k)
                                         - (1/c_ii) sum_{j>i} c_ij z_j^(k-1) */
        cplx lower = 0, upper = 0;
        for (int64_t e = m->row_ptr[i]; e < m->row_ptr[i + 1]; ++e) {
            int64_t j = m->col[e];
            if (j < i) lower += orc_entry(m, e) * z[j * stride];
            else if (j > i) upper += orc_entry(m, e) * z[j * stride];
        }
        z[i * stride] = phi * alpha[i] - inv_d[i] * lower - inv_d[i] * upper;
        /* Eq. 5: w_i = phi_i/sqrt(c*_ii) - (1/c*_ii) sum_{j<i} c*_ji w_j^(k)
                                          - (1/c*_ii) sum_{j>i} c*_ji w_j^(k-1) */
        cplx wl = 0, wu = 0;
        for (int64_t p = cols->col_ptr[i]; p < cols->col_ptr[i + 1]; ++p) {
            int64_t j = cols->row_idx[p];
            cplx cji = orc_entry(m, cols->entry[p]);
            if (j < i) wl += conj(cji) * w[j * stride];
            else if (j > i) wu += conj(cji) * w[j * stride];
        }
        w[i * stride] = phi * beta[i] - conj(inv_d[i]) * wl - conj(inv_d[i]) * wu;
    }
}

/*
 * Run chains [0, K) (global ids chain0 + c) for cycles cycle0 .. cycle0+ncycles-1.
 *
 * z, w      : state, [n][K] interleaved re,im (2*n*K doubles), updated in place.
 * acc_from  : cycles with global index >= acc_from are accumulated (Eq. 1/C).
 * cpg       : chains per group; group g = c / cpg; G = ceil(K / cpg).
 * diag_acc  : [G][n] interleaved, += sum over the group's chains of z_i conj(w_i);
 *             may be NULL.
 * blk_acc   : [G][nR][nS] interleaved, += z_{R[a]} conj(w_{S[b]}); may be NULL.
 * q, tser   : if both set, tser[g][k] += sum_i q_i Re(z_i conj(w_i)) over the group's
 *             chains for every accumulated cycle k (k counted from acc_from): the
 *             realised trace values whose Monte Carlo error Sec. 2.3 estimates.
 * threads   : OpenMP threads over groups (1 = serial); groups are independent.
 *
 * Returns 0, or a negative row index - 1 if D is singular.
 */
int64_t orc_cc_run(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                   int is_complex, int64_t K, int64_t chain0, uint64_t seed, uint32_t matrix,
                   int64_t cycle0, int64_t ncycles, int64_t acc_from,
                   double *z, double *w, int64_t cpg,
                   double *diag_acc, const int64_t *R, int64_t nR, const int64_t *S, int64_t nS,
                   double *blk_acc, const double *q, double *tser, int threads)
{
    orc_matrix m = {n, row_ptr, col, val, is_complex};
    double *abuf = malloc(sizeof(double) * 6 * (size_t)(n ? n : 1));
    if (!abuf) return -(1LL << 62);
    int64_t bad = orc_row_constants(n, row_ptr, col, val, is_complex, abuf, abuf + 2 * n, abuf + 4 * n);
    if (bad) { free(abuf); return bad; }
    cplx *alpha = malloc(sizeof(cplx) * (size_t)(n ? n : 1));
    cplx *beta = malloc(sizeof(cplx) * (size_t)(n ? n : 1));
    cplx *inv_d = malloc(sizeof(cplx) * (size_t)(n ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        alpha[i] = abuf[2 * i] + I * abuf[2 * i + 1];
        beta[i] = abuf[2 * n + 2 * i] + I * abuf[2 * n + 2 * i + 1];
        inv_d[i] = abuf[4 * n + 2 * i] + I * abuf[4 * n + 2 * i + 1];
    }
    free(abuf);
    orc_columns cols;
    orc_build_columns(&m, &cols);

    cplx *Z = (cplx *)z, *Wv = (cplx *)w;
    cplx *DA = (cplx *)diag_acc, *BA = (cplx *)blk_acc;
    int64_t G = (K + cpg - 1) / cpg;
#ifdef _OPENMP
    if (threads < 1) threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
#endif
    for (int64_t g = 0; g < G; ++g) {
        int64_t c_end = (g + 1) * cpg < K ? (g + 1) * cpg : K;
        for (int64_t c = g * cpg; c < c_end; ++c) {
            /* Algorithm 1, steps 6-8, for one chain pair (z, w). */
            for (int64_t k = 0; k < ncycles; ++k) {
                int64_t cyc = cycle0 + k;
                orc_cycle_one_chain(&m, &cols, alpha, beta, inv_d, seed, matrix,
                                    (uint32_t)(chain0 + c), (uint32_t)cyc, Z + c, Wv + c, K);
                if (cyc < acc_from) continue;
                if (q && tser) {
                    /* cycles of this call that are accumulated: first .. cycle0+ncycles-1 */
                    const int64_t first = acc_from > cycle0 ? acc_from : cycle0;
                    double t = 0.0;
                    for (int64_t i = 0; i < n; ++i) t += q[i] * creal(Z[i * K + c] * conj(Wv[i * K + c]));
                    tser[g * (cycle0 + ncycles - first) + (cyc - first)] += t;
                }
                if (DA)
                    for (int64_t i = 0; i < n; ++i)
                        DA[g * n + i] += Z[i * K + c] * conj(Wv[i * K + c]);
                if (BA)
                    for (int64_t a = 0; a < nR; ++a)
                        for (int64_t b = 0; b < nS; ++b)
                            BA[(g * nR + a) * nS + b] += Z[R[a] * K + c] * conj(Wv[S[b] * K + c]);
            }
        }
    }
    orc_free_columns(&cols);
    free(alpha); free(beta); free(inv_d);
    return 0;
}

/*
 * Coupling run of Algorithm 1, steps 1-5, for one chain: paths (z, w) from 0
 * and (z*, w*) from z*_i = w*_i = i+1 (the paper's 1-based "i"), same noise.
 * Returns the number of cycles p after which max_i |z_i - z*_i| < tol and
 * max_i |w_i - w*_i| < tol (the garbled "z'z* < tol" of step 5 read as this
 * sup-norm), or -1 if that does not happen within max_cycles.  The final
 * states are left in z, w (length-n interleaved vectors).
 */
int64_t orc_coupling_burnin(int64_t n, const int64_t *row_ptr, const int32_t *col,
                            const double *val, int is_complex, uint64_t seed, uint32_t matrix,
                            uint32_t chain, double tol, int64_t max_cycles,
                            double *z, double *w)
{
    orc_matrix m = {n, row_ptr, col, val, is_complex};
    double *abuf = malloc(sizeof(double) * 6 * (size_t)(n ? n : 1));
    if (orc_row_constants(n, row_ptr, col, val, is_complex, abuf, abuf + 2 * n, abuf + 4 * n)) {
        free(abuf);
        return -2;
    }
    cplx *alpha = malloc(sizeof(cplx) * (size_t)n), *beta = malloc(sizeof(cplx) * (size_t)n);
    cplx *inv_d = malloc(sizeof(cplx) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        alpha[i] = abuf[2 * i] + I * abuf[2 * i + 1];
        beta[i] = abuf[2 * n + 2 * i] + I * abuf[2 * n + 2 * i + 1];
        inv_d[i] = abuf[4 * n + 2 * i] + I * abuf[4 * n + 2 * i + 1];
    }
    free(abuf);
    orc_columns cols;
    orc_build_columns(&m, &cols);
    cplx *Z = (cplx *)z, *Wv = (cplx *)w;
    cplx *zs = malloc(sizeof(cplx) * (size_t)n), *ws = malloc(sizeof(cplx) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) { Z[i] = 0; Wv[i] = 0; zs[i] = (double)(i + 1); ws[i] = (double)(i + 1); }
    int64_t p = 0, result = -1;
    while (p < max_cycles) {
        orc_cycle_one_chain(&m, &cols, alpha, beta, inv_d, seed, matrix, chain, (uint32_t)p, Z, Wv, 1);
        orc_cycle_one_chain(&m, &cols, alpha, beta, inv_d, seed, matrix, chain, (uint32_t)p, zs, ws, 1);
        ++p;
        double dz = 0, dw = 0;
        for (int64_t i = 0; i < n; ++i) {
            double a = cabs(Z[i] - zs[i]), b = cabs(Wv[i] - ws[i]);
            if (a > dz) dz = a;
            if (b > dw) dw = b;
        }
        if (dz < tol && dw < tol) { result = p; break; }
    }
    free(zs); free(ws);
    orc_free_columns(&cols);
    free(alpha); free(beta); free(inv_d);
    return result;
}
