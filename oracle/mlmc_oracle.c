/*
 * CPU oracle for the multilevel Monte Carlo estimator of x = exp(beta A) u
 * (Acebron, Herrero, Monteiro, "A highly parallel algorithm for computing the
 * action of a matrix exponential on a vector based on a multilevel Monte Carlo
 * method").
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, written to be checked against the
 * paper by eye.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load it.  It shares no code with the GPU library.
 *
 * Contents
 *   - Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11).
 *   - neglog: -ln(u) after reducing u to m 2^e, m in [sqrt(1/2), sqrt(2)):
 *     FP64 by the series ln m = 2 atanh((m-1)/(m+1)), FP32 by a fitted
 *     polynomial in m - 1, written out so that both sides of a replay
 *     comparison make identical decisions.
 *   - The splitting A = D - T of Sec. 2.1 (Eq. 1): a_ii, L_ii, d_i.
 *   - Per-row Vose alias tables for the jump law k_ij = |a_ij| / L_ii
 *     (Sec. 3, Eq. 12).
 *   - The walk of Algorithm 2 (MLMCL), one interval of length Delta t_l at a
 *     time, with the coupled fine (eta_2) and coarse (eta_1) weights, plus the
 *     paired-step form of Eq. 7 (Lemma 2's xi_j) for an accurate difference.
 *
 * Readings of the paper taken here (the GPU path makes the same ones):
 *   R1  every holding time uses the rate L_jj of the state being occupied
 *       (the CTMC of Eq. 12); the listing draws S before the new state is
 *       chosen, which read literally uses the old state's rate.  Variant
 *       ORC_LITERAL_RATE reproduces that literal reading for comparison.
 *   R2  one exponential clock per holding segment, carried across interval
 *       boundaries (equal in law to redrawing tau at each interval, by
 *       memorylessness).  Variant ORC_REDRAW redraws per interval as the
 *       listing does.
 *   R3  scaled time s = tau/beta in [0,1]: rate beta*L_jj, grid points k/N.
 *       A jump at exactly s = k/N happens after grid point k is sampled; a
 *       jump at s >= 1 is not taken.
 *   R19 (not in the paper) a proposal may change with time: K equal pieces
 *       [p/K, (p+1)/K) of s, each with its own rates, jump law and d_i
 *       (orc_ctx.pieces).  A holding time that reaches the piece's end b is
 *       carried into the next piece by memorylessness: the pending jump time
 *       s becomes b + (s - b) * inv_rate_next / inv_rate_now (one fused
 *       multiply-add after the quotient; infinite when either inverse rate
 *       is), which is the unused part of the exponential at the new rate.
 *       The grid's integrand takes each interval's own piece at both of its
 *       ends, so a grid point on a piece boundary gets the mean of the two
 *       pieces' values (the trapezoid of each piece); N must be a multiple
 *       of K on every level walked.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (FMA contraction
 * must be off so that every rounding is the IEEE one written here).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                       */
/* ------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------ */
/* Uniforms and -ln(u)                                                 */
/* ------------------------------------------------------------------ */
/* u = (2k+1) 2^-53 with k the top 52 bits of (x0:x1): exact, in (0,1). */
double orc_uniform64(uint32_t x0, uint32_t x1)
{
    uint64_t w = ((uint64_t)x0 << 32) | (uint64_t)x1;
    return (double)((w >> 11) | 1ull) * 0x1p-53;
}

/* u = (2k+1) 2^-24 with k the top 23 bits of x0: exact, in (0,1). */
float orc_uniform32(uint32_t x0)
{
    return (float)((x0 >> 8) | 1u) * 0x1p-24f;
}

/* ln 2 split so that e*LN2_HI is exact for |e| < 2^11 (FP64) or 2^8 (FP32). */
static const double ORC_LN2_HI64 = 0x1.62e42fefa3800p-1;
static const double ORC_LN2_LO64 = 0x1.ef35793c76730p-45;
static const float ORC_LN2_HI32 = 0x1.62e400p-1f;
static const float ORC_LN2_LO32 = 0x1.7f7d1cp-20f;
static const double ORC_SQRT_HALF64 = 0x1.6a09e667f3bcdp-1;
static const float ORC_SQRT_HALF32 = 0x1.6a09e6p-1f;

#define ORC_NEGLOG_TERMS64 12
static double orc_c64[ORC_NEGLOG_TERMS64];
static int orc_coeffs_ready = 0;

static void orc_init_coeffs(void)
{
    if (orc_coeffs_ready) return;
    for (int k = 0; k < ORC_NEGLOG_TERMS64; ++k) orc_c64[k] = 1.0 / (double)(2 * k + 1);
    orc_coeffs_ready = 1;
}

/* FP32: ln(1+f) = f + f^2 Q(f) for f = m - 1 in [sqrt(1/2) - 1, sqrt(2) - 1],
 * Q of degree 8 with these FP32 coefficients (constant term first): the
 * FP64 least-squares fit of the relative error of f + f^2 Q(f) against
 * ln(1+f) on 1000 Chebyshev (Gauss) points of the interval, each rounded to
 * FP32 (oracle/fit_neglog32.py computes them).  They define the FP32 -ln(u)
 * of this implementation (reading R4).  With fused
 * multiply-adds the result is within 0.87 ulp of -ln(u) and strictly
 * decreasing over all 2^23 FP32 uniforms (both checked exhaustively by the
 * tests). */
#define ORC_NEGLOG_DEG32 8
static const float orc_q32[ORC_NEGLOG_DEG32 + 1] = {
    -0x1.fffff8p-2f, 0x1.555558p-2f, -0x1.000422p-2f, 0x1.999fc2p-3f, -0x1.5424e0p-3f,
    0x1.22bf86p-3f, -0x1.0f9b0cp-3f, 0x1.068b2ap-3f, -0x1.321a4cp-4f};

/* -ln(u) for normal u in (0,1).  u = m 2^e with m in [sqrt(1/2), sqrt(2));
 * ln m = 2 z (1 + z^2/3 + z^4/5 + ...), z = (m-1)/(m+1), |z| <= 0.1716,
 * 12 terms (FP64).  ln u = e ln2 + ln m. */
double orc_neglog64(double u)
{
    orc_init_coeffs();
    uint64_t b;
    memcpy(&b, &u, sizeof b);
    int e = (int)((b >> 52) & 0x7ff) - 1022;
    b = (b & 0x000fffffffffffffull) | (0x3feull << 52);
    double m;
    memcpy(&m, &b, sizeof m);
    if (m < ORC_SQRT_HALF64) {
        m = m * 2.0;
        e = e - 1;
    }
    double z = (m - 1.0) / (m + 1.0);
    double z2 = z * z;
    double p = orc_c64[ORC_NEGLOG_TERMS64 - 1];
    for (int k = ORC_NEGLOG_TERMS64 - 2; k >= 0; --k) p = p * z2 + orc_c64[k];
    double lnm = (2.0 * z) * p;
    double lnu = (double)e * ORC_LN2_HI64 + ((double)e * ORC_LN2_LO64 + lnm);
    return -lnu;
}

/* FP32 version: the same range reduction; ln m = f + f^2 Q(f), f = m - 1
 * (exact), Q by Horner's rule with fused multiply-adds (fmaf rounds once). */
float orc_neglog32(float u)
{
    uint32_t b;
    memcpy(&b, &u, sizeof b);
    int e = (int)((b >> 23) & 0xff) - 126;
    b = (b & 0x007fffffu) | (0x7eu << 23);
    float m;
    memcpy(&m, &b, sizeof m);
    if (m < ORC_SQRT_HALF32) {
        m = m * 2.0f;
        e = e - 1;
    }
    float f = m - 1.0f;
    float q = orc_q32[ORC_NEGLOG_DEG32];
    for (int k = ORC_NEGLOG_DEG32 - 1; k >= 0; --k) q = fmaf(q, f, orc_q32[k]);
    float lnm = fmaf(f * f, q, f);
    float ef = (float)e;
    float lnu = fmaf(ef, ORC_LN2_HI32, fmaf(ef, ORC_LN2_LO32, lnm));
    return -lnu;
}

void orc_neglog64_batch(const double *u, double *out, int64_t count)
{
    for (int64_t i = 0; i < count; ++i) out[i] = orc_neglog64(u[i]);
}

void orc_neglog32_batch(const float *u, float *out, int64_t count)
{
    for (int64_t i = 0; i < count; ++i) out[i] = orc_neglog32(u[i]);
}

/* ------------------------------------------------------------------ */
/* Splitting A = D - T (Sec. 2.1, Eq. 1)                               */
/* ------------------------------------------------------------------ */
/* Per row i, scanning the CSR row in stored order:
 *   a_ii   = the diagonal entry (0 if absent)
 *   L_ii   = sum_{j != i} |a_ij|      (FP64, left to right)
 *   deg_i  = number of stored off-diagonal entries
 *   d_i    = a_ii + L_ii
 * and the scaled quantities used by the walk in scaled time s = tau/t:
 *   rate_i = t L_ii,   dl_i = t d_i,   inv_rate_i = 1/rate_i (inf if 0),
 *   inv_rate32_i = (float)inv_rate_i,  dl32_i = (float)dl_i.            */
int orc_split(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
              double t, double *a_ii, double *L, int32_t *deg, double *dl,
              double *inv_rate, float *inv_rate32, float *dl32)
{
    for (int64_t i = 0; i < n; ++i) {
        double diag = 0.0, lsum = 0.0;
        int32_t k = 0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            if ((int64_t)col[p] == i) {
                diag = val[p];
            } else {
                lsum = lsum + fabs(val[p]);
                k = k + 1;
            }
        }
        a_ii[i] = diag;
        L[i] = lsum;
        deg[i] = k;
        double rate = t * lsum;
        dl[i] = t * (diag + lsum);
        inv_rate[i] = (rate > 0.0) ? 1.0 / rate : INFINITY;
        inv_rate32[i] = (float)inv_rate[i];
        dl32[i] = (float)dl[i];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Alias tables for the jump law k_ij = |a_ij| / L_ii (Eq. 12)         */
/* ------------------------------------------------------------------ */
/* Row i's off-diagonal entries, in stored order, become buckets
 * b = 0..deg_i-1 stored at positions row_ptr[i] + b.  Vose's method:
 *   p_b = (|a_b| * deg) / L_ii in FP64;
 *   small = FIFO of b with p_b < 1, large = FIFO of b with p_b >= 1, both
 *   filled in ascending b;
 *   while both non-empty: l = pop(small), g = pop(large);
 *       prob_l = p_l, alias_l = g;  p_g = (p_g + p_l) - 1;
 *       push g to small if p_g < 1 else to large;
 *   every bucket left in either queue keeps itself with probability 1.
 * threshold_b = min(floor(prob_b 2^32), 2^32 - 1); a draw keeps bucket b's
 * own column when x3 < threshold_b and takes the alias column otherwise.
 * A row with L_ii = 0 (every off-diagonal stored as zero) never jumps; its
 * buckets keep themselves. */
/* Vose over one row's bucket probabilities p[0..k-1] (modified in place);
 * prob/alias receive each bucket's keep probability and alias bucket. */
static void orc_vose_row(int32_t k, double *p, double *prob, int32_t *alias, int32_t *small,
                         int32_t *large)
{
    int32_t s_head = 0, s_len = 0, g_head = 0, g_len = 0;
    for (int32_t b = 0; b < k; ++b) {
        if (p[b] < 1.0) small[(s_head + s_len++) % k] = b;
        else large[(g_head + g_len++) % k] = b;
    }
    while (s_len > 0 && g_len > 0) {
        int32_t l = small[s_head];
        s_head = (s_head + 1) % k; s_len--;
        int32_t g = large[g_head];
        g_head = (g_head + 1) % k; g_len--;
        prob[l] = p[l];
        alias[l] = g;
        p[g] = (p[g] + p[l]) - 1.0;
        if (p[g] < 1.0) small[(s_head + s_len++) % k] = g;
        else large[(g_head + g_len++) % k] = g;
    }
    while (g_len > 0) {
        int32_t g = large[g_head];
        g_head = (g_head + 1) % k; g_len--;
        prob[g] = 1.0;
        alias[g] = g;
    }
    while (s_len > 0) {
        int32_t l = small[s_head];
        s_head = (s_head + 1) % k; s_len--;
        prob[l] = 1.0;
        alias[l] = l;
    }
}

static uint32_t orc_threshold(double prob)
{
    double scaled = floor(prob * 4294967296.0);
    return (scaled >= 4294967295.0) ? 0xFFFFFFFFu : (uint32_t)scaled;
}

/* Alias tables for the jump law of Eq. 12 (see the comment above), or, when
 * h != NULL, for the importance-sampling proposal
 *   q_b = (1 - alpha) |a_b| h(col_b) / sum_c |a_c| h(col_c) + alpha |a_b| / L_ii
 * (a defensive mixture with the paper's law k_b = |a_b| / L_ii), with
 * p_b = q_b deg and lr_b = log(k_b / q_b) recorded for the kept and alias
 * columns of each bucket.  The walk adds lr of every jump to its exponent,
 * which keeps the estimator unbiased whatever h > 0 is. */
static int orc_alias_impl(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                          const double *L, const int32_t *deg, const float *h, double alpha,
                          const double *lam, uint32_t *thr, int32_t *keep_col, uint8_t *keep_neg,
                          int32_t *alias_col, uint8_t *alias_neg, float *lr_keep, float *lr_alias)
{
    int64_t max_deg = 0;
    for (int64_t i = 0; i < n; ++i)
        if (deg[i] > max_deg) max_deg = deg[i];
    size_t cap = (size_t)(max_deg + 1);
    double *p = (double *)malloc(sizeof(double) * cap);
    double *lr = (double *)malloc(sizeof(double) * cap);
    int32_t *bcol = (int32_t *)malloc(sizeof(int32_t) * cap);
    uint8_t *bneg = (uint8_t *)malloc(cap);
    int32_t *small = (int32_t *)malloc(sizeof(int32_t) * cap);
    int32_t *large = (int32_t *)malloc(sizeof(int32_t) * cap);
    double *prob = (double *)malloc(sizeof(double) * cap);
    int32_t *alias = (int32_t *)malloc(sizeof(int32_t) * cap);
    if (!p || !lr || !bcol || !bneg || !small || !large || !prob || !alias) return -1;

    for (int64_t i = 0; i < n; ++i) {
        int32_t k = deg[i];
        if (k == 0) continue;
        int32_t b = 0;
        double hsum = 0.0;
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
            if ((int64_t)col[q] == i) continue;
            bcol[b] = col[q];
            bneg[b] = (uint8_t)(val[q] < 0.0);
            if (h) hsum = hsum + fabs(val[q]) * (double)h[col[q]];
            ++b;
        }
        /* clock tilt: every jump out of row i also carries log(L_ii / lambda_i) */
        double lr_clock = (lam && L[i] > 0.0 && lam[i] > 0.0) ? log(L[i] / lam[i]) : 0.0;
        b = 0;
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
            if ((int64_t)col[q] == i) continue;
            double w = fabs(val[q]);
            if (L[i] <= 0.0) {
                p[b] = 1.0;
                lr[b] = 0.0;
            } else if (!h || !(hsum > 0.0)) {
                p[b] = (w * (double)k) / L[i];
                lr[b] = lr_clock;
            } else {
                double kb = w / L[i];
                double qb = (1.0 - alpha) * ((w * (double)h[col[q]]) / hsum) + alpha * kb;
                p[b] = qb * (double)k;
                lr[b] = ((qb > 0.0) ? log(kb / qb) : 0.0) + lr_clock;
            }
            ++b;
        }
        orc_vose_row(k, p, prob, alias, small, large);
        for (b = 0; b < k; ++b) {
            int64_t pos = row_ptr[i] + b;
            thr[pos] = orc_threshold(prob[b]);
            keep_col[pos] = bcol[b];
            keep_neg[pos] = bneg[b];
            alias_col[pos] = bcol[alias[b]];
            alias_neg[pos] = bneg[alias[b]];
            if (lr_keep) lr_keep[pos] = (float)lr[b];
            if (lr_alias) lr_alias[pos] = (float)lr[alias[b]];
        }
    }
    free(p); free(lr); free(bcol); free(bneg); free(small); free(large); free(prob); free(alias);
    return 0;
}

int orc_alias(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
              const double *L, const int32_t *deg, uint32_t *thr, int32_t *keep_col,
              uint8_t *keep_neg, int32_t *alias_col, uint8_t *alias_neg)
{
    return orc_alias_impl(n, row_ptr, col, val, L, deg, NULL, 0.0, NULL, thr, keep_col, keep_neg,
                          alias_col, alias_neg, NULL, NULL);
}

int orc_alias_is(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                 const double *L, const int32_t *deg, const float *h, double alpha, uint32_t *thr,
                 int32_t *keep_col, uint8_t *keep_neg, int32_t *alias_col, uint8_t *alias_neg,
                 float *lr_keep, float *lr_alias)
{
    return orc_alias_impl(n, row_ptr, col, val, L, deg, h, alpha, NULL, thr, keep_col, keep_neg,
                          alias_col, alias_neg, lr_keep, lr_alias);
}

/* ------------------------------------------------------------------ */
/* Tilted clocks: the h-transform of the walk (importance sampling of  */
/* the holding times; not in the paper)                                */
/* ------------------------------------------------------------------ */
/* Any walk with rates lambda_j > 0 (where row j has off-diagonals), jump
 * law q and, per jump j -> k, the factor a_jk / (lambda_j q_jk) (sign
 * included), weighted by exp(int beta (a_XX + lambda_X) ds), has the
 * expectation of the level-l Strang product of the split
 *   A = D' - T',  D' = diag(a_ii + lambda_i),  T' = diag(lambda) - (A - diag(a)),
 * which tends to exp(tA) v like the paper's split (D' = D, T' = T when
 * lambda = L).  The paper's walk has lambda = L and q = k (Eq. 1, Eq. 12).
 * The h-transform takes, for h > 0,
 *   lambda_i = sum_{j != i} |a_ij| h_j / h_i
 * (clamped to [L_ii / 1024, max(L_ii, 2/t)]: a clock faster than the
 * paper's only where its scaled rate t lambda stays below 2, because the
 * weight grows like e^{t lambda s} wherever h misjudges the row, and at a
 * row whose h is too small the unclamped rate would be large exactly where
 * t L_ii is) and the proposal q of orc_alias_is,
 * so that with h = the exact solution the factors of a path telescope to
 * h(start) / h(end) and the exponent stays near its mean: the variance that
 * the hubs' holding times give the paper's walk (weight e^{t d_j S} against an
 * Exp(t L_jj) clock with d = L) disappears.  In the walk this changes only
 * the tables: rate t lambda_i, dl_i = t (a_ii + lambda_i), and each jump out
 * of row i adds log(L_ii / lambda_i) to the exponent on top of log(k / q).
 * The sum over the row runs in stored order with separate multiply and add
 * (the GPU builds the same tables with the same operations). */
#define ORC_TILT_MIN (1.0 / 1024.0)
#define ORC_TILT_SCALED_MAX 2.0

int orc_tilt_rates(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                   const double *L, const float *h, double t, double *lam)
{
    for (int64_t i = 0; i < n; ++i) {
        double hsum = 0.0;
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
            if ((int64_t)col[q] == i) continue;
            hsum = hsum + fabs(val[q]) * (double)h[col[q]];
        }
        if (!(L[i] > 0.0)) {
            lam[i] = 0.0;
            continue;
        }
        double r = hsum / (double)h[i];
        double lo = L[i] * ORC_TILT_MIN;
        double cap = (t > 0.0) ? ORC_TILT_SCALED_MAX / t : 0.0;
        double hi = L[i] > cap ? L[i] : cap;
        lam[i] = r < lo ? lo : (r > hi ? hi : r);
    }
    return 0;
}

/* The walk's scaled row quantities for rates lambda (as orc_split does for
 * lambda = L): rate_i = t lambda_i, dl_i = t (a_ii + lambda_i),
 * inv_rate_i = 1/rate_i (inf if 0), and their FP32 copies. */
int orc_tilted_split(int64_t n, double t, const double *a_ii, const double *lam, double *dl,
                     double *inv_rate, float *inv_rate32, float *dl32)
{
    for (int64_t i = 0; i < n; ++i) {
        double rate = t * lam[i];
        dl[i] = t * (a_ii[i] + lam[i]);
        inv_rate[i] = (rate > 0.0) ? 1.0 / rate : INFINITY;
        inv_rate32[i] = (float)inv_rate[i];
        dl32[i] = (float)dl[i];
    }
    return 0;
}

/* Proposal tables of the h-transform: the jump law of orc_alias_is and, per
 * entry, lr = log(k/q) + log(L_ii / lambda_i). */
int orc_alias_tilt(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                   const double *L, const int32_t *deg, const float *h, double alpha,
                   const double *lam, uint32_t *thr, int32_t *keep_col, uint8_t *keep_neg,
                   int32_t *alias_col, uint8_t *alias_neg, float *lr_keep, float *lr_alias)
{
    return orc_alias_impl(n, row_ptr, col, val, L, deg, h, alpha, lam, thr, keep_col, keep_neg,
                          alias_col, alias_neg, lr_keep, lr_alias);
}

/* ------------------------------------------------------------------ */
/* The walk (Algorithm 2, MLMCL)                                       */
/* ------------------------------------------------------------------ */
/* Variants select the Philox stream (counter word 3, bits 6-7): stream 1 is
 * reserved for forward-mode walks. */
enum { ORC_RESIDUAL = 0, ORC_REDRAW = 2, ORC_LITERAL_RATE = 3 };
enum { ORC_FP64 = 0, ORC_FP32 = 1 };
enum { ORC_OK = 0, ORC_WALK_LIMIT = 1 };

typedef struct {
    int64_t n;
    const int64_t *row_ptr;
    const int32_t *deg;
    const double *dl;          /* t d_i */
    const double *inv_rate;    /* 1/(t L_ii) */
    const float *inv_rate32;
    const uint32_t *thr;
    const int32_t *keep_col;
    const uint8_t *keep_neg;
    const int32_t *alias_col;
    const uint8_t *alias_neg;
    const double *v;           /* right-hand side u of the paper */
    const float *lr_keep;      /* NULL, or log(k/q) of each bucket's kept column */
    const float *lr_alias;     /* ... and of its alias column (proposal tables) */
    uint64_t seed;
    int32_t precision;         /* ORC_FP64 or ORC_FP32 time arithmetic */
    int32_t variant;           /* ORC_RESIDUAL, ORC_REDRAW, ORC_LITERAL_RATE */
    int64_t max_jumps;
    const double *f;           /* NULL, or the constant source vector F of Algorithm 3 */
    double t;                  /* the time t (the source term's quadrature step is t/N) */
    int32_t pieces;            /* 0 or 1: one law; K > 1: R19's time pieces, with dl,
                                * inv_rate and inv_rate32 holding K blocks of n rows and
                                * the alias arrays K blocks of row_ptr[n] entries */
    int32_t pad_pieces;
} orc_ctx;

typedef struct {
    int32_t end;       /* state at s = 1 */
    int32_t jumps;
    int32_t sign;      /* product of the jump signs phi */
    uint32_t hash;     /* FNV-1a over the states entered by each jump */
    double y;          /* contribution: sign u_end (eta_f - eta_c), or sign u_end eta_f */
    double y_alg2;     /* the same from Algorithm 2's running products eta_2, eta_1 */
    double log_f;      /* fine exponent */
    double log_c;      /* coarse exponent (0 at the coarsest level) */
    int32_t status;
    int32_t pad;
    double src;        /* source part (Algorithm 3): fine minus coarse Simpson sums */
    double src_abs;    /* |fine part| + |coarse part| (scale of its rounding) */
} orc_walk_rec;

/* Counter layout: (rep bits 0-31, row, draw index, level | variant<<6 |
 * rep bits 32-55 << 8); key = seed.  Which words of which draw a walk uses:
 *   FP64 (and the per-interval variant ORC_REDRAW): draw k gives the k-th
 *     holding time (words 0, 1) and the (k+1)-th jump (words 2, 3), so the
 *     draw index equals the number of jumps taken so far.
 *   FP32 (one 32-bit word per uniform): draw k gives the (k+1)-th jump
 *     (words 2, 3) and the holding time that follows it (word 0); the first
 *     holding time takes word 1 of draw 0, or the shared block word below.
 *     A walk with J >= 1 jumps then uses draws 0 .. J-1 and no word twice. */
/* The three fixed counter words of one walk.  Backward: (rep bits 0-31,
 * row, -, level | variant << 6 | rep bits 32-55 << 8).  Forward walk g:
 * (g bits 0-31, g bits 32-63, -, level | 1 << 6). */
typedef struct {
    uint32_t w0, w1, w3;
} orc_ctr;

static orc_ctr orc_ctr_backward(const orc_ctx *c, int64_t row, int64_t rep, int level)
{
    orc_ctr k;
    k.w0 = (uint32_t)((uint64_t)rep & 0xFFFFFFFFull);
    k.w1 = (uint32_t)row;
    k.w3 = (uint32_t)level | ((uint32_t)c->variant << 6) |
           ((uint32_t)(((uint64_t)rep >> 32) & 0xFFFFFFull) << 8);
    return k;
}

static orc_ctr orc_ctr_forward(uint64_t g, int level)
{
    orc_ctr k;
    k.w0 = (uint32_t)(g & 0xFFFFFFFFull);
    k.w1 = (uint32_t)(g >> 32);
    k.w3 = (uint32_t)level | (1u << 6);
    return k;
}

static void orc_draw_k(const orc_ctx *c, orc_ctr k, uint32_t event, uint32_t x[4])
{
    uint32_t ctr[4], key[2];
    ctr[0] = k.w0;
    ctr[1] = k.w1;
    ctr[2] = event;
    ctr[3] = k.w3;
    key[0] = (uint32_t)(c->seed & 0xFFFFFFFFull);
    key[1] = (uint32_t)(c->seed >> 32);
    orc_philox4x32_10(ctr, key, x);
}

/* Holding time in state j from draw x, in the walk's time precision, added
 * to the clock value `from`.  With time pieces j indexes the piece's block
 * (piece * n + state). */
static double orc_hold(const orc_ctx *c, int64_t j, const uint32_t x[4], double from)
{
    if (c->precision == ORC_FP32) {
        float s = orc_neglog32(orc_uniform32(x[0])) * c->inv_rate32[j];
        return (double)((float)from + s);
    }
    double s = orc_neglog64(orc_uniform64(x[0], x[1])) * c->inv_rate[j];
    return from + s;
}

/* FP32 holding time in state j from the single uniform word w. */
static double orc_hold32_word(const orc_ctx *c, int64_t j, uint32_t w, double from)
{
    float s = orc_neglog32(orc_uniform32(w)) * c->inv_rate32[j];
    return (double)((float)from + s);
}

/* Choose the next state from row j's alias table (of time piece `piece`)
 * with draw words x2, x3; *lr receives log(k/q) of the chosen column (0
 * without a proposal). */
static int64_t orc_jump(const orc_ctx *c, int64_t j, const uint32_t x[4], int32_t *sign,
                        double *lr, int32_t piece)
{
    uint32_t b = (uint32_t)(((uint64_t)x[2] * (uint64_t)(uint32_t)c->deg[j]) >> 32);
    int64_t pos = (int64_t)piece * c->row_ptr[c->n] + c->row_ptr[j] + b;
    int64_t to;
    int neg;
    *lr = 0.0;
    if (x[3] < c->thr[pos]) {
        to = c->keep_col[pos];
        neg = c->keep_neg[pos];
        if (c->lr_keep) *lr = (double)c->lr_keep[pos];
    } else {
        to = c->alias_col[pos];
        neg = c->alias_neg[pos];
        if (c->lr_alias) *lr = (double)c->lr_alias[pos];
    }
    if (neg) *sign = -*sign;
    return to;
}

/* R19: the pending jump time t_next >= b of state j carried from piece p
 * into piece p + 1 at the boundary b = step / N. */
static double orc_cross(const orc_ctx *c, int64_t j, int32_t p, double t_next, int64_t step,
                        int64_t N)
{
    const int64_t now = (int64_t)p * c->n + j, next = now + c->n;
    if (c->precision == ORC_FP32) {
        const float b = (float)step / (float)N;
        const float ir = c->inv_rate32[now], irn = c->inv_rate32[next];
        if (isinf(ir) || isinf(irn)) return (double)INFINITY;
        return (double)fmaf((float)t_next - b, irn / ir, b);
    }
    const double b = (double)step / (double)N;
    const double ir = c->inv_rate[now], irn = c->inv_rate[next];
    if (isinf(ir) || isinf(irn)) return INFINITY;
    return fma(t_next - b, irn / ir, b);
}

static int orc_before(const orc_ctx *c, double t_next, int64_t n_step, int64_t N)
{
    /* t_next < n/N in the time precision (n/N is exact in both). */
    if (c->precision == ORC_FP32) return (float)t_next < (float)n_step / (float)N;
    return t_next < (double)n_step / (double)N;
}

/* One walk of row `row`, replica `rep`, at level `level` (N = 2^level fine
 * intervals on [0,1]).  coarse != 0: level > l0, so the walk also carries the
 * coarse weight of level - 1 on the same path (Fig. 1).
 *
 * Algorithm 2's loop over n = 1..N: eta_2 (fine) takes e^{d_j dt/2} at both
 * ends of every interval; eta_1 (coarse) takes e^{d_j dt} at the start of odd
 * intervals and the end of even ones; between, every jump inside the interval
 * flips both signs by sigma.  dt d_j is dl_j/N in scaled time.
 *
 * The returned y uses the paired-step form (Eq. 7): with X_k the state at
 * grid point k and pairs (X_{2j-2}, X_{2j-1}, X_{2j}),
 *   log_f = sum_j dt (d/2 + d + d/2),  log_c = sum_j dt (d + d),
 *   diff  = sum_j dt (-d_{X_{2j-2}}/2 + d_{X_{2j-1}} - d_{X_{2j}}/2) (xi_j of
 *           Lemma 2), so y = sign u_end e^{log_c} expm1(diff) avoids the
 *           cancellation in eta_2 - eta_1. */
/* Intermediate times (the paper's Sec. 5 and Fig. 7 read the solution at
 * the grid times of the same walks): with n_times > 0 the walk also writes
 * y_times[k-1], k = 1..n_times-1, the sample of x(t k / n_times) from its
 * prefix up to grid point g = k N / n_times: the same expression as y with
 * the exponents summed over grid points 0..g (half weights at 0 and g; the
 * coarse rule on the even points) and v at the state at g.  n_times divides
 * N (and N/2 when coarse); the last time is y itself.  A walk stopped at the
 * jump limit keeps the samples of the times it passed (a sample depends only
 * on the path up to its time) and has 0 at the later ones. */
static int orc_walk_core(const orc_ctx *c, int64_t row, orc_ctr kc, int level, int coarse,
                         int use_v_end, int backward, int64_t rep, orc_walk_rec *out,
                         int32_t n_times, double *y_times)
{
    const int64_t N = (int64_t)1 << level;
    /* R19: K time pieces of `per` intervals each; the walk's current piece
     * is that of the interval being walked. */
    const int32_t K = c->pieces > 1 ? c->pieces : 1;
    if (K > 1 && (N % K != 0 || c->f != NULL || n_times > 1 || c->variant != ORC_RESIDUAL)) {
        memset(out, 0, sizeof(*out));
        out->status = -1;
        return -1;
    }
    const int64_t per = N / K;
    int32_t sign = 1;
    int64_t j = row;
    uint32_t ndraw = 0;   /* Philox draws used so far */
    int64_t jumps = 0;
    uint32_t hash = 2166136261u;
    int status = ORC_OK;
    uint32_t x[4];
    double eta2 = 1.0, eta1 = 1.0;
    double log_f = 0.0, log_c = 0.0, diff = 0.0;
    double log_is = 0.0;  /* sum of log(k/q) over the jumps (proposal tables) */
    int64_t x_prev2 = row, x_prev1 = row; /* states at grid points 2j-2, 2j-1 */
    /* Algorithm 3 (reading R17): Simpson sums over the grid points of
     * w_n sign(t_n) eta(t_n) F at the state occupied at t_n; the fine rule
     * on the N steps (weights 1, 4, 2, ..., 4, 1), the coarse one on the
     * N/2 steps of level l-1 (the even grid points).  Grid point 0: weight
     * 1, eta 1, the start row. */
    const int src_on = c->f != NULL && N >= 2;
    for (int32_t k = 0; k + 1 < n_times; ++k) y_times[k] = 0.0;
    double integ2 = src_on ? c->f[row] : 0.0;
    double integ1 = integ2;

    /* FP32 walks pack the holding time that follows a jump into the jump's
     * draw (the counter layout above); the per-interval variant keeps one
     * draw per clock. */
    const int packed = c->precision == ORC_FP32 && c->variant != ORC_REDRAW;
    orc_draw_k(c, kc, ndraw++, x);
    double t_next;
    if (packed) {
        uint32_t w_first = x[1];
        /* FP32 backward walk in a row with 1/(t L) >= 1 (rows where most
         * walks never jump): the first holding time takes its uniform from
         * word (rep mod 4) of the shared block of the four walks 4g..4g+3,
         * g = floor(rep/4), counter (g bits 0-31, row, 0xFFFFFFFE, level |
         * variant << 6 | g bits 32-55 << 8).  The law is unchanged: the
         * four words of one block are independent uniforms. */
        if (backward && c->variant == ORC_RESIDUAL && c->inv_rate32[row] >= 1.0f) {
            const uint64_t g = (uint64_t)rep >> 2;
            orc_ctr kg;
            kg.w0 = (uint32_t)(g & 0xFFFFFFFFull);
            kg.w1 = (uint32_t)row;
            kg.w3 = (uint32_t)level | ((uint32_t)c->variant << 6) |
                    ((uint32_t)((g >> 32) & 0xFFFFFFull) << 8);
            uint32_t xg[4];
            orc_draw_k(c, kg, 0xFFFFFFFEu, xg);
            w_first = xg[(uint64_t)rep & 3u];
        }
        t_next = orc_hold32_word(c, j, w_first, 0.0);
    } else {
        t_next = orc_hold(c, j, x, 0.0);
    }

    for (int64_t step = 1; step <= N; ++step) {
        const int32_t pc = (int32_t)((step - 1) / per);  /* piece of this interval */
        const double *dlp = c->dl + (int64_t)pc * c->n;
        double g = dlp[j] / (double)N;
        eta2 = eta2 * exp(g / 2.0);
        if (step % 2 != 0) eta1 = eta1 * exp(g);
        if (c->variant == ORC_REDRAW) {
            /* Fresh clock at the start of the interval (the listing's tau). */
            orc_draw_k(c, kc, ndraw++, x);
            t_next = orc_hold(c, j, x, (double)(step - 1) / (double)N);
        }
        while (orc_before(c, t_next, step, N)) {
            if (jumps >= c->max_jumps) {
                status = ORC_WALK_LIMIT;
                goto done;
            }
            int64_t from = j;
            double lr = 0.0;
            /* FP32: jump k + 1 takes draw k (draw 0 is already at hand). */
            if (packed && jumps > 0) orc_draw_k(c, kc, ndraw++, x);
            j = orc_jump(c, j, x, &sign, &lr, pc);
            log_is = log_is + lr;
            hash = (hash ^ (uint32_t)j) * 16777619u;
            jumps = jumps + 1;
            /* R1: the new holding time uses the new state's rate; the
             * literal reading uses the state just left. */
            const int64_t rate_state = ((c->variant == ORC_LITERAL_RATE) ? from : j) +
                                       (int64_t)pc * c->n;
            if (packed) {
                t_next = orc_hold32_word(c, rate_state, x[0], t_next);
            } else {
                orc_draw_k(c, kc, ndraw++, x);
                t_next = orc_hold(c, rate_state, x, t_next);
            }
        }
        g = dlp[j] / (double)N;
        eta2 = eta2 * exp(g / 2.0);
        if (step % 2 == 0) eta1 = eta1 * exp(g);
        if (src_on) {
            double w = (step == N) ? 1.0 : ((step % 2 != 0) ? 4.0 : 2.0);
            integ2 = integ2 + w * (double)sign * eta2 * c->f[j];
            if (step % 2 == 0) {
                int64_t m = step / 2;
                double wc = (m == N / 2) ? 1.0 : ((m % 2 != 0) ? 4.0 : 2.0);
                integ1 = integ1 + wc * (double)sign * eta1 * c->f[j];
            }
        }
        if (step % 2 == 0) {
            /* Pair (X_{step-2}, X_{step-1}, X_step) of Eq. 7.  Each point
             * takes the piece of the pair's interval next to it (R19); the
             * middle point, between intervals step-1 and step, the mean of
             * both (one value when they share a piece). */
            const double *dla = c->dl + (int64_t)((step - 2) / per) * c->n;
            double d0 = dla[x_prev2] / (double)N;
            double d1 = ((dla[x_prev1] + dlp[x_prev1]) / 2.0) / (double)N;
            double d2 = dlp[j] / (double)N;
            log_f = log_f + (d0 / 2.0 + d1 + d2 / 2.0);
            log_c = log_c + (d0 + d2);
            diff = diff + ((d1 - d0 / 2.0) - d2 / 2.0);
            x_prev2 = j;
        } else {
            x_prev1 = j;
        }
        if (n_times > 1 && step < N && step % (N / n_times) == 0) {
            /* prefix sample at grid point `step` (state j) */
            double uj = use_v_end ? c->v[j] : 1.0;
            double y;
            if (coarse) {
                y = (double)sign * uj * (exp(log_c + log_is) * expm1(diff));
            } else {
                double lf = log_f;
                if (step % 2 != 0) /* the pairs end at step - 1 */
                    lf = lf + (c->dl[x_prev2] / (double)N / 2.0 + c->dl[j] / (double)N / 2.0);
                y = (double)sign * uj * exp(lf + log_is);
            }
            y_times[step / (N / n_times) - 1] = y;
        }
        /* R19: the pending jump time passes into the next piece. */
        if (K > 1 && step % per == 0 && step < N) t_next = orc_cross(c, j, pc, t_next, step, N);
    }
    if (N == 1) {
        /* Level 0 has one interval and no pair: the fine exponent is
         * dt (d_{X_0} + d_{X_1}) / 2 with dt = 1 in scaled time. */
        log_f = c->dl[row] / 2.0 + c->dl[j] / 2.0;
    }
done:
    out->end = (int32_t)j;
    out->jumps = (int32_t)jumps;
    out->sign = sign;
    out->hash = hash;
    out->status = status;
    out->pad = 0;
    out->src = 0.0;
    out->src_abs = 0.0;
    if (status != ORC_OK) {
        out->y = 0.0;
        out->y_alg2 = 0.0;
        out->log_f = 0.0;
        out->log_c = 0.0;
        return status;
    }
    if (src_on) {
        double sf = c->t / (3.0 * (double)N) * integ2;
        double sc = (coarse && N >= 4) ? 2.0 * c->t / (3.0 * (double)N) * integ1 : 0.0;
        out->src = sf - sc;
        out->src_abs = fabs(sf) + fabs(sc);
    }
    double uj = use_v_end ? c->v[j] : 1.0;
    out->log_f = log_f;
    out->log_c = coarse ? log_c : 0.0;
    if (coarse) {
        out->y = (double)sign * uj * (exp(log_c + log_is) * expm1(diff));
        out->y_alg2 = (double)sign * uj * (eta2 - eta1) * exp(log_is);
    } else {
        out->y = (double)sign * uj * exp(log_f + log_is);
        out->y_alg2 = (double)sign * uj * eta2 * exp(log_is);
    }
    return status;
}

int orc_walk(const orc_ctx *c, int64_t row, int64_t rep, int level, int coarse,
             orc_walk_rec *out)
{
    return orc_walk_core(c, row, orc_ctr_backward(c, row, rep, level), level, coarse, 1, 1, rep,
                         out, 0, NULL);
}

/* orc_walk with the samples of the intermediate times (see orc_walk_core):
 * y_times[0 .. n_times-2]. */
int orc_walk_times(const orc_ctx *c, int64_t row, int64_t rep, int level, int coarse,
                   int32_t n_times, orc_walk_rec *out, double *y_times)
{
    return orc_walk_core(c, row, orc_ctr_backward(c, row, rep, level), level, coarse, 1, 1, rep,
                         out, n_times, y_times);
}

/* Forward mode (Eq. 5; reading R6): the tables in c are those of B = A^T.
 * Walk g draws its start from the integer weights w (prefix sums cdf,
 * total W): r = floor(u W / 2^64) with u the 64-bit word (x0:x1) of the
 * draw at index 0xFFFFFFFF, start = the smallest s with cdf[s] > r.  Its
 * contribution is y = v_s (W / w_s) sign e^{...}, added to x[end]. */
int orc_walk_fwd(const orc_ctx *c, const int64_t *cdf, const int64_t *w, uint64_t W, uint64_t g,
                 int level, int coarse, orc_walk_rec *out)
{
    orc_ctr kc = orc_ctr_forward(g, level);
    uint32_t x[4];
    orc_draw_k(c, kc, 0xFFFFFFFFu, x);
    uint64_t u = ((uint64_t)x[0] << 32) | (uint64_t)x[1];
    uint64_t r = (uint64_t)(((unsigned __int128)u * (unsigned __int128)W) >> 64);
    int64_t lo = 0, hi = c->n - 1;
    while (lo < hi) { /* binary search: smallest s with cdf[s] > r */
        int64_t mid = (lo + hi) / 2;
        if ((uint64_t)cdf[mid] > r) hi = mid; else lo = mid + 1;
    }
    int status = orc_walk_core(c, lo, kc, level, coarse, 0, 0, 0, out, 0, NULL);
    double f = c->v[lo] * ((double)W / (double)w[lo]);
    out->y = out->y * f;
    out->y_alg2 = out->y_alg2 * f;
    out->pad = (int32_t)lo;
    return status;
}

int orc_walk_fwd_many(const orc_ctx *c, const int64_t *cdf, const int64_t *w, uint64_t W,
                      uint64_t g0, int64_t count, int level, int coarse, orc_walk_rec *out)
{
    int bad = 0;
    for (int64_t k = 0; k < count; ++k)
        if (orc_walk_fwd(c, cdf, w, W, g0 + (uint64_t)k, level, coarse, &out[k]) != ORC_OK) bad = 1;
    return bad;
}

/* Algorithm 2 in forward mode for walks g0 .. g0+count-1: sum_x[end] += y. */
int orc_mlmcl_fwd(const orc_ctx *c, const int64_t *cdf, const int64_t *w, uint64_t W, uint64_t g0,
                  int64_t count, int level, int coarse, double *sum_x, double *sum_y2,
                  int64_t *jumps, int64_t *limit_hits)
{
    orc_walk_rec r;
    for (int64_t k = 0; k < count; ++k) {
        if (orc_walk_fwd(c, cdf, w, W, g0 + (uint64_t)k, level, coarse, &r) != ORC_OK)
            *limit_hits = *limit_hits + 1;
        sum_x[r.end] = sum_x[r.end] + r.y;
        *sum_y2 = *sum_y2 + r.y * r.y;
        *jumps = *jumps + r.jumps;
    }
    return 0;
}

int orc_walk_many(const orc_ctx *c, int64_t count, const int64_t *rows, const int64_t *reps,
                  int level, int coarse, orc_walk_rec *out)
{
    int bad = 0;
    for (int64_t k = 0; k < count; ++k)
        if (orc_walk(c, rows[k], reps[k], level, coarse, &out[k]) != ORC_OK) bad = 1;
    return bad;
}

/* MLMCL (Algorithm 2) for rows [row_begin, row_end) and replicas
 * [rep_begin, rep_begin + reps): per-row sums of y into sum_y[row], and the
 * totals sum y^2, jumps and walk-limit hits.  Rows are split over OpenMP
 * threads; each row's sum is formed in replica order. */
/* Walks rows[k], reps[k] with their intermediate-time samples:
 * y_times[k*(n_times-1) + j]. */
int orc_walk_times_many(const orc_ctx *c, int64_t count, const int64_t *rows, const int64_t *reps,
                        int level, int coarse, int32_t n_times, orc_walk_rec *out,
                        double *y_times)
{
    int bad = 0;
    for (int64_t k = 0; k < count; ++k)
        if (orc_walk_times(c, rows[k], reps[k], level, coarse, n_times, &out[k],
                           y_times + k * (int64_t)(n_times - 1)) != ORC_OK)
            bad = 1;
    return bad;
}

int orc_mlmcl(const orc_ctx *c, int64_t row_begin, int64_t row_end, int64_t rep_begin,
              int64_t reps, int level, int coarse, int nthreads, double *sum_y,
              double *sum_y2, int64_t *jumps, int64_t *limit_hits)
{
    double tot_y2 = 0.0;
    int64_t tot_j = 0, tot_lim = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : tot_y2, tot_j, tot_lim)
#endif
    for (int64_t i = row_begin; i < row_end; ++i) {
        double s = 0.0, s2 = 0.0;
        int64_t jj = 0, lim = 0;
        orc_walk_rec r;
        for (int64_t k = 0; k < reps; ++k) {
            if (orc_walk(c, i, rep_begin + k, level, coarse, &r) != ORC_OK) lim++;
            double yt = r.y + r.src;  /* with a source term: both parts of the sample */
            s = s + yt;
            s2 = s2 + yt * yt;
            jj += r.jumps;
        }
        sum_y[i] = sum_y[i] + s;
        tot_y2 += s2;
        tot_j += jj;
        tot_lim += lim;
    }
    *sum_y2 = *sum_y2 + tot_y2;
    *jumps = *jumps + tot_j;
    *limit_hits = *limit_hits + tot_lim;
    return 0;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
