/*
 * fc_oracle.c -- plain, slow CPU oracle for the Feldman-Cousins grid fit.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA library; both are
 * written independently from the method's definition:
 *
 *   Eq. 1        chi2 = (a - b)^T M (a - b), M the inverse covariance
 *   Algorithm 2  calcChi2: residual d = a - b, then d^T M d
 *   Algorithm 1  buildDeltaChi2: per universe fluctuate s = S(p), scan every
 *                q in the grid with a strict "<" update, dchi2 = chi2(a, c) - chi2_min
 *   §2 (steps 1-6 of the per-universe procedure): after the scan, rebuild M at
 *                q_min and rescan until the best fit is stable.
 *
 * Readings (the paper does not define them; the same reading is used by the
 * CUDA library):
 *   - the covariance is M(q) = C [diag(s_q) F diag(s_q) + diag(s_q)] C^T in fit
 *     space (C = bin collapse), and the fit uses A = M^-1;
 *   - the central vector c of Algorithm 1 is S(p), the true point's spectrum;
 *   - a scan stops when its best-fit index equals the index whose covariance it
 *     used, or after max_iter scans; dchi2 uses the last scan's A for both terms;
 *   - "fluctuation of s": d = Poisson(max(0, s + L z)), L = chol of the
 *     systematic part diag(s) F diag(s), z standard normal, in the full-bin
 *     space, then collapsed with integer sums;
 *   - the random numbers come from Philox4x32-10 (Salmon et al., SC'11) with
 *     key = seed and counter = (block, universe, point, stream tag).
 *
 * Precision.  The fit (covariance, Cholesky, inverse, chi2, argmin) is IEEE
 * binary64.  The fluctuation takes its integer decisions (the Poisson counts)
 * in binary32, the precision the CUDA sampler computes in; every binary32 step
 * below is a correctly rounded IEEE operation (+ - * / sqrt, fmaf, floor,
 * rint) in a fixed order, so the counts are reproducible bit for bit.  The
 * elementary functions log, exp, sin, cos are this file's own polynomial
 * evaluations (coefficients are the Taylor / atanh series terms 1/n!, 1/(2n+1)),
 * not libm.  Compile with -ffp-contract=off.
 *
 * Pins (tests/test_oracle_*.py): Philox known-answer vector; log/exp/sincos
 * against numpy float64; normal KS test; Poisson goodness of fit against the
 * exact pmf; Cholesky/inverse against numpy.linalg; chi2 scan against an
 * independent numpy brute force; A = I against a k-d tree nearest neighbour;
 * Wilks chi2_D law for a linear-Gaussian model; dchi2 >= 0.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_FLUCT_POISSON_SYS 0
#define ORC_FLUCT_GAUSS 1
#define ORC_COV_ITERATE 0
#define ORC_COV_FIXED 1
#define ORC_COV_IDENTITY 2

/* ------------------------------------------------------------------------- */
/* Philox4x32-10                                                              */
/* ------------------------------------------------------------------------- */

static void orc_philox_round(uint32_t c[4], const uint32_t k[2]) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        orc_philox_round(c, k);
    }
    memcpy(out, c, sizeof c);
}

/* u = ((x >> 9) + 1/2) * 2^-23, exactly representable, in [2^-24, 1 - 2^-24]. */
float oracle_u01(uint32_t x) {
    float m = (float)(x >> 9);
    m = m + 0.5f;
    return m * 1.1920928955078125e-07f;
}

/* ------------------------------------------------------------------------- */
/* binary32 elementary functions written from their series                   */
/* ------------------------------------------------------------------------- */

static float orc_bits_to_float(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t orc_float_to_bits(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

#define ORC_LN2_HI 0.693145751953125f          /* 0x3F317200: 15 significant bits */
#define ORC_LN2_LO 1.428606765330187e-06f      /* ln 2 - ORC_LN2_HI               */
#define ORC_SQRT2 1.41421353816986083984375f   /* nearest binary32 to sqrt 2      */

/* ln x for normal positive x: x = m 2^e, m in [sqrt(1/2), sqrt 2),
 * ln m = 2 atanh(t), t = (m-1)/(m+1), series t + t^3/3 + ... + t^9/9. */
float oracle_logf(float x) {
    uint32_t bits = orc_float_to_bits(x);
    int e = (int)(bits >> 23) - 127;
    float m = orc_bits_to_float((bits & 0x007FFFFFu) | 0x3F800000u);
    if (m > ORC_SQRT2) {
        m = m * 0.5f;
        e = e + 1;
    }
    const float num = m - 1.0f;
    const float den = m + 1.0f;
    const float t = num / den;
    const float t2 = t * t;
    float p = fmaf(t2, 0.111111111111111111f, 0.142857142857142857f);
    p = fmaf(t2, p, 0.2f);
    p = fmaf(t2, p, 0.333333333333333333f);
    const float tt = t + t;
    const float tt3 = tt * t2;
    const float lnm = fmaf(tt3, p, tt);
    const float fe = (float)e;
    float r = fmaf(fe, ORC_LN2_LO, lnm);
    r = fmaf(fe, ORC_LN2_HI, r);
    return r;
}

/* e^x for x in [-87, 88]: x = n ln2 + r, |r| <= ln2/2, Taylor degree 8 in r. */
float oracle_expf(float x) {
    const float kf = rintf(x * 1.44269502162933349609375f);
    float r = fmaf(-kf, ORC_LN2_HI, x);
    r = fmaf(-kf, ORC_LN2_LO, r);
    float p = fmaf(r, 2.48015873015873015873e-05f, 1.98412698412698412698e-04f);
    p = fmaf(r, p, 1.38888888888888888889e-03f);
    p = fmaf(r, p, 8.33333333333333333333e-03f);
    p = fmaf(r, p, 4.16666666666666666667e-02f);
    p = fmaf(r, p, 1.66666666666666666667e-01f);
    p = fmaf(r, p, 0.5f);
    p = fmaf(r, p, 1.0f);
    p = fmaf(r, p, 1.0f);
    const int n = (int)kf;
    const float scale = orc_bits_to_float((uint32_t)(n + 127) << 23);
    return p * scale;
}

/* sin and cos of 2 pi u for u in (0, 1): quarter-turn reduction, then Taylor
 * series in x = f pi/2 with |f| <= 1/2. */
void oracle_sincos_turns(float u, float* s_out, float* c_out) {
    const float w = u * 4.0f;
    const float jf = rintf(w);
    const float f = w - jf;
    const float x = f * 1.57079637050628662109375f;
    const float x2 = x * x;
    float ps = fmaf(x2, 2.75573192239858906526e-06f, -1.98412698412698412698e-04f);
    ps = fmaf(x2, ps, 8.33333333333333333333e-03f);
    ps = fmaf(x2, ps, -1.66666666666666666667e-01f);
    const float x3 = x2 * x;
    const float s = fmaf(x3, ps, x);
    float pc = fmaf(x2, -2.75573192239858906526e-07f, 2.48015873015873015873e-05f);
    pc = fmaf(x2, pc, -1.38888888888888888889e-03f);
    pc = fmaf(x2, pc, 4.16666666666666666667e-02f);
    pc = fmaf(x2, pc, -0.5f);
    const float c = fmaf(x2, pc, 1.0f);
    const int q = ((int)jf) & 3;
    switch (q) {
        case 0: *c_out = c; *s_out = s; break;
        case 1: *c_out = -s; *s_out = c; break;
        case 2: *c_out = -c; *s_out = -s; break;
        default: *c_out = s; *s_out = -c; break;
    }
}

/* ------------------------------------------------------------------------- */
/* Random streams                                                             */
/* ------------------------------------------------------------------------- */

typedef struct {
    uint32_t key[2];
    uint32_t ctr[4];
    uint32_t buf[4];
    int pos;
} orc_stream;

static void orc_stream_init(orc_stream* st, uint64_t seed, uint32_t u, uint32_t p, uint32_t tag) {
    st->key[0] = (uint32_t)seed;
    st->key[1] = (uint32_t)(seed >> 32);
    st->ctr[0] = 0;
    st->ctr[1] = u;
    st->ctr[2] = p;
    st->ctr[3] = tag;
    st->pos = 4;
}

static float orc_stream_uniform(orc_stream* st) {
    if (st->pos == 4) {
        oracle_philox4x32_10(st->ctr, st->key, st->buf);
        st->ctr[0] += 1;
        st->pos = 0;
    }
    return oracle_u01(st->buf[st->pos++]);
}

#define ORC_TAG_NORMAL 0u
#define ORC_TAG_POISSON 0x80000000u

/* n standard normals for (seed, point p, universe u): Box-Muller on the pairs
 * (u0,u1), (u2,u3) of each Philox block j = 0, 1, ...; z[4j..4j+3]. */
void oracle_normals(uint64_t seed, uint32_t p, uint32_t u, int n, float* z) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int j = 0; 4 * j < n; ++j) {
        const uint32_t ctr[4] = {(uint32_t)j, u, p, ORC_TAG_NORMAL};
        uint32_t x[4];
        oracle_philox4x32_10(ctr, key, x);
        for (int h = 0; h < 2; ++h) {
            const float ua = oracle_u01(x[2 * h]);
            const float ub = oracle_u01(x[2 * h + 1]);
            float t = oracle_logf(ua);
            t = t * -2.0f;
            const float R = sqrtf(t);
            float sn, cs;
            oracle_sincos_turns(ub, &sn, &cs);
            const int i0 = 4 * j + 2 * h;
            if (i0 < n) z[i0] = R * cs;
            if (i0 + 1 < n) z[i0 + 1] = R * sn;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Poisson sampler (binary32)                                                 */
/* ------------------------------------------------------------------------- */

/* ln k! for k = 0..9 as a running sum of logs. */
static float orc_logfact_small(float k) {
    float s = 0.0f;
    for (float j = 2.0f; j <= k; j = j + 1.0f) s = s + oracle_logf(j);
    return s;
}

/* Stirling remainder ln k! - (k ln k - k + ln(2 pi k)/2) for k >= 10:
 * 1/(12k) - 1/(360k^3) + 1/(1260k^5). */
static float orc_stirlerr(float k) {
    const float ik = 1.0f / k;
    const float ik2 = ik * ik;
    float p = fmaf(-ik2, 7.93650793650793650794e-04f, 2.77777777777777777778e-03f);
    p = fmaf(-ik2, p, 8.33333333333333333333e-02f);
    return ik * p;
}

/* Deviance term k ln(k/lam) + lam - k (Loader 2000), series in v = (k-lam)/(k+lam)
 * when |v| < 0.1: (k-lam) v + 2k sum_{j>=1} v^(2j+1)/(2j+1), six terms. */
static float orc_bd0(float k, float lam) {
    const float diff = k - lam;
    const float sum = k + lam;
    if (fabsf(diff) < 0.1f * sum) {
        const float v = diff / sum;
        float s = diff * v;
        float ej = (k + k) * v;
        const float v2 = v * v;
        for (int j = 1; j <= 6; ++j) {
            ej = ej * v2;
            s = s + ej / (float)(2 * j + 1);
        }
        return s;
    }
    float t = k / lam;
    t = oracle_logf(t);
    t = k * t;
    t = t + lam;
    return t - k;
}

/* ln P(k; lam) */
static float orc_logpmf(float k, float lam, float loglam) {
    if (k < 10.0f) {
        float t = k * loglam;
        t = t - lam;
        return t - orc_logfact_small(k);
    }
    const float t1 = orc_bd0(k, lam);
    const float t2 = oracle_logf(6.28318548202514648438f * k) * 0.5f;
    const float t3 = orc_stirlerr(k);
    float r = -t1;
    r = r - t2;
    return r - t3;
}

/* Poisson(lam): 0 for lam <= 0; sequential-search inversion for lam < 10;
 * Hormann's transformed rejection with squeeze (PTRS, 1993) for lam >= 10. */
static int32_t orc_poisson(float lam, orc_stream* st) {
    if (!(lam > 0.0f)) return 0;
    if (lam < 10.0f) {
        float pk = oracle_expf(-lam);
        float F = pk;
        int32_t k = 0;
        const float u = orc_stream_uniform(st);
        while (u > F && k < 64) {
            k = k + 1;
            pk = pk * lam;
            pk = pk / (float)k;
            F = F + pk;
        }
        return k;
    }
    const float slam = sqrtf(lam);
    const float loglam = oracle_logf(lam);
    const float b = fmaf(2.53f, slam, 0.931f);
    const float a = fmaf(0.02483f, b, -0.059f);
    const float twoa = a + a;
    const float invalpha = 1.1239f + 1.1328f / (b - 3.4f);
    const float vr = 0.9277f - 3.6224f / (b - 2.0f);
    for (int it = 0; it < 64; ++it) {
        const float U = orc_stream_uniform(st) - 0.5f;
        const float V = orc_stream_uniform(st);
        const float us = 0.5f - fabsf(U);
        float t = twoa / us;
        t = t + b;
        t = t * U;
        t = t + lam;
        t = t + 0.43f;
        const float kf = floorf(t);
        if (us >= 0.07f && V <= vr) return (int32_t)kf;
        if (kf < 0.0f || (us < 0.013f && V > us)) continue;
        const float d1 = us * us;
        const float d2 = a / d1;
        const float d3 = d2 + b;
        const float n1 = V * invalpha;
        const float lhs = oracle_logf(n1 / d3);
        if (lhs <= orc_logpmf(kf, lam, loglam)) return (int32_t)kf;
    }
    return (int32_t)floorf(lam);
}

/* n draws of Poisson(lam) from the stream of (seed, p, u, bin). */
void oracle_poisson_draws(float lam, uint64_t seed, uint32_t p, uint32_t u, uint32_t bin, int n, int32_t* out) {
    orc_stream st;
    orc_stream_init(&st, seed, u, p, ORC_TAG_POISSON | bin);
    for (int i = 0; i < n; ++i) out[i] = orc_poisson(lam, &st);
}

/* n independent single draws of Poisson(lam): draw i uses universe i's stream. */
void oracle_poisson_indep(float lam, uint64_t seed, uint32_t p, uint32_t bin, int n, int32_t* out) {
    for (int i = 0; i < n; ++i) {
        orc_stream st;
        orc_stream_init(&st, seed, (uint32_t)i, p, ORC_TAG_POISSON | bin);
        out[i] = orc_poisson(lam, &st);
    }
}

/* ------------------------------------------------------------------------- */
/* binary64 linear algebra                                                    */
/* ------------------------------------------------------------------------- */

/* Cholesky-Banachiewicz, lower triangle of M read, L row-major lower (upper
 * part zeroed).  Each sum runs k = 0..j-1 with separately rounded * and -.
 * Returns 0, or -1 if a pivot is not positive. */
int oracle_cholesky(int n, const double* M, double* L) {
    memset(L, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int j = 0; j < n; ++j) {
        double acc = M[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) {
            const double pr = L[(size_t)j * n + k] * L[(size_t)j * n + k];
            acc = acc - pr;
        }
        if (!(acc > 0.0)) return -1;
        const double dj = sqrt(acc);
        L[(size_t)j * n + j] = dj;
        for (int i = j + 1; i < n; ++i) {
            double a2 = M[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) {
                const double pr = L[(size_t)i * n + k] * L[(size_t)j * n + k];
                a2 = a2 - pr;
            }
            L[(size_t)i * n + j] = a2 / dj;
        }
    }
    return 0;
}

/* Systematic covariance of point s in the full-bin space:
 * Msys_ij = (s_i F_ij) s_j, lower triangle (i >= j) filled, upper mirrored. */
static void orc_sys_cov(int n, const double* s, const double* F, double* M) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            const double t = s[i] * F[(size_t)i * n + j];
            const double v = t * s[j];
            M[(size_t)i * n + j] = v;
            M[(size_t)j * n + i] = v;
        }
}

/* L_p = chol(diag(s) F diag(s)) (gauss = 0) or chol(diag(s) F diag(s) + diag(s)) (gauss = 1). */
int oracle_chol_sys(int n, const double* s, const double* F, int gauss, double* L) {
    double* M = (double*)malloc(sizeof(double) * (size_t)n * n);
    orc_sys_cov(n, s, F, M);
    if (gauss)
        for (int i = 0; i < n; ++i) M[(size_t)i * n + i] = M[(size_t)i * n + i] + s[i];
    const int rc = oracle_cholesky(n, M, L);
    free(M);
    return rc;
}

/* Fit-space covariance M(q) = C [diag(s) F diag(s) + diag(s)] C^T, where C sums
 * the full bins i with collapse[i] = j into fit bin j (identity when collapse is NULL). */
static void orc_fit_cov(int nf, int nfit, const int32_t* collapse, const double* s, const double* F, double* Mfit) {
    memset(Mfit, 0, sizeof(double) * (size_t)nfit * nfit);
    for (int i = 0; i < nf; ++i) {
        const int ji = collapse ? collapse[i] : i;
        for (int m = 0; m < nf; ++m) {
            const int jm = collapse ? collapse[m] : m;
            double v = (s[i] * F[(size_t)i * nf + m]) * s[m];
            if (i == m) v = v + s[i];
            Mfit[(size_t)ji * nfit + jm] += v;
        }
    }
}

/* A = M^-1 from the Cholesky factor: solve L y = e_k, L^T x = y for every k. */
static int orc_inverse_spd(int n, const double* M, double* A, double* Lbuf, double* col) {
    if (oracle_cholesky(n, M, Lbuf) != 0) return -1;
    for (int k = 0; k < n; ++k) {
        for (int i = 0; i < n; ++i) {
            double acc = (i == k) ? 1.0 : 0.0;
            for (int j = 0; j < i; ++j) acc -= Lbuf[(size_t)i * n + j] * col[j];
            col[i] = acc / Lbuf[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double acc = col[i];
            for (int j = i + 1; j < n; ++j) acc -= Lbuf[(size_t)j * n + i] * A[(size_t)j * n + k];
            A[(size_t)i * n + k] = acc / Lbuf[(size_t)i * n + i];
        }
    }
    return 0;
}

/* A(q) = M(q)^-1 in fit space for the grid spectrum s (full bins). */
int oracle_inv_cov(int nf, int nfit, const int32_t* collapse, const double* s, const double* F, double* A) {
    double* M = (double*)malloc(sizeof(double) * (size_t)nfit * nfit);
    double* Lb = (double*)malloc(sizeof(double) * (size_t)nfit * nfit);
    double* col = (double*)malloc(sizeof(double) * (size_t)nfit);
    orc_fit_cov(nf, nfit, collapse, s, F, M);
    const int rc = orc_inverse_spd(nfit, M, A, Lb, col);
    free(M);
    free(Lb);
    free(col);
    return rc;
}

/* Fit-space spectra: S_fit[g][j] = sum over full bins i with collapse[i] = j, in i order. */
void oracle_collapse_spectra(int64_t G, int nf, int nfit, const int32_t* collapse, const double* S, double* Sfit) {
    for (int64_t g = 0; g < G; ++g) {
        double* o = Sfit + (size_t)g * nfit;
        for (int j = 0; j < nfit; ++j) o[j] = 0.0;
        for (int i = 0; i < nf; ++i) {
            const int j = collapse ? collapse[i] : i;
            o[j] = o[j] + S[(size_t)g * nf + i];
        }
    }
}

/* Algorithm 2: r = a - b, chi2 = sum_i r_i sum_j A_ij r_j. */
static double orc_chi2(int n, const double* a, const double* b, const double* A, double* r) {
    for (int i = 0; i < n; ++i) r[i] = a[i] - b[i];
    double chi2 = 0.0;
    for (int i = 0; i < n; ++i) {
        double t = 0.0;
        for (int j = 0; j < n; ++j) t += A[(size_t)i * n + j] * r[j];
        chi2 += r[i] * t;
    }
    return chi2;
}

/* chi2 of the fit-space data d against every grid spectrum under A. */
void oracle_scan(int64_t G, int nfit, const double* Sfit, const double* A, const double* d, double* chi2) {
    double* r = (double*)malloc(sizeof(double) * (size_t)nfit);
    for (int64_t g = 0; g < G; ++g) chi2[g] = orc_chi2(nfit, Sfit + (size_t)g * nfit, d, A, r);
    free(r);
}

/* ------------------------------------------------------------------------- */
/* Fake data (§2 step 2)                                                     */
/* ------------------------------------------------------------------------- */

/* One universe: lam_i = max(0, s_i + sum_{j<=i} L_ij z_j) in binary32 with
 * fmaf accumulation in j order; n_i = Poisson(lam_i) on bin i's own stream
 * (or n_i = lam_i without truncation in the Gaussian test mode); fit bins
 * are the sums of their full bins in i order. */
static void orc_fake_one(int nf, int nfit, const int32_t* collapse, const float* sf, const float* Lf,
                         uint64_t seed, uint32_t p, uint32_t u, int fluct, float* z, float* dfit) {
    oracle_normals(seed, p, u, nf, z);
    for (int j = 0; j < nfit; ++j) dfit[j] = 0.0f;
    for (int i = 0; i < nf; ++i) {
        float acc = 0.0f;
        for (int j = 0; j <= i; ++j) acc = fmaf(Lf[(size_t)i * nf + j], z[j], acc);
        float lam = sf[i] + acc;
        float v;
        if (fluct == ORC_FLUCT_GAUSS) {
            v = lam;
        } else {
            if (!(lam > 0.0f)) lam = 0.0f;
            orc_stream st;
            orc_stream_init(&st, seed, u, p, ORC_TAG_POISSON | (uint32_t)i);
            v = (float)orc_poisson(lam, &st);
        }
        const int jf = collapse ? collapse[i] : i;
        dfit[jf] = dfit[jf] + v;
    }
}

/* ------------------------------------------------------------------------- */
/* Grid fit per universe (§2 steps 3-6, Algorithm 1)                           */
/* ------------------------------------------------------------------------- */

typedef struct {
    const double* S;       /* [G][nf] */
    const double* Sfit;    /* [G][nfit] */
    const double* F;
    const int32_t* collapse;
    int64_t G;
    int nf, nfit;
    const int64_t* ps;
    const int32_t* us;     /* sample mode: universe of sample i (ps[i] its point), else NULL */
    const float* data;     /* given-data mode: every fit uses this [nfit] vector instead of fake data */
    int P, U;
    uint64_t seed;
    int max_iter, fluct, cov;
    const float* Lf;       /* [P][nf][nf] binary32 copy of L_p */
    const float* sf;       /* [P][nf] binary32 copy of s_p */
    double* dchi2;
    int64_t* bestfit;
    int8_t* nscans;
    float* dfit_out;       /* optional [P][U][nfit] */
    int nthreads, tid;
    int status;
} orc_job;

static void orc_fit_universe(orc_job* jb, int ip, int u, double* A, double* M, double* Lb, double* col,
                             double* r, double* d, float* z, float* dfitf, double* dres, int64_t* bres, int8_t* nres) {
    const int nf = jb->nf, nfit = jb->nfit;
    const int64_t p = jb->ps[ip];
    if (jb->data)
        memcpy(dfitf, jb->data, sizeof(float) * nfit);
    else
        orc_fake_one(nf, nfit, jb->collapse, jb->sf + (size_t)ip * nf, jb->Lf + (size_t)ip * nf * nf, jb->seed,
                     (uint32_t)p, (uint32_t)u, jb->fluct, z, dfitf);
    if (jb->dfit_out) memcpy(jb->dfit_out + ((size_t)ip * jb->U + u) * nfit, dfitf, sizeof(float) * nfit);
    for (int j = 0; j < nfit; ++j) d[j] = (double)dfitf[j];
    int64_t q = p;
    int64_t best_idx = p;
    double best = INFINITY, chi2p = NAN;
    int t = 0;
    const int max_iter = (jb->cov == ORC_COV_ITERATE) ? jb->max_iter : 1;
    for (t = 0; t < max_iter; ++t) {
        if (jb->cov == ORC_COV_IDENTITY) {
            for (int i = 0; i < nfit; ++i)
                for (int j = 0; j < nfit; ++j) A[(size_t)i * nfit + j] = (i == j) ? 1.0 : 0.0;
        } else {
            orc_fit_cov(nf, nfit, jb->collapse, jb->S + (size_t)q * nf, jb->F, M);
            if (orc_inverse_spd(nfit, M, A, Lb, col) != 0) {
                jb->status = -2;
                return;
            }
        }
        best = INFINITY;
        best_idx = -1;
        for (int64_t g = 0; g < jb->G; ++g) {
            const double c = orc_chi2(nfit, jb->Sfit + (size_t)g * nfit, d, A, r);
            if (c < best) {
                best = c;
                best_idx = g;
            }
            if (g == p) chi2p = c;
        }
        if (best_idx == q) {
            t = t + 1;
            break;
        }
        q = best_idx;
    }
    if (t > max_iter) t = max_iter;
    *dres = chi2p - best;
    *bres = best_idx;
    *nres = (int8_t)t;
}

static void* orc_worker(void* arg) {
    orc_job* jb = (orc_job*)arg;
    const int nf = jb->nf, nfit = jb->nfit;
    double* A = (double*)malloc(sizeof(double) * (size_t)nfit * nfit);
    double* M = (double*)malloc(sizeof(double) * (size_t)nfit * nfit);
    double* Lb = (double*)malloc(sizeof(double) * (size_t)nfit * nfit);
    double* col = (double*)malloc(sizeof(double) * (size_t)nfit);
    double* r = (double*)malloc(sizeof(double) * (size_t)nfit);
    double* d = (double*)malloc(sizeof(double) * (size_t)nfit);
    float* z = (float*)malloc(sizeof(float) * (size_t)(nf + 4));
    float* dfitf = (float*)malloc(sizeof(float) * (size_t)nfit);
    const int64_t total = jb->us ? (int64_t)jb->P : (int64_t)jb->P * jb->U;
    for (int64_t w = jb->tid; w < total && jb->status == 0; w += jb->nthreads) {
        const int ip = jb->us ? (int)w : (int)(w / jb->U);
        const int u = jb->us ? jb->us[w] : (int)(w % jb->U);
        const size_t o = jb->us ? (size_t)w : (size_t)ip * jb->U + u;
        double dr = NAN;
        int64_t br = -1;
        int8_t nr = 0;
        orc_fit_universe(jb, ip, u, A, M, Lb, col, r, d, z, dfitf, &dr, &br, &nr);
        jb->dchi2[o] = dr;
        if (jb->bestfit) jb->bestfit[o] = br;
        if (jb->nscans) jb->nscans[o] = nr;
    }
    free(A); free(M); free(Lb); free(col); free(r); free(d); free(z); free(dfitf);
    return NULL;
}

/* Prepare L_p and s_p in binary32 for every true point. */
static int orc_prepare_points(const double* S, const double* F, int nf, const int64_t* ps, int P, int fluct,
                              float* Lf, float* sf) {
    double* L = (double*)malloc(sizeof(double) * (size_t)nf * nf);
    int rc = 0;
    for (int ip = 0; ip < P && rc == 0; ++ip) {
        const double* s = S + (size_t)ps[ip] * nf;
        if (oracle_chol_sys(nf, s, F, fluct == ORC_FLUCT_GAUSS, L) != 0) { rc = -2; break; }
        for (size_t e = 0; e < (size_t)nf * nf; ++e) Lf[(size_t)ip * nf * nf + e] = (float)L[e];
        for (int i = 0; i < nf; ++i) sf[(size_t)ip * nf + i] = (float)s[i];
    }
    free(L);
    return rc;
}

/* Fake data only: dfit[P][U][nfit]. Returns 0 or -2 (not SPD). */
int oracle_fake_data(const double* S, int64_t G, int nf, const int32_t* collapse, int nfit, const double* F,
                     const int64_t* ps, int P, uint64_t seed, int U, int fluct, float* dfit) {
    (void)G;
    float* Lf = (float*)malloc(sizeof(float) * (size_t)P * nf * nf);
    float* sf = (float*)malloc(sizeof(float) * (size_t)P * nf);
    float* z = (float*)malloc(sizeof(float) * (size_t)(nf + 4));
    int rc = orc_prepare_points(S, F, nf, ps, P, fluct, Lf, sf);
    for (int ip = 0; ip < P && rc == 0; ++ip)
        for (int u = 0; u < U; ++u)
            orc_fake_one(nf, nfit, collapse, sf + (size_t)ip * nf, Lf + (size_t)ip * nf * nf, seed,
                         (uint32_t)ps[ip], (uint32_t)u, fluct, z, dfit + ((size_t)ip * U + u) * nfit);
    free(Lf); free(sf); free(z);
    return rc;
}

static int orc_run(const double* S, int64_t G, int nf, const int32_t* collapse, int nfit, const double* F,
                   const int64_t* ps, const int32_t* us, const float* data, int P, uint64_t seed, int U, int max_iter,
                   int fluct, int cov, int nthreads, double* dchi2, int64_t* bestfit, int8_t* nscans,
                   float* dfit_out);

/* Full FC pass: for every true point ps[ip] and universe u, the dchi2 of
 * Algorithm 1 with the covariance refit of §2.  Threaded over universes.
 * Returns 0, -1 (bad argument) or -2 (covariance not SPD). */
int oracle_run_points(const double* S, int64_t G, int nf, const int32_t* collapse, int nfit, const double* F,
                      const int64_t* ps, int P, uint64_t seed, int U, int max_iter, int fluct, int cov,
                      int nthreads, double* dchi2, int64_t* bestfit, int8_t* nscans, float* dfit_out) {
    return orc_run(S, G, nf, collapse, nfit, F, ps, NULL, NULL, P, seed, U, max_iter, fluct, cov, nthreads, dchi2,
                   bestfit, nscans, dfit_out);
}

/* The same procedure for n sampled universes: sample i is universe us[i] of
 * true point ps[i] (each universe's random numbers depend only on (seed,
 * point, universe), so a sample equals that entry of a full pass). */
int oracle_run_samples(const double* S, int64_t G, int nf, const int32_t* collapse, int nfit, const double* F,
                       const int64_t* ps, const int32_t* us, int n, uint64_t seed, int max_iter, int fluct, int cov,
                       int nthreads, double* dchi2, int64_t* bestfit, int8_t* nscans) {
    if (!us) return -1;
    for (int i = 0; i < n; ++i)
        if (us[i] < 0) return -1;
    return orc_run(S, G, nf, collapse, nfit, F, ps, us, NULL, n, seed, 1, max_iter, fluct, cov, nthreads, dchi2,
                   bestfit, nscans, NULL);
}

/* The observed data's dchi2 at each grid point ps[i]: the per-universe
 * procedure of §2 with the given fit-space data vector in place of fake data
 * (first covariance at ps[i], refit, dchi2 under the last scan's A), so it is
 * comparable with the distribution of ps[i]'s universes (Fig. 1 critical
 * values). */
int oracle_run_data(const double* S, int64_t G, int nf, const int32_t* collapse, int nfit, const double* F,
                    const int64_t* ps, int n, const float* data, int max_iter, int cov, int nthreads, double* dchi2,
                    int64_t* bestfit, int8_t* nscans) {
    if (!data) return -1;
    return orc_run(S, G, nf, collapse, nfit, F, ps, NULL, data, n, 0, 1, max_iter, ORC_FLUCT_POISSON_SYS, cov,
                   nthreads, dchi2, bestfit, nscans, NULL);
}

static int orc_run(const double* S, int64_t G, int nf, const int32_t* collapse, int nfit, const double* F,
                   const int64_t* ps, const int32_t* us, const float* data, int P, uint64_t seed, int U, int max_iter,
                   int fluct, int cov, int nthreads, double* dchi2, int64_t* bestfit, int8_t* nscans,
                   float* dfit_out) {
    if (G <= 0 || nf <= 0 || nfit <= 0 || P < 0 || U < 0 || max_iter < 1) return -1;
    for (int ip = 0; ip < P; ++ip)
        if (ps[ip] < 0 || ps[ip] >= G) return -1;
    if (nthreads < 1) nthreads = 1;
    double* Sfit = (double*)malloc(sizeof(double) * (size_t)G * nfit);
    oracle_collapse_spectra(G, nf, nfit, collapse, S, Sfit);
    float* Lf = (float*)malloc(sizeof(float) * (size_t)(P > 0 ? P : 1) * nf * nf);
    float* sf = (float*)malloc(sizeof(float) * (size_t)(P > 0 ? P : 1) * nf);
    int rc = orc_prepare_points(S, F, nf, ps, P, fluct, Lf, sf);
    if (rc == 0) {
        orc_job* jobs = (orc_job*)calloc((size_t)nthreads, sizeof(orc_job));
        pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
        for (int t = 0; t < nthreads; ++t) {
            orc_job* jb = &jobs[t];
            jb->S = S; jb->Sfit = Sfit; jb->F = F; jb->collapse = collapse; jb->G = G;
            jb->nf = nf; jb->nfit = nfit; jb->ps = ps; jb->us = us; jb->data = data; jb->P = P; jb->U = U;
            jb->seed = seed;
            jb->max_iter = max_iter; jb->fluct = fluct; jb->cov = cov; jb->Lf = Lf; jb->sf = sf;
            jb->dchi2 = dchi2; jb->bestfit = bestfit; jb->nscans = nscans; jb->dfit_out = dfit_out;
            jb->nthreads = nthreads; jb->tid = t; jb->status = 0;
        }
        if (nthreads == 1) {
            orc_worker(&jobs[0]);
        } else {
            for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_worker, &jobs[t]);
            for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
        }
        for (int t = 0; t < nthreads; ++t)
            if (jobs[t].status != 0) rc = jobs[t].status;
        free(jobs);
        free(th);
    }
    free(Sfit); free(Lf); free(sf);
    return rc;
}
