/*
 * fse_oracle.c -- plain FP64 CPU reference of complex-valued Frequency
 * Selective Extrapolation (cFSE, Seiler & Kaup, arXiv 2204.14193).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * Every function follows the paper's definitions literally, in double
 * precision, without blocking, fusion or reordering:
 *   - oracle_fft2 / oracle_dft2_direct: the 2-D DFT of Eq. (7) (forward sign
 *     e^{-j}), the transform Algorithm 1 calls FFT, and its inverse.
 *   - oracle_weight: the weighting function of Eq. (3).
 *   - oracle_cfse: Algorithm 1 (frequency-domain cFSE), steps in the
 *     algorithm's order.
 *   - oracle_cfse_spatial: the spatial-domain definition of Section III
 *     (residual, weighted projection, selection criterion, model and residual
 *     updates) evaluated by brute force.
 *
 * Readings of points the paper leaves open (also listed in the design notes):
 *   - the DFT period is the FFT size F (Eq. (1) writes M, N; Section IV uses a
 *     64x64 FFT for a 48x48 area), so "MN" in Eq. (15) is F*F;
 *   - argmax ties go to the smallest linear index k*F+l;
 *   - a support with zero total weight (W[0,0] == 0) yields the zero model.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------ */
/* 1-D radix-2 decimation-in-time FFT, in place, length n (power of two).   */
/* sign = -1: X[k] = sum_t x[t] e^{-j 2 pi k t / n}; sign = +1: e^{+j...}.  */
/* Twiddles are evaluated directly with cos/sin of the exact angle.         */
/* ------------------------------------------------------------------------ */
static void fft1d(int n, double *re, double *im, long stride, int sign)
{
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double tr = re[i * stride], ti = im[i * stride];
            re[i * stride] = re[j * stride]; im[i * stride] = im[j * stride];
            re[j * stride] = tr; im[j * stride] = ti;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int k = 0; k < half; ++k) {
            double ang = sign * 2.0 * ORACLE_PI * (double)k / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int start = 0; start < n; start += len) {
                long a = (long)(start + k) * stride, b = (long)(start + k + half) * stride;
                double xr = re[b] * wr - im[b] * wi;
                double xi = re[b] * wi + im[b] * wr;
                re[b] = re[a] - xr; im[b] = im[a] - xi;
                re[a] += xr;        im[a] += xi;
            }
        }
    }
}

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* 2-D DFT of an F x F row-major complex array, in place, unnormalised.
 * Returns 0 on success, -1 if F is not a power of two. */
int oracle_fft2(int F, double *re, double *im, int sign)
{
    if (!is_pow2(F)) return -1;
    for (int r = 0; r < F; ++r) fft1d(F, re + (long)r * F, im + (long)r * F, 1, sign);
    for (int c = 0; c < F; ++c) fft1d(F, re + c, im + c, F, sign);
    return 0;
}

/* The 2-D DFT written out as the double sum of Eq. (7): O(F^4). */
void oracle_dft2_direct(int F, const double *re, const double *im,
                        double *ore, double *oim, int sign)
{
    for (int k = 0; k < F; ++k)
        for (int l = 0; l < F; ++l) {
            double sr = 0.0, si = 0.0;
            for (int m = 0; m < F; ++m)
                for (int n = 0; n < F; ++n) {
                    long ph = ((long)k * m + (long)l * n) % F;
                    double ang = sign * 2.0 * ORACLE_PI * (double)ph / (double)F;
                    double c = cos(ang), s = sin(ang);
                    double xr = re[m * F + n], xi = im[m * F + n];
                    sr += xr * c - xi * s;
                    si += xr * s + xi * c;
                }
            ore[k * F + l] = sr;
            oim[k * F + l] = si;
        }
}

/* Eq. (3): w[m,n] = rho^sqrt((m-(M-1)/2)^2 + (n-(N-1)/2)^2) on the support
 * area A (support[m*N+n] != 0) and 0 on the loss area B. */
void oracle_weight(int M, int N, double rho, const uint8_t *support, double *w)
{
    double cm = 0.5 * (M - 1), cn = 0.5 * (N - 1);
    for (int m = 0; m < M; ++m)
        for (int n = 0; n < N; ++n) {
            double d = sqrt((m - cm) * (m - cm) + (n - cn) * (n - cn));
            w[m * N + n] = support[m * N + n] ? pow(rho, d) : 0.0;
        }
}

/*
 * Algorithm 1 on an F x F grid.
 *   s, s_im   : input signal (F*F, row-major); s_im = NULL for a real
 *               signal (images), else its imaginary part;
 *   w         : weighting function (F*F), 0 wherever a sample is not support.
 *   gamma     : orthogonality-deficiency compensation factor.
 *   iters     : I, number of selections.
 *   forced    : NULL (free run) or I linear indices k*F+l that replace the
 *               argmax of each iteration (guided replay).
 * Outputs (any may be NULL):
 *   sel[I]        selected linear index per iteration,
 *   coef[2I]      (re, im) of c-hat per iteration,
 *   e_sel[I]      |R_w[u,v]|^2 of the selected bin before the update,
 *   e_max[I]      max_k |R_w[k]|^2 before the update,
 *   e_second[I]   largest |R_w[k]|^2 over the bins other than the argmax,
 *   g[2F^2]       the complex model g = IFFT{G} (interleaved re, im),
 *   R_out[2F^2]   the weighted-residual spectrum after the last iteration,
 *   W_out[2F^2]   the spectrum W of w.
 * Returns 0, or -1 on a bad argument.
 */
int oracle_cfse_fixw(int F, const double *s, const double *s_im, const double *w,
                     double gamma, int iters, int wfix_from, const int32_t *forced, int32_t *sel,
                     double *coef, double *e_sel, double *e_max, double *e_second,
                     double *g, double *R_out, double *W_out);

int oracle_cfse(int F, const double *s, const double *s_im, const double *w,
                double gamma, int iters, const int32_t *forced, int32_t *sel, double *coef,
                double *e_sel, double *e_max, double *e_second,
                double *g, double *R_out, double *W_out)
{
    return oracle_cfse_fixw(F, s, s_im, w, gamma, iters, iters, forced, sel, coef, e_sel, e_max,
                            e_second, g, R_out, W_out);
}

/* The 16-bit fixed-point code of a spectrum value x of W: x / W[0,0] in
 * units of 1/32767, rounded to the nearest integer (ties to even) and held
 * to [-32767, 32767].  |W[k,l]| <= W[0,0] for a non-negative weight, so the
 * codes cover W without overflow.  The rounding decision is taken in FP32
 * (x and 1 / W[0,0] rounded to FP32, their product with 32767 rounded to
 * FP32), the precision in which the reduced-precision kernel decides it;
 * the value a code stands for, code W[0,0] / 32767, is FP64. */
int oracle_fix_code(double x, double W00)
{
    float rinv = 1.0f / (float)W00;
    float qs = 32767.0f * rinv;
    float t = (float)x * qs;
    double c = nearbyint((double)t);   /* default rounding mode: to nearest, ties to even */
    if (c > 32767.0) c = 32767.0;
    if (c < -32767.0) c = -32767.0;
    return (int)c;
}

/*
 * Algorithm 1 with reduced-precision residual storage: as oracle_cfse, but
 * the updates of iterations nu >= wfix_from (0-based) read W in 16-bit fixed
 * point (each real and imaginary part replaced by the value of its code,
 * oracle_fix_code; everything else stays FP64, and c-hat still divides by
 * the exact W[0,0]).  wfix_from >= iters is oracle_cfse itself.
 */
int oracle_cfse_fixw(int F, const double *s, const double *s_im, const double *w,
                     double gamma, int iters, int wfix_from, const int32_t *forced, int32_t *sel,
                     double *coef, double *e_sel, double *e_max, double *e_second,
                     double *g, double *R_out, double *W_out)
{
    if (!is_pow2(F) || iters < 0) return -1;
    long P = (long)F * F;
    double *Rr = calloc(P, sizeof(double)), *Ri = calloc(P, sizeof(double));
    double *Wr = calloc(P, sizeof(double)), *Wi = calloc(P, sizeof(double));
    double *Gr = calloc(P, sizeof(double)), *Gi = calloc(P, sizeof(double));
    if (!Rr || !Ri || !Wr || !Wi || !Gr || !Gi) {
        free(Rr); free(Ri); free(Wr); free(Wi); free(Gr); free(Gi);
        return -1;
    }
    /* R_w = FFT{s w}, W = FFT{w}, W0bar = 1 / W[0,0] */
    for (long p = 0; p < P; ++p) {
        Rr[p] = s[p] * w[p];
        Ri[p] = s_im ? s_im[p] * w[p] : 0.0;
        Wr[p] = w[p];
    }
    oracle_fft2(F, Rr, Ri, -1);
    oracle_fft2(F, Wr, Wi, -1);
    int have_support = Wr[0] > 0.0;
    double W0bar = have_support ? 1.0 / Wr[0] : 0.0;
    /* the fixed-point W read by the updates from iteration wfix_from on */
    double *Hr = NULL, *Hi = NULL;
    if (wfix_from < iters && have_support) {
        Hr = malloc(P * sizeof(double));
        Hi = malloc(P * sizeof(double));
        if (!Hr || !Hi) {
            free(Hr); free(Hi); free(Rr); free(Ri); free(Wr); free(Wi); free(Gr); free(Gi);
            return -1;
        }
        for (long p = 0; p < P; ++p) {
            Hr[p] = oracle_fix_code(Wr[p], Wr[0]) * Wr[0] / 32767.0;
            Hi[p] = oracle_fix_code(Wi[p], Wr[0]) * Wr[0] / 32767.0;
        }
    }

    for (int nu = 0; nu < iters; ++nu) {
        /* basis function selection: argmax |R_w|^2, ties -> smallest index */
        long best = 0;
        double bmax = -1.0;
        for (long p = 0; p < P; ++p) {
            double e = Rr[p] * Rr[p] + Ri[p] * Ri[p];
            if (e > bmax) { bmax = e; best = p; }
        }
        double sec = -1.0;
        for (long p = 0; p < P; ++p) {
            if (p == best) continue;
            double e = Rr[p] * Rr[p] + Ri[p] * Ri[p];
            if (e > sec) sec = e;
        }
        long pick = forced ? (long)forced[nu] : best;
        if (pick < 0 || pick >= P) pick = best;
        int u = (int)(pick / F), v = (int)(pick % F);
        double er = Rr[pick] * Rr[pick] + Ri[pick] * Ri[pick];
        /* expansion coefficient estimation: c = gamma R_w[u,v] W0bar */
        double cr = gamma * Rr[pick] * W0bar, ci = gamma * Ri[pick] * W0bar;
        if (sel) sel[nu] = (int32_t)pick;
        if (coef) { coef[2 * nu] = cr; coef[2 * nu + 1] = ci; }
        if (e_sel) e_sel[nu] = er;
        if (e_max) e_max[nu] = bmax;
        if (e_second) e_second[nu] = sec;
        /* model update: G[u,v] += F^2 c */
        Gr[pick] += (double)P * cr;
        Gi[pick] += (double)P * ci;
        /* residual update: R_w[k,l] -= c W[k-u, l-v] (indices modulo F) */
        const double *Ur = (Hr && nu >= wfix_from) ? Hr : Wr, *Ui = (Hr && nu >= wfix_from) ? Hi : Wi;
        for (int k = 0; k < F; ++k)
            for (int l = 0; l < F; ++l) {
                long q = (long)(((k - u) % F + F) % F) * F + (((l - v) % F + F) % F);
                double wr = Ur[q], wi = Ui[q];
                Rr[(long)k * F + l] -= cr * wr - ci * wi;
                Ri[(long)k * F + l] -= cr * wi + ci * wr;
            }
    }
    /* g = IFFT{G} (1/F^2 normalisation) */
    if (g) {
        oracle_fft2(F, Gr, Gi, +1);
        for (long p = 0; p < P; ++p) { g[2 * p] = Gr[p] / (double)P; g[2 * p + 1] = Gi[p] / (double)P; }
    }
    if (R_out) for (long p = 0; p < P; ++p) { R_out[2 * p] = Rr[p]; R_out[2 * p + 1] = Ri[p]; }
    if (W_out) for (long p = 0; p < P; ++p) { W_out[2 * p] = Wr[p]; W_out[2 * p + 1] = Wi[p]; }
    free(Rr); free(Ri); free(Wr); free(Wi); free(Gr); free(Gi); free(Hr); free(Hi);
    return 0;
}

/*
 * Section III in the spatial domain, brute force (O(I F^4)):
 *   r = s - g;  p_(k,l) = sum r phi* w / sum phi* w phi;
 *   (u,v) = argmax |p|^2 sum phi* w phi;  c = gamma p_(u,v);
 *   g += c phi_(u,v).
 * phi_(k,l)[m,n] = e^{j 2 pi (k m + l n) / F}.  Ties -> smallest k*F+l.
 * s_im = NULL for a real signal.  Outputs sel[I], coef[2I], crit[I] (the
 * maximised criterion) and g[2F^2].
 */
int oracle_cfse_spatial(int F, const double *s, const double *s_im, const double *w,
                        double gamma, int iters, int32_t *sel, double *coef, double *crit,
                        double *g)
{
    if (F <= 0 || iters < 0) return -1;
    long P = (long)F * F;
    double *gr = calloc(P, sizeof(double)), *gi = calloc(P, sizeof(double));
    double *ct = malloc(F * sizeof(double)), *st = malloc(F * sizeof(double));
    if (!gr || !gi || !ct || !st) { free(gr); free(gi); free(ct); free(st); return -1; }
    for (int t = 0; t < F; ++t) {
        ct[t] = cos(2.0 * ORACLE_PI * t / F);
        st[t] = sin(2.0 * ORACLE_PI * t / F);
    }
    for (int nu = 0; nu < iters; ++nu) {
        long best = 0;
        double bcrit = -1.0, bpr = 0.0, bpi = 0.0;
        for (int k = 0; k < F; ++k)
            for (int l = 0; l < F; ++l) {
                double nr = 0.0, ni = 0.0, den = 0.0;
                for (int m = 0; m < F; ++m)
                    for (int n = 0; n < F; ++n) {
                        long p = (long)m * F + n;
                        int ph = (int)(((long)k * m + (long)l * n) % F);
                        /* r phi* w with phi* = cos - j sin */
                        double rr = s[p] - gr[p], ri = (s_im ? s_im[p] : 0.0) - gi[p];
                        nr += w[p] * (rr * ct[ph] + ri * st[ph]);
                        ni += w[p] * (ri * ct[ph] - rr * st[ph]);
                        /* phi* w phi = w */
                        den += w[p] * (ct[ph] * ct[ph] + st[ph] * st[ph]);
                    }
                double pr = den > 0.0 ? nr / den : 0.0, pi = den > 0.0 ? ni / den : 0.0;
                double c = (pr * pr + pi * pi) * den;
                if (c > bcrit) { bcrit = c; best = (long)k * F + l; bpr = pr; bpi = pi; }
            }
        int u = (int)(best / F), v = (int)(best % F);
        double cr = gamma * bpr, ci = gamma * bpi;
        if (sel) sel[nu] = (int32_t)best;
        if (coef) { coef[2 * nu] = cr; coef[2 * nu + 1] = ci; }
        if (crit) crit[nu] = bcrit;
        for (int m = 0; m < F; ++m)
            for (int n = 0; n < F; ++n) {
                int ph = (int)(((long)u * m + (long)v * n) % F);
                long p = (long)m * F + n;
                gr[p] += cr * ct[ph] - ci * st[ph];
                gi[p] += cr * st[ph] + ci * ct[ph];
            }
    }
    if (g) for (long p = 0; p < P; ++p) { g[2 * p] = gr[p]; g[2 * p + 1] = gi[p]; }
    free(gr); free(gi); free(ct); free(st);
    return 0;
}
