/*
 * fse3_oracle.c -- plain FP64 CPU reference of complex-valued FSE on video
 * volumes (TEST INFRASTRUCTURE ONLY; shares nothing with the CUDA path).
 *
 * The paper states that the method extends to higher-dimensional data such as
 * video (Section II, and the Conclusion, both citing Meisinger's extension):
 * the same Algorithm 1 with a 3-D transform, 3-D basis functions
 *   phi_(w,u,v)[t,m,n] = e^{j 2 pi (w t / Ft + u m / F + v n / F)}
 * and 3-D circular shifts.  Readings (also in the design notes):
 *   - the extrapolation volume is M x M samples in each of T consecutive
 *     frames centred on the lost block's frame; B is the b x b block in the
 *     centre frame; the transform grid is Ft x F x F (Ft >= T, F >= M, powers
 *     of two), the volume sitting at offset ((Ft - T) / 2, (F - M) / 2,
 *     (F - M) / 2) with weight 0 on the padding;
 *   - the weighting function is Eq. (3) with the Euclidean distance in
 *     samples extended by the frame offset:
 *       w[t,m,n] = rho^sqrt((t - (T-1)/2)^2 + (m - (M-1)/2)^2 + (n - (M-1)/2)^2);
 *   - bins are indexed p = (w Ft-plane, u, v) -> (w F + u) F + v, argmax ties
 *     to the smallest p; a support of zero total weight gives the zero model.
 * Every function follows the definitions literally, in double precision.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE3_PI 3.14159265358979323846264338327950288

static int pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* 1-D DFT of length n at the given stride, by the definition (O(n^2)); the
 * 3-D oracle transforms are small enough for that and it keeps this file
 * independent of the 2-D oracle's FFT. */
static void dft1d(int n, double *re, double *im, long stride, int sign, double *tr, double *ti,
                  const double *cs, const double *sn)
{
    for (int k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (int t = 0; t < n; ++t) {
            const int q = (int)(((long)k * t) % n);   /* angle sign * 2 pi q / n */
            double c = cs[q], s = sign * sn[q];
            double xr = re[t * stride], xi = im[t * stride];
            sr += xr * c - xi * s;
            si += xr * s + xi * c;
        }
        tr[k] = sr;
        ti[k] = si;
    }
    for (int k = 0; k < n; ++k) { re[k * stride] = tr[k]; im[k * stride] = ti[k]; }
}

/* 3-D DFT of an Ft x F x F row-major complex array, in place, unnormalised
 * (sign -1 forward).  Returns 0, or -1 on bad sizes. */
int oracle_fft3(int Ft, int F, double *re, double *im, int sign)
{
    if (!pow2(F) || !pow2(Ft)) return -1;
    int nmax = F > Ft ? F : Ft;
    double *tr = malloc(sizeof(double) * nmax), *ti = malloc(sizeof(double) * nmax);
    double *cF = malloc(sizeof(double) * F), *sF = malloc(sizeof(double) * F);
    double *cT = malloc(sizeof(double) * Ft), *sT = malloc(sizeof(double) * Ft);
    if (!tr || !ti || !cF || !sF || !cT || !sT) {
        free(tr); free(ti); free(cF); free(sF); free(cT); free(sT);
        return -1;
    }
    for (int q = 0; q < F; ++q) { cF[q] = cos(2.0 * ORACLE3_PI * q / F); sF[q] = sin(2.0 * ORACLE3_PI * q / F); }
    for (int q = 0; q < Ft; ++q) { cT[q] = cos(2.0 * ORACLE3_PI * q / Ft); sT[q] = sin(2.0 * ORACLE3_PI * q / Ft); }
    long FF = (long)F * F;
    for (int t = 0; t < Ft; ++t)
        for (int m = 0; m < F; ++m)
            dft1d(F, re + t * FF + (long)m * F, im + t * FF + (long)m * F, 1, sign, tr, ti, cF, sF);
    for (int t = 0; t < Ft; ++t)
        for (int n = 0; n < F; ++n) dft1d(F, re + t * FF + n, im + t * FF + n, F, sign, tr, ti, cF, sF);
    for (long q = 0; q < FF; ++q) dft1d(Ft, re + q, im + q, FF, sign, tr, ti, cT, sT);
    free(tr); free(ti); free(cF); free(sF); free(cT); free(sT);
    return 0;
}

/* Weighting function on a T x M x M volume (support[t*M*M + m*M + n] != 0
 * marks A). */
void oracle_weight3(int T, int M, double rho, const uint8_t *support, double *w)
{
    double ct = 0.5 * (T - 1), c = 0.5 * (M - 1);
    for (int t = 0; t < T; ++t)
        for (int m = 0; m < M; ++m)
            for (int n = 0; n < M; ++n) {
                long p = ((long)t * M + m) * M + n;
                double d = sqrt((t - ct) * (t - ct) + (m - c) * (m - c) + (n - c) * (n - c));
                w[p] = support[p] ? pow(rho, d) : 0.0;
            }
}

/*
 * Algorithm 1 on an Ft x F x F grid.  Arguments and outputs as the 2-D
 * oracle_cfse (s_im NULL for a real signal; forced NULL or I indices);
 * g receives the complex model over the grid (interleaved re, im).
 */
int oracle_cfse3(int Ft, int F, const double *s, const double *s_im, const double *w, double gamma,
                 int iters, const int32_t *forced, int32_t *sel, double *coef, double *e_sel,
                 double *e_max, double *g)
{
    if (!pow2(F) || !pow2(Ft) || iters < 0) return -1;
    long FF = (long)F * F, P = (long)Ft * FF;
    double *Rr = calloc(P, sizeof(double)), *Ri = calloc(P, sizeof(double));
    double *Wr = calloc(P, sizeof(double)), *Wi = calloc(P, sizeof(double));
    double *Gr = calloc(P, sizeof(double)), *Gi = calloc(P, sizeof(double));
    if (!Rr || !Ri || !Wr || !Wi || !Gr || !Gi) {
        free(Rr); free(Ri); free(Wr); free(Wi); free(Gr); free(Gi);
        return -1;
    }
    /* R_w = DFT{s w}, W = DFT{w}, W0bar = 1 / W[0,0,0] */
    for (long p = 0; p < P; ++p) {
        Rr[p] = s[p] * w[p];
        Ri[p] = s_im ? s_im[p] * w[p] : 0.0;
        Wr[p] = w[p];
    }
    oracle_fft3(Ft, F, Rr, Ri, -1);
    oracle_fft3(Ft, F, Wr, Wi, -1);
    double W0bar = Wr[0] > 0.0 ? 1.0 / Wr[0] : 0.0;
    for (int nu = 0; nu < iters; ++nu) {
        long best = 0;
        double bmax = -1.0;
        for (long p = 0; p < P; ++p) {
            double e = Rr[p] * Rr[p] + Ri[p] * Ri[p];
            if (e > bmax) { bmax = e; best = p; }
        }
        long pick = forced ? (long)forced[nu] : best;
        if (pick < 0 || pick >= P) pick = best;
        int tw = (int)(pick / FF), u = (int)((pick / F) % F), v = (int)(pick % F);
        double cr = gamma * Rr[pick] * W0bar, ci = gamma * Ri[pick] * W0bar;
        if (sel) sel[nu] = (int32_t)pick;
        if (coef) { coef[2 * nu] = cr; coef[2 * nu + 1] = ci; }
        if (e_sel) e_sel[nu] = Rr[pick] * Rr[pick] + Ri[pick] * Ri[pick];
        if (e_max) e_max[nu] = bmax;
        /* model: G[w,u,v] += Ft F^2 c;  residual: R[t,k,l] -= c W[t-w, k-u, l-v] */
        Gr[pick] += (double)P * cr;
        Gi[pick] += (double)P * ci;
        for (int t = 0; t < Ft; ++t)
            for (int k = 0; k < F; ++k)
                for (int l = 0; l < F; ++l) {
                    long q = (((long)((t - tw + Ft) % Ft) * F + (k - u + F) % F) * F) + (l - v + F) % F;
                    long p = ((long)t * F + k) * F + l;
                    Rr[p] -= cr * Wr[q] - ci * Wi[q];
                    Ri[p] -= cr * Wi[q] + ci * Wr[q];
                }
    }
    if (g) {
        oracle_fft3(Ft, F, Gr, Gi, +1);
        for (long p = 0; p < P; ++p) { g[2 * p] = Gr[p] / (double)P; g[2 * p + 1] = Gi[p] / (double)P; }
    }
    free(Rr); free(Ri); free(Wr); free(Wi); free(Gr); free(Gi);
    return 0;
}

/*
 * The spatial-domain definitions of Section III on the 3-D grid, brute force:
 * residual r = s - g, weighted projection onto every basis function,
 * criterion |p|^2 sum phi* w phi, c = gamma p, g += c phi.  O(I (Ft F^2)^2).
 */
int oracle_cfse3_spatial(int Ft, int F, const double *s, const double *s_im, const double *w,
                         double gamma, int iters, int32_t *sel, double *coef, double *g)
{
    if (F <= 0 || Ft <= 0 || iters < 0) return -1;
    long FF = (long)F * F, P = (long)Ft * FF;
    double *gr = calloc(P, sizeof(double)), *gi = calloc(P, sizeof(double));
    if (!gr || !gi) { free(gr); free(gi); return -1; }
    for (int nu = 0; nu < iters; ++nu) {
        long best = 0;
        double bcrit = -1.0, bpr = 0.0, bpi = 0.0;
        for (long b = 0; b < P; ++b) {
            int bw = (int)(b / FF), bu = (int)((b / F) % F), bv = (int)(b % F);
            double nr = 0.0, ni = 0.0, den = 0.0;
            for (long p = 0; p < P; ++p) {
                int t = (int)(p / FF), m = (int)((p / F) % F), n = (int)(p % F);
                double ang = 2.0 * ORACLE3_PI * ((double)(((long)bw * t) % Ft) / Ft +
                                                 (double)(((long)bu * m + (long)bv * n) % F) / F);
                double c = cos(ang), sn = sin(ang);
                double rr = s[p] - gr[p], ri = (s_im ? s_im[p] : 0.0) - gi[p];
                nr += w[p] * (rr * c + ri * sn);
                ni += w[p] * (ri * c - rr * sn);
                den += w[p];
            }
            double pr = den > 0.0 ? nr / den : 0.0, pi = den > 0.0 ? ni / den : 0.0;
            double crit = (pr * pr + pi * pi) * den;
            if (crit > bcrit) { bcrit = crit; best = b; bpr = pr; bpi = pi; }
        }
        int bw = (int)(best / FF), bu = (int)((best / F) % F), bv = (int)(best % F);
        double cr = gamma * bpr, ci = gamma * bpi;
        if (sel) sel[nu] = (int32_t)best;
        if (coef) { coef[2 * nu] = cr; coef[2 * nu + 1] = ci; }
        for (long p = 0; p < P; ++p) {
            int t = (int)(p / FF), m = (int)((p / F) % F), n = (int)(p % F);
            double ang = 2.0 * ORACLE3_PI * ((double)(((long)bw * t) % Ft) / Ft +
                                             (double)(((long)bu * m + (long)bv * n) % F) / F);
            gr[p] += cr * cos(ang) - ci * sin(ang);
            gi[p] += cr * sin(ang) + ci * cos(ang);
        }
    }
    if (g) for (long p = 0; p < P; ++p) { g[2 * p] = gr[p]; g[2 * p + 1] = gi[p]; }
    free(gr);
    free(gi);
    return 0;
}
