/*
 * cnn_oracle.c -- plain FP64 CPU reference of the learned-initialisation
 * network (TEST INFRASTRUCTURE ONLY; shares nothing with the CUDA path).
 *
 * The network maps a 2 x H x W input (support samples / 255 on the support
 * area, 0 elsewhere; the support indicator) to a 1 x H x W estimate of the
 * extrapolation area.  Four 3x3 convolutions with "same" zero padding and
 * dilations 1, 2, 4, 8; channels 2 -> 32 -> 32 -> 32 -> 1; ReLU after the
 * first three.  Parameters are one flat vector:
 *   W1[32][2][3][3] b1[32] W2[32][32][3][3] b2[32] W3[32][32][3][3] b3[32]
 *   W4[1][32][3][3] b4[1]                                  (19393 values)
 * Convolution (cross-correlation, as in common CNN practice):
 *   y[co][i][j] = b[co] + sum_ci sum_ky sum_kx W[co][ci][ky][kx]
 *                 * x[ci][i + (ky-1) d][j + (kx-1) d]     (0 outside)
 * Loss: L = sum over the batch of lam[i][j] (out[i][j] - t[i][j])^2 / count,
 * count = N H W.  Optimiser: Adam with bias correction.
 *
 * With round_bf16 != 0 the weights, the input and every stored activation are
 * rounded to bfloat16 (round to nearest, ties to even) as the GPU kernels
 * store them; arithmetic stays FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CNN_LAYERS 4
static const int kCin[CNN_LAYERS] = {2, 32, 32, 32};
static const int kCout[CNN_LAYERS] = {32, 32, 32, 1};
static const int kDil[CNN_LAYERS] = {1, 2, 4, 8};

int oracle_cnn_param_count(void)
{
    int n = 0;
    for (int l = 0; l < CNN_LAYERS; ++l) n += kCout[l] * kCin[l] * 9 + kCout[l];
    return n;
}

/* bfloat16 rounding of a value representable as float: round the FP32
 * significand to 8 bits, ties to even (NaN and infinity are not expected). */
double oracle_bf16(double v)
{
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    u &= 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

void oracle_conv3x3_fwd(int N, int H, int W, int Cin, int Cout, int dil, const double *x,
                        const double *w, const double *b, double *y)
{
    for (int n = 0; n < N; ++n)
        for (int co = 0; co < Cout; ++co)
            for (int i = 0; i < H; ++i)
                for (int j = 0; j < W; ++j) {
                    double acc = b ? b[co] : 0.0;
                    for (int ci = 0; ci < Cin; ++ci)
                        for (int ky = 0; ky < 3; ++ky)
                            for (int kx = 0; kx < 3; ++kx) {
                                int yy = i + (ky - 1) * dil, xx = j + (kx - 1) * dil;
                                if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                                acc += w[((co * Cin + ci) * 3 + ky) * 3 + kx] *
                                       x[((long)(n * Cin + ci) * H + yy) * W + xx];
                            }
                    y[((long)(n * Cout + co) * H + i) * W + j] = acc;
                }
}

/* Gradients of the convolution given dL/dy: dx (may be NULL), dw, db
 * (accumulated into, caller zeroes them). */
void oracle_conv3x3_bwd(int N, int H, int W, int Cin, int Cout, int dil, const double *x,
                        const double *w, const double *dy, double *dx, double *dw, double *db)
{
    if (dx) memset(dx, 0, sizeof(double) * (size_t)N * Cin * H * W);
    for (int n = 0; n < N; ++n)
        for (int co = 0; co < Cout; ++co)
            for (int i = 0; i < H; ++i)
                for (int j = 0; j < W; ++j) {
                    double g = dy[((long)(n * Cout + co) * H + i) * W + j];
                    if (db) db[co] += g;
                    for (int ci = 0; ci < Cin; ++ci)
                        for (int ky = 0; ky < 3; ++ky)
                            for (int kx = 0; kx < 3; ++kx) {
                                int yy = i + (ky - 1) * dil, xx = j + (kx - 1) * dil;
                                if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                                long xi = ((long)(n * Cin + ci) * H + yy) * W + xx;
                                int wi = ((co * Cin + ci) * 3 + ky) * 3 + kx;
                                if (dw) dw[wi] += g * x[xi];
                                if (dx) dx[xi] += g * w[wi];
                            }
                }
}

static const double *layer_w(const double *p, int l)
{
    for (int k = 0; k < l; ++k) p += kCout[k] * kCin[k] * 9 + kCout[k];
    return p;
}

/* Forward pass.  acts (optional) receives the four layer outputs after the
 * activation (layer 4: no activation), each N x Cout x H x W, concatenated.
 * out: N x H x W. */
int oracle_cnn_forward(int N, int H, int W, const double *params, const double *x_in, double *out,
                       double *acts, int round_bf16)
{
    long plane = (long)H * W;
    double *cur = malloc(sizeof(double) * N * 2 * plane);
    double *wtmp = malloc(sizeof(double) * 32 * 32 * 9);
    if (!cur || !wtmp) { free(cur); free(wtmp); return -1; }
    for (long t = 0; t < N * 2 * plane; ++t) cur[t] = round_bf16 ? oracle_bf16(x_in[t]) : x_in[t];
    long aoff = 0;
    for (int l = 0; l < CNN_LAYERS; ++l) {
        const double *w = layer_w(params, l);
        int nw = kCout[l] * kCin[l] * 9;
        const double *b = w + nw;
        for (int t = 0; t < nw; ++t) wtmp[t] = round_bf16 ? oracle_bf16(w[t]) : w[t];
        double *nxt = malloc(sizeof(double) * N * kCout[l] * plane);
        if (!nxt) { free(cur); free(wtmp); return -1; }
        oracle_conv3x3_fwd(N, H, W, kCin[l], kCout[l], kDil[l], cur, wtmp, b, nxt);
        long cnt = (long)N * kCout[l] * plane;
        for (long t = 0; t < cnt; ++t) {
            double v = nxt[t];
            if (l < CNN_LAYERS - 1) {
                v = v > 0.0 ? v : 0.0;
                if (round_bf16) v = oracle_bf16(v);
            }
            nxt[t] = v;
        }
        if (acts) { memcpy(acts + aoff, nxt, sizeof(double) * cnt); aoff += cnt; }
        free(cur);
        cur = nxt;
    }
    memcpy(out, cur, sizeof(double) * N * plane);
    free(cur);
    free(wtmp);
    return 0;
}

/* Loss and gradient with respect to all parameters (and optionally the
 * input).  Backward: dL/dout = 2 lam (out - t) / (N H W); for each layer,
 * ReLU gates the gradient by (activation > 0); weight and bias gradients of
 * the convolution; data gradient through the (bf16-rounded) weights. */
double oracle_cnn_loss_grad(int N, int H, int W, const double *params, const double *x_in,
                            const double *target, const double *lam, double *grad, double *grad_x,
                            int round_bf16)
{
    long plane = (long)H * W;
    long act_total = 0;
    for (int l = 0; l < CNN_LAYERS; ++l) act_total += (long)N * kCout[l] * plane;
    double *acts = malloc(sizeof(double) * act_total);
    double *out = malloc(sizeof(double) * N * plane);
    double *x0 = malloc(sizeof(double) * N * 2 * plane);
    double *wtmp = malloc(sizeof(double) * 32 * 32 * 9);
    double *dcur = malloc(sizeof(double) * N * 32 * plane);
    double *dprev = malloc(sizeof(double) * N * 32 * plane);
    if (!acts || !out || !x0 || !wtmp || !dcur || !dprev) {
        free(acts); free(out); free(x0); free(wtmp); free(dcur); free(dprev);
        return NAN;
    }
    oracle_cnn_forward(N, H, W, params, x_in, out, acts, round_bf16);
    for (long t = 0; t < N * 2 * plane; ++t) x0[t] = round_bf16 ? oracle_bf16(x_in[t]) : x_in[t];
    double count = (double)N * plane, loss = 0.0;
    for (long t = 0; t < N * plane; ++t) {
        double e = out[t] - target[t];
        double lw = lam ? lam[t] : 1.0;
        loss += lw * e * e;
        dcur[t] = 2.0 * lw * e / count;
    }
    loss /= count;
    memset(grad, 0, sizeof(double) * oracle_cnn_param_count());
    long aoff[CNN_LAYERS];
    {
        long o = 0;
        for (int l = 0; l < CNN_LAYERS; ++l) { aoff[l] = o; o += (long)N * kCout[l] * plane; }
    }
    for (int l = CNN_LAYERS - 1; l >= 0; --l) {
        const double *w = layer_w(params, l);
        int nw = kCout[l] * kCin[l] * 9;
        long goff = layer_w(params, l) - params;
        for (int t = 0; t < nw; ++t) wtmp[t] = round_bf16 ? oracle_bf16(w[t]) : w[t];
        const double *xin = l == 0 ? x0 : acts + aoff[l - 1];
        int need_dx = l > 0 || grad_x;
        oracle_conv3x3_bwd(N, H, W, kCin[l], kCout[l], kDil[l], xin, wtmp, dcur, need_dx ? dprev : NULL,
                           grad + goff, grad + goff + nw);
        if (l > 0) {
            const double *a = acts + aoff[l - 1];
            long cnt = (long)N * kCin[l] * plane;
            for (long t = 0; t < cnt; ++t) dcur[t] = a[t] > 0.0 ? dprev[t] : 0.0;
        } else if (grad_x) {
            memcpy(grad_x, dprev, sizeof(double) * N * 2 * plane);
        }
    }
    free(acts); free(out); free(x0); free(wtmp); free(dcur); free(dprev);
    return loss;
}

/* One Adam step on a flat parameter vector (step t >= 1). */
void oracle_adam(int n, double *p, double *m, double *v, const double *g, double lr, double b1, double b2,
                 double eps, int t)
{
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}
