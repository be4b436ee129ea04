// fse_cnn.cu -- C ABI of the learned-initialisation network (see
// include/fse.h): parameter handling, inference, gradient evaluation and
// Adam training steps, all on the GPU with the kernels of fse_cnn.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "fse.h"
#include "fse_alloc.cuh"
#include "fse_cnn.cuh"

using namespace fse_net;

struct fse_cnn {
    int device = 0;
    int H = 0, W = 0, max_batch = 0;
    float *params = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    __nv_bfloat16 *wb = nullptr;
    float *wt = nullptr;
    __nv_bfloat16 *xin = nullptr, *act[3] = {nullptr, nullptr, nullptr};
    float *y = nullptr, *gy = nullptr, *g0 = nullptr, *g1 = nullptr, *part = nullptr;
    double *lpart = nullptr, *loss = nullptr;
    int nparts_max = 0;
    int step = 0;
    std::string err = "no error";
};

namespace {

thread_local std::string g_cnn_err = "no error";

fse_status cfail(fse_cnn *c, fse_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_cnn_err = buf;
    return st;
}

#define CNN_CUDA(c, call)                                                                                 \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return cfail((c), e_ == cudaErrorMemoryAllocation ? FSE_ERR_OOM : FSE_ERR_CUDA, "%s: %s", #call, \
                         cudaGetErrorString(e_));                                                         \
    } while (0)

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

long long pixels(const fse_cnn *c, int n) { return (long long)n * c->H * c->W; }

fse_status pack(fse_cnn *c, cudaStream_t s) {
    const int n = std::max(kWbTotal, kWtTotal);
    pack_weights_kernel<<<(n + 255) / 256, 256, 0, s>>>(c->params, c->wb, c->wt);
    CNN_CUDA(c, cudaGetLastError());
    return FSE_OK;
}

// forward over n areas already converted into c->xin
fse_status forward_from_xin(fse_cnn *c, int n, float *out, cudaStream_t s) {
    const long long P = pixels(c, n);
    const unsigned grid = (unsigned)((P + 127) / 128);
    conv_fwd_kernel<0><<<grid, 128, 0, s>>>(c->xin, c->wb, c->params, c->act[0], n, c->H, c->W);
    conv_fwd_kernel<1><<<grid, 128, 0, s>>>(c->act[0], c->wb, c->params, c->act[1], n, c->H, c->W);
    conv_fwd_kernel<2><<<grid, 128, 0, s>>>(c->act[1], c->wb, c->params, c->act[2], n, c->H, c->W);
    conv_fwd_kernel<3><<<grid, 128, 0, s>>>(c->act[2], c->wb, c->params, out, n, c->H, c->W);
    CNN_CUDA(c, cudaGetLastError());
    return FSE_OK;
}

fse_status check_batch(fse_cnn *c, const void *x, int n) {
    if (!c) return cfail(nullptr, FSE_ERR_INVALID_ARG, "cnn handle is NULL");
    if (n < 1 || n > c->max_batch) return cfail(c, FSE_ERR_INVALID_ARG, "batch %d not in [1, %d]", n, c->max_batch);
    if (!x) return cfail(c, FSE_ERR_INVALID_ARG, "input is NULL");
    return FSE_OK;
}

// loss and gradient of the mean weighted squared error; gradient in c->grad
fse_status loss_and_grad(fse_cnn *c, const float *x, const float *target, const float *lam, int n, cudaStream_t s) {
    const long long P = pixels(c, n);
    const int HW = c->H * c->W;
    input_kernel<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(x, reinterpret_cast<__nv_bfloat162 *>(c->xin), n, HW);
    fse_status st = forward_from_xin(c, n, c->y, s);
    if (st != FSE_OK) return st;
    const unsigned lgrid = (unsigned)((P + 255) / 256);
    out_grad_kernel<<<lgrid, 256, 0, s>>>(c->y, target, lam, c->gy, c->lpart, P, (float)(2.0 / (double)P));
    sum_loss_kernel<<<1, 32, 0, s>>>(c->lpart, (int)lgrid, c->loss, 1.0 / (double)P);
    const int nparts = (int)std::min<long long>(c->nparts_max, std::max<long long>(1, (P + HW - 1) / HW));
    const long long span = (P + nparts - 1) / nparts;
    const unsigned dgrid = (unsigned)((P + 127) / 128);
    // layer 4 (32 -> 1): weights, then data gradient gated by act[2]
    conv_bwd_weight_kernel<3><<<nparts, 256, 0, s>>>(c->gy, c->act[2], c->part, n, c->H, c->W, span);
    reduce_grad_kernel<3><<<(1 * 9 * 32 + 1 + 255) / 256, 256, 0, s>>>(c->part, nparts, c->grad);
    conv_bwd_data_kernel<3><<<dgrid, 128, 0, s>>>(c->gy, c->wt, c->act[2], c->g0, n, c->H, c->W);
    // layer 3
    conv_bwd_weight_kernel<2><<<nparts, 256, 0, s>>>(c->g0, c->act[1], c->part, n, c->H, c->W, span);
    reduce_grad_kernel<2><<<(32 * 9 * 32 + 32 + 255) / 256, 256, 0, s>>>(c->part, nparts, c->grad);
    conv_bwd_data_kernel<2><<<dgrid, 128, 0, s>>>(c->g0, c->wt, c->act[1], c->g1, n, c->H, c->W);
    // layer 2
    conv_bwd_weight_kernel<1><<<nparts, 256, 0, s>>>(c->g1, c->act[0], c->part, n, c->H, c->W, span);
    reduce_grad_kernel<1><<<(32 * 9 * 32 + 32 + 255) / 256, 256, 0, s>>>(c->part, nparts, c->grad);
    conv_bwd_data_kernel<1><<<dgrid, 128, 0, s>>>(c->g1, c->wt, c->act[0], c->g0, n, c->H, c->W);
    // layer 1 (2 -> 32): weights only
    conv_bwd_weight_kernel<0><<<nparts, 256, 0, s>>>(c->g0, c->xin, c->part, n, c->H, c->W, span);
    reduce_grad_kernel<0><<<(32 * 9 * 2 + 32 + 255) / 256, 256, 0, s>>>(c->part, nparts, c->grad);
    CNN_CUDA(c, cudaGetLastError());
    return FSE_OK;
}

}  // namespace

extern "C" {

fse_status fse_cnn_create(fse_cnn **out, int device, int height, int width, int max_batch) {
    if (!out) return cfail(nullptr, FSE_ERR_INVALID_ARG, "out is NULL");
    if (height < 1 || width < 1 || height > 256 || width > 256)
        return cfail(nullptr, FSE_ERR_INVALID_ARG, "area %d x %d not in [1, 256]^2", height, width);
    if (max_batch < 1 || (long long)max_batch * height * width > (1LL << 31))
        return cfail(nullptr, FSE_ERR_INVALID_ARG, "max_batch %d out of range", max_batch);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return cfail(nullptr, FSE_ERR_CUDA, "device %d not available", device);
    DevGuard guard(device);
    fse_cnn *c = new fse_cnn();
    c->device = device;
    c->H = height;
    c->W = width;
    c->max_batch = max_batch;
    const long long P = (long long)max_batch * height * width;
    c->nparts_max = (int)std::min<long long>(1024, std::max<long long>(1, max_batch));
    cudaError_t e = cudaSuccess;
    auto M = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = fse::dev_malloc(p, bytes);
    };
    M((void **)&c->params, kParams * sizeof(float));
    M((void **)&c->m, kParams * sizeof(float));
    M((void **)&c->v, kParams * sizeof(float));
    M((void **)&c->grad, kParams * sizeof(float));
    M((void **)&c->wb, kWbTotal * sizeof(__nv_bfloat16));
    M((void **)&c->wt, kWtTotal * sizeof(float));
    M((void **)&c->xin, P * 2 * sizeof(__nv_bfloat16));
    for (auto &a : c->act) M((void **)&a, P * 32 * sizeof(__nv_bfloat16));
    M((void **)&c->y, P * sizeof(float));
    M((void **)&c->gy, P * sizeof(float));
    M((void **)&c->g0, P * 32 * sizeof(float));
    M((void **)&c->g1, P * 32 * sizeof(float));
    M((void **)&c->part, (size_t)c->nparts_max * (32 * 9 * 32 + 32) * sizeof(float));
    M((void **)&c->lpart, (size_t)((P + 255) / 256) * sizeof(double));
    M((void **)&c->loss, sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(c->params, 0, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(c->m, 0, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(c->v, 0, kParams * sizeof(float));
    if (e != cudaSuccess) {
        g_cnn_err = std::string("allocation: ") + cudaGetErrorString(e);
        fse_cnn_destroy(c);
        return e == cudaErrorMemoryAllocation ? FSE_ERR_OOM : FSE_ERR_CUDA;
    }
    *out = c;
    return FSE_OK;
}

size_t fse_cnn_param_count(void) { return (size_t)kParams; }

fse_status fse_cnn_set_params(fse_cnn *c, const float *params, size_t n) {
    if (!c) return cfail(nullptr, FSE_ERR_INVALID_ARG, "cnn handle is NULL");
    if (!params || n != (size_t)kParams) return cfail(c, FSE_ERR_INVALID_ARG, "need %d parameters", kParams);
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(params[i])) return cfail(c, FSE_ERR_INVALID_ARG, "parameter %zu is not finite", i);
    DevGuard guard(c->device);
    CNN_CUDA(c, cudaMemcpy(c->params, params, n * sizeof(float), cudaMemcpyHostToDevice));
    CNN_CUDA(c, cudaMemset(c->m, 0, n * sizeof(float)));
    CNN_CUDA(c, cudaMemset(c->v, 0, n * sizeof(float)));
    c->step = 0;
    fse_status st = pack(c, nullptr);
    if (st != FSE_OK) return st;
    CNN_CUDA(c, cudaDeviceSynchronize());
    return FSE_OK;
}

fse_status fse_cnn_get_params(fse_cnn *c, float *params, size_t n) {
    if (!c) return cfail(nullptr, FSE_ERR_INVALID_ARG, "cnn handle is NULL");
    if (!params || n != (size_t)kParams) return cfail(c, FSE_ERR_INVALID_ARG, "need %d parameters", kParams);
    DevGuard guard(c->device);
    CNN_CUDA(c, cudaDeviceSynchronize());
    CNN_CUDA(c, cudaMemcpy(params, c->params, n * sizeof(float), cudaMemcpyDeviceToHost));
    return FSE_OK;
}

fse_status fse_cnn_get_state(fse_cnn *c, float *params, float *m, float *v, long long *step) {
    if (!c) return cfail(nullptr, FSE_ERR_INVALID_ARG, "cnn handle is NULL");
    if (!params || !m || !v || !step) return cfail(c, FSE_ERR_INVALID_ARG, "a state pointer is NULL");
    DevGuard guard(c->device);
    CNN_CUDA(c, cudaDeviceSynchronize());
    CNN_CUDA(c, cudaMemcpy(params, c->params, kParams * sizeof(float), cudaMemcpyDeviceToHost));
    CNN_CUDA(c, cudaMemcpy(m, c->m, kParams * sizeof(float), cudaMemcpyDeviceToHost));
    CNN_CUDA(c, cudaMemcpy(v, c->v, kParams * sizeof(float), cudaMemcpyDeviceToHost));
    *step = c->step;
    return FSE_OK;
}

fse_status fse_cnn_set_state(fse_cnn *c, const float *params, const float *m, const float *v, long long step) {
    if (!c) return cfail(nullptr, FSE_ERR_INVALID_ARG, "cnn handle is NULL");
    if (!params || !m || !v) return cfail(c, FSE_ERR_INVALID_ARG, "a state pointer is NULL");
    if (step < 0 || step > (1LL << 24)) return cfail(c, FSE_ERR_INVALID_ARG, "step %lld not in [0, 2^24]", step);
    for (int i = 0; i < kParams; ++i)
        if (!std::isfinite(params[i]) || !std::isfinite(m[i]) || !(v[i] >= 0.f) || !std::isfinite(v[i]))
            return cfail(c, FSE_ERR_INVALID_ARG, "state entry %d is not finite (or v < 0)", i);
    DevGuard guard(c->device);
    CNN_CUDA(c, cudaDeviceSynchronize());
    CNN_CUDA(c, cudaMemcpy(c->params, params, kParams * sizeof(float), cudaMemcpyHostToDevice));
    CNN_CUDA(c, cudaMemcpy(c->m, m, kParams * sizeof(float), cudaMemcpyHostToDevice));
    CNN_CUDA(c, cudaMemcpy(c->v, v, kParams * sizeof(float), cudaMemcpyHostToDevice));
    c->step = (int)step;
    fse_status st = pack(c, nullptr);
    if (st != FSE_OK) return st;
    CNN_CUDA(c, cudaDeviceSynchronize());
    return FSE_OK;
}

fse_status fse_cnn_forward(fse_cnn *c, const float *x, int n, float *y, void *stream) {
    fse_status st = check_batch(c, x, n);
    if (st != FSE_OK) return st;
    if (!y) return cfail(c, FSE_ERR_INVALID_ARG, "output is NULL");
    DevGuard guard(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long P = pixels(c, n);
    input_kernel<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(x, reinterpret_cast<__nv_bfloat162 *>(c->xin), n,
                                                             c->H * c->W);
    return forward_from_xin(c, n, y, s);
}

fse_status fse_cnn_loss_grad(fse_cnn *c, const float *x, const float *target, const float *lam, int n,
                             float *grad_host, float *loss_host, void *stream) {
    fse_status st = check_batch(c, x, n);
    if (st != FSE_OK) return st;
    if (!target) return cfail(c, FSE_ERR_INVALID_ARG, "target is NULL");
    DevGuard guard(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = loss_and_grad(c, x, target, lam, n, s);
    if (st != FSE_OK) return st;
    CNN_CUDA(c, cudaStreamSynchronize(s));
    if (grad_host) CNN_CUDA(c, cudaMemcpy(grad_host, c->grad, kParams * sizeof(float), cudaMemcpyDeviceToHost));
    if (loss_host) {
        double l = 0.0;
        CNN_CUDA(c, cudaMemcpy(&l, c->loss, sizeof(double), cudaMemcpyDeviceToHost));
        *loss_host = (float)l;
    }
    return FSE_OK;
}

fse_status fse_cnn_train_step(fse_cnn *c, const float *x, const float *target, const float *lam, int n, float lr,
                              float *loss_host, void *stream) {
    fse_status st = check_batch(c, x, n);
    if (st != FSE_OK) return st;
    if (!target) return cfail(c, FSE_ERR_INVALID_ARG, "target is NULL");
    if (!(lr > 0.f && lr < 1.f)) return cfail(c, FSE_ERR_INVALID_ARG, "learning rate %g not in (0, 1)", (double)lr);
    DevGuard guard(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = loss_and_grad(c, x, target, lam, n, s);
    if (st != FSE_OK) return st;
    c->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)c->step), c2 = 1.f - std::pow(b2, (float)c->step);
    adam_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(c->params, c->m, c->v, c->grad, kParams, lr, b1, b2, 1e-8f,
                                                       c1, c2);
    st = pack(c, s);
    if (st != FSE_OK) return st;
    if (loss_host) {
        double l = 0.0;
        CNN_CUDA(c, cudaMemcpyAsync(&l, c->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
        CNN_CUDA(c, cudaStreamSynchronize(s));
        *loss_host = (float)l;
    }
    return FSE_OK;
}

const char *fse_cnn_last_error(const fse_cnn *c) { return c ? c->err.c_str() : g_cnn_err.c_str(); }

void fse_cnn_destroy(fse_cnn *c) {
    if (!c) return;
    {
        DevGuard guard(c->device);
        cudaDeviceSynchronize();
        fse::dev_free(c->params);
        fse::dev_free(c->m);
        fse::dev_free(c->v);
        fse::dev_free(c->grad);
        fse::dev_free(c->wb);
        fse::dev_free(c->wt);
        fse::dev_free(c->xin);
        for (auto a : c->act) fse::dev_free(a);
        fse::dev_free(c->y);
        fse::dev_free(c->gy);
        fse::dev_free(c->g0);
        fse::dev_free(c->g1);
        fse::dev_free(c->part);
        fse::dev_free(c->lpart);
        fse::dev_free(c->loss);
    }
    delete c;
}

}  // extern "C"
