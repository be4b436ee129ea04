// fse_api.cu -- host runtime behind the C ABI of include/fse.h.
//
// Responsibilities: argument validation (nothing is enqueued for a rejected
// call), the uneven-batch planner (blocks bucketed by class, largest FFT
// first, grouped into work items of one F=64 / four F=32 / sixteen F=16
// blocks), the CUDA-graph cache (memset of the work-queue head + one
// persistent launch, re-captured only when the plan or a pointer changes),
// the grid-size autotuner, and the host-buffer entry point (a pipeline of
// chunked uploads, launches and read-backs on three streams).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "fse.h"
#include "fse_alloc.cuh"
#include "fse_cnn.cuh"
#include "fse_cnn_tc.cuh"
#include "fse_device.cuh"
#include "fse_kernels.cuh"
#include "fse_tables.cuh"

using fse::BlockRec;
using fse::DevParams;

namespace {

thread_local std::string g_create_error = "no error";

// chunks of the pipelined host-buffer path (upload / conceal / read back)
constexpr int kHostChunks = 8;

struct DeviceGuard {  // restores the caller's current device
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

uint64_t fnv1a(const void *data, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char *p = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

// 64-bit word hash for large arrays (multiply-xorshift per word).
uint64_t hash_words(const void *data, size_t n, uint64_t h) {
    const unsigned char *p = static_cast<const unsigned char *>(data);
    size_t i = 0;
    for (; i + 8 <= n; i += 8) {
        uint64_t w;
        std::memcpy(&w, p + i, 8);
        h ^= w + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
        h *= 0xff51afd7ed558ccdull;
        h ^= h >> 33;
    }
    return fnv1a(p + i, n - i, h);
}

}  // namespace

// Sets the text fse_last_error(NULL) returns (used by the handle-free entry
// point in fse_noalloc.cu).
void fse_internal_set_global_error(const char *msg) { g_create_error = msg; }

struct fse_handle {
    fse_config cfg{};
    int device = 0;
    int sm_count = 0;
    int cc = 0;                    // compute capability, major * 10 + minor
    int max_ctas[fse::kNumSets][2] = {};   // CTAs per SM of each kernel set (fse_device.cuh) x {128, 256} threads
    size_t smem_bytes = 0;
    cudaStream_t cap_stream = nullptr;
    float *d_wtab[FSE_MAX_CLASSES] = {};
    float2 *d_tw = nullptr;
    int *d_counter = nullptr;
    // block list
    BlockRec *d_blocks = nullptr;
    size_t blocks_cap = 0;
    BlockRec *h_blocks = nullptr;  // pinned staging
    size_t h_blocks_cap = 0;
    cudaEvent_t upload_done = nullptr;
    // trace
    int *d_tr_sel = nullptr;
    float *d_tr_energy = nullptr;
    float2 *d_tr_coef = nullptr;
    float *d_tr_second = nullptr;   // largest energy besides the pick, per selection
    size_t tr_cap = 0;
    int tr_stride = 0;
    int last_n_blocks = 0;
    cudaStream_t last_stream = nullptr;
    // plan / graph cache
    uint64_t plan_key = 0;
    bool graph_valid = false;
    cudaGraphExec_t gexec = nullptr;
    DevParams params{};
    int grid = 0;
    int nt = 128;                  // threads per CTA of the captured launch
    int ks = fse::kSetImage;       // kernel set of the captured launch
    // autotuner: chosen (threads per CTA, CTAs per SM) per class-mix signature
    std::vector<std::pair<uint64_t, std::pair<int, int>>> tuned;
    int tune_mode = FSE_TUNE_SYNC;
    // FSE_TUNE_ASYNC: candidates timed on the handle's real launches, one
    // per call, until each class mix has a choice
    struct TuneSession {
        uint64_t tune_key = 0, mix_sig = 0;
        int n = 0;
        int nt[4] = {}, cps[4] = {};
        cudaEvent_t e0[4] = {}, e1[4] = {};
        int state[4] = {};     // 0 not launched, 1 launched (events recorded), 2 timed
        float ms[4] = {};
    };
    std::vector<TuneSession> sessions;
    // host-buffer staging
    void *d_img = nullptr;
    size_t img_cap = 0;
    uint8_t *d_mask = nullptr;
    size_t mask_cap = 0;
    float *d_patch = nullptr;
    size_t patch_cap = 0;
    // learned initialisation (FSE_INIT_LEARNED)
    bool weights_loaded = false;
    float *d_cnn_params = nullptr;
    __nv_bfloat16 *d_cnn_wb = nullptr;
    float *d_cnn_wt = nullptr;
    int cnn_M = 0;                  // area edge shared by every class
    int cnn_chunk = 2048;           // areas per CNN pass inside the graph
    __nv_bfloat16 *d_cnn_x = nullptr, *d_cnn_a0 = nullptr, *d_cnn_a1 = nullptr;
    float *d_cnn_out = nullptr;
    float *d_est = nullptr;         // per-block estimates (sample units)
    size_t est_cap = 0;
    bool learned_launch = false;   // the captured graph runs the CNN first
    int learned_n = 0;
    uint8_t *d_tc_w = nullptr;      // tensor-core network: packed B operands
    bool tc_net = false;            // 16x16 blocks with a 16-sample border: tcgen05 kernel
    int *d_err = nullptr;           // device status word (fse::kErr* bits, read by fse_sync)
    unsigned long long wait_ns = 1000000000ull;   // limit of every bounded device wait
    // ordered concealment (FSE_FLAG_ORDERED): neighbour lists and done flags
    int *d_nb_start = nullptr, *d_nb_list = nullptr, *d_done = nullptr;
    size_t nb_start_cap = 0, nb_list_cap = 0, done_cap = 0;
    int ordered_n = 0;
    bool ext = false;               // video volumes or ordered concealment: the EXT kernel
    // pipelined host-buffer path: upload and read-back streams, per-chunk
    // events, the chunks' sorted block lists and work-queue heads
    bool pipe_ready = false;
    cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_out = nullptr;
    cudaEvent_t ev_in[kHostChunks] = {}, ev_k[kHostChunks] = {};
    BlockRec *d_cblocks = nullptr;
    size_t cblocks_cap = 0;
    BlockRec *h_cblocks = nullptr;  // pinned staging
    size_t h_cblocks_cap = 0;
    int *d_ccounter = nullptr;
    std::vector<fse_block> hb_stage;   // host copy of a device-resident block list
    std::string err = "no error";
};

namespace {

fse_status fail(fse_handle *h, fse_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_create_error = buf;
    return st;
}

fse_status cuda_fail(fse_handle *h, cudaError_t e, const char *what) {
    const fse_status st = (e == cudaErrorMemoryAllocation) ? FSE_ERR_OOM : FSE_ERR_CUDA;
    return fail(h, st, "%s: %s", what, cudaGetErrorString(e));
}

#define FSE_CUDA(h, call)                                           \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);    \
    } while (0)

fse_status validate_config(const fse_config *cfg) {
    if (!cfg) return fail(nullptr, FSE_ERR_INVALID_ARG, "config is NULL");
    if (cfg->n_classes < 1 || cfg->n_classes > FSE_MAX_CLASSES)
        return fail(nullptr, FSE_ERR_INVALID_ARG, "n_classes %d not in [1, %d]", cfg->n_classes,
                    FSE_MAX_CLASSES);
    for (int i = 0; i < cfg->n_classes; ++i) {
        const fse_class &c = cfg->cls[i];
        if (c.fft != 16 && c.fft != 32 && c.fft != 64) {
            if (c.fft > 0 && (c.fft & (c.fft - 1)) == 0)
                return fail(nullptr, FSE_ERR_UNSUPPORTED, "class %d: fft %d not supported (16, 32, 64)", i, c.fft);
            return fail(nullptr, FSE_ERR_INVALID_ARG, "class %d: fft %d is not a power of two", i, c.fft);
        }
        if (c.block < 1 || 2 * c.block > c.fft)
            return fail(nullptr, FSE_ERR_INVALID_ARG, "class %d: block %d not in [1, fft/2]", i, c.block);
        if (c.border < 1 || c.block + 2 * c.border > c.fft)
            return fail(nullptr, FSE_ERR_INVALID_ARG, "class %d: border %d needs 1 <= d and b + 2d <= fft", i,
                        c.border);
        if (!(c.rho > 0.f && c.rho <= 1.f))
            return fail(nullptr, FSE_ERR_INVALID_ARG, "class %d: rho %g not in (0, 1]", i, (double)c.rho);
        if (!(c.gamma > 0.f && c.gamma < 2.f))
            return fail(nullptr, FSE_ERR_INVALID_ARG, "class %d: gamma %g not in (0, 2)", i, (double)c.gamma);
        if (c.iters < 0 || c.iters > 4096)
            return fail(nullptr, FSE_ERR_INVALID_ARG, "class %d: iters %d not in [0, 4096]", i, c.iters);
        if (c.frames < 0 || c.frames == 2 || c.frames > 3)
            return fail(nullptr, c.frames > 3 ? FSE_ERR_UNSUPPORTED : FSE_ERR_INVALID_ARG,
                        "class %d: frames %d (0 or 1: images, 3: video volumes)", i, c.frames);
        if (c.frames == 3 && c.fft == 64)
            return fail(nullptr, FSE_ERR_UNSUPPORTED, "class %d: video volumes need fft 16 or 32", i);
    }
    if (cfg->init != FSE_INIT_ZERO && cfg->init != FSE_INIT_LEARNED)
        return fail(nullptr, FSE_ERR_INVALID_ARG, "init mode %d unknown", cfg->init);
    if (cfg->init == FSE_INIT_LEARNED) {
        if (cfg->n_classes != 1)
            return fail(nullptr, FSE_ERR_UNSUPPORTED, "learned initialisation supports one block class per handle");
        if (cfg->cls[0].frames > 1)
            return fail(nullptr, FSE_ERR_UNSUPPORTED, "learned initialisation is for image areas");
        if (cfg->init_iters < 0 || cfg->init_iters > 4096)
            return fail(nullptr, FSE_ERR_INVALID_ARG, "init_iters %d not in [0, 4096]", cfg->init_iters);
    }
    if (cfg->flags & ~(FSE_FLAG_TRACE | FSE_FLAG_ORDERED | FSE_FLAG_CLAMP_U8 | FSE_FLAG_FIXED_W))
        return fail(nullptr, FSE_ERR_INVALID_ARG, "unknown flag bits 0x%x", cfg->flags);
    if (cfg->flags & FSE_FLAG_FIXED_W) {
        // the 16-bit spectrum lives in the FFT-64 chunk layout
        for (int c = 0; c < cfg->n_classes; ++c)
            if (cfg->cls[c].fft != 64 || cfg->cls[c].frames > 1)
                return fail(nullptr, FSE_ERR_UNSUPPORTED,
                            "reduced-precision residual storage: image classes of fft 64 only");
        if (cfg->flags & FSE_FLAG_ORDERED)
            return fail(nullptr, FSE_ERR_UNSUPPORTED, "reduced-precision residual storage with ordered concealment");
    }
    if (cfg->flags & FSE_FLAG_ORDERED) {
        // fft 16 is excluded: its blocks share warps, and a lane waiting for an
        // earlier block of its own warp would stall that warp's synchronisation
        if (cfg->n_classes != 1 || cfg->init != FSE_INIT_ZERO || cfg->cls[0].frames > 1 || cfg->cls[0].fft < 32)
            return fail(nullptr, FSE_ERR_UNSUPPORTED,
                        "ordered concealment: one image class of fft 32 or 64 with the zero initialisation");
        if (!(cfg->reuse_weight > 0.f && cfg->reuse_weight <= 1.f))
            return fail(nullptr, FSE_ERR_INVALID_ARG, "reuse_weight %g not in (0, 1]", (double)cfg->reuse_weight);
    }
    return FSE_OK;
}

// The sorted plan of one batch call.
struct Plan {
    std::vector<BlockRec> sorted;
    int n_seg = 0;
    int seg_cls[FSE_MAX_CLASSES] = {};
    int seg_item_end[FSE_MAX_CLASSES] = {};
    int seg_block_start[FSE_MAX_CLASSES] = {};
    int seg_block_count[FSE_MAX_CLASSES] = {};
    int total_items = 0;
    long long patch_total = 0;
    uint64_t mix_sig = 0;      // class mix of the batch (per handle: class indices)
    uint64_t tune_key = 0;     // the same by class parameters, for the process-wide tuning cache
    int ks = fse::kSetImage;   // kernel set that covers the batch's classes
};

// Argument checks of one batch call (geometry, every block's class and
// position); *patch_total = sum of b^2 over the blocks.
fse_status validate_batch(fse_handle *h, const void *images, int dtype, int n_images, int height, int width,
                          size_t pitch, const uint8_t *mask, const fse_block *blocks, int n_blocks,
                          long long *patch_total) {
    *patch_total = 0;
    if (n_blocks < 0) return fail(h, FSE_ERR_INVALID_ARG, "n_blocks %d < 0", n_blocks);
    if (dtype != FSE_DTYPE_U8 && dtype != FSE_DTYPE_F32) return fail(h, FSE_ERR_INVALID_ARG, "dtype %d unknown", dtype);
    if (n_blocks == 0) return FSE_OK;
    if (!images || !mask || !blocks) return fail(h, FSE_ERR_INVALID_ARG, "images, loss_mask and blocks must be non-NULL");
    if (n_images < 1 || height < 1 || width < 1)
        return fail(h, FSE_ERR_INVALID_ARG, "bad geometry %d x %d x %d", n_images, height, width);
    const size_t es = dtype == FSE_DTYPE_U8 ? 1 : 4;
    if (pitch < (size_t)width * es) return fail(h, FSE_ERR_INVALID_ARG, "pitch %zu < width * %zu", pitch, es);
    if (dtype == FSE_DTYPE_F32 && (pitch % 4 != 0 || (reinterpret_cast<uintptr_t>(images) & 3)))
        return fail(h, FSE_ERR_INVALID_ARG, "FP32 images need 4-byte aligned base and pitch");
    const fse_config &cfg = h->cfg;
    long long acc = 0;
    for (int i = 0; i < n_blocks; ++i) {
        const fse_block &bk = blocks[i];
        if (bk.cls < 0 || bk.cls >= cfg.n_classes)
            return fail(h, FSE_ERR_INVALID_ARG, "block %d: class %d not in [0, %d)", i, bk.cls, cfg.n_classes);
        const int b = cfg.cls[bk.cls].block;
        if (bk.image < 0 || bk.image >= n_images || bk.x < 0 || bk.y < 0 || bk.x + b > width || bk.y + b > height)
            return fail(h, FSE_ERR_INVALID_ARG, "block %d (image %d, x %d, y %d, b %d) is not inside the image", i,
                        bk.image, bk.x, bk.y, b);
        acc += (long long)b * b;
    }
    *patch_total = acc;
    return FSE_OK;
}

// Validation and plan of one batch call: blocks bucketed by class (largest F
// first), work items per class, patch offsets in the caller's order.
fse_status validate_and_plan(fse_handle *h, const void *images, int dtype, int n_images, int height, int width,
                             size_t pitch, const uint8_t *mask, const fse_block *blocks, int n_blocks, Plan &pl) {
    fse_status st = validate_batch(h, images, dtype, n_images, height, width, pitch, mask, blocks, n_blocks,
                                   &pl.patch_total);
    if (st != FSE_OK || n_blocks == 0) return st;
    const fse_config &cfg = h->cfg;
    // class order of the queue: largest F first, then class index
    int order[FSE_MAX_CLASSES];
    for (int i = 0; i < cfg.n_classes; ++i) order[i] = i;
    std::stable_sort(order, order + cfg.n_classes,
                     [&](int a, int b) { return cfg.cls[a].fft > cfg.cls[b].fft; });
    std::vector<int> cnt(cfg.n_classes, 0);
    for (int i = 0; i < n_blocks; ++i) cnt[blocks[i].cls]++;
    std::vector<long long> poff(n_blocks);
    long long acc = 0;
    for (int i = 0; i < n_blocks; ++i) {
        poff[i] = acc;
        const int b = cfg.cls[blocks[i].cls].block;
        acc += (long long)b * b;
    }
    std::vector<int> start(cfg.n_classes, 0);
    int pos = 0, items = 0;
    pl.n_seg = 0;
    for (int oi = 0; oi < cfg.n_classes; ++oi) {
        const int c = order[oi];
        start[c] = pos;
        if (cnt[c] == 0) continue;
        const int F = cfg.cls[c].fft;
        const int bpi = 4096 / (F * F * (cfg.cls[c].frames > 1 ? 4 : 1));
        items += (cnt[c] + bpi - 1) / bpi;
        pl.seg_cls[pl.n_seg] = c;
        pl.seg_item_end[pl.n_seg] = items;
        pl.seg_block_start[pl.n_seg] = pos;
        pl.seg_block_count[pl.n_seg] = cnt[c];
        pl.n_seg++;
        pos += cnt[c];
    }
    pl.total_items = items;
    pl.sorted.resize(n_blocks);
    std::vector<int> fillp(start);
    for (int i = 0; i < n_blocks; ++i) {
        const fse_block &bk = blocks[i];
        BlockRec r;
        r.image = bk.image;
        r.x = bk.x;
        r.y = bk.y;
        r.orig = i;
        r.patch_off = poff[i];
        r.pad = 0;
        pl.sorted[fillp[bk.cls]++] = r;
    }
    uint64_t sig = 1469598103934665603ull, tkey = 1469598103934665603ull;
    for (int s = 0; s < pl.n_seg; ++s) {
        const int c = pl.seg_cls[s];
        const int bucket = 32 - __builtin_clz((unsigned)pl.seg_block_count[s]);  // log2 size bucket
        const int key[3] = {c, bucket, cfg.cls[c].iters};
        sig = fnv1a(key, sizeof key, sig);
        const fse_class &k = cfg.cls[c];
        const int tk[6] = {k.fft, k.block, k.border, k.frames, k.iters, bucket};
        tkey = fnv1a(tk, sizeof tk, tkey);
    }
    pl.mix_sig = sig;
    bool all_f64 = true;
    for (int sg = 0; sg < pl.n_seg; ++sg) {
        const fse_class &k = cfg.cls[pl.seg_cls[sg]];
        all_f64 = all_f64 && k.fft == 64 && k.frames <= 1;
    }
    pl.ks = fse::kernel_set_for(h->ext, all_f64, (cfg.flags & FSE_FLAG_TRACE) != 0,
                                (cfg.flags & FSE_FLAG_FIXED_W) != 0);
    const long long dev_key[5] = {pl.ks, h->sm_count, h->cc, (long long)h->smem_bytes,
                                  (long long)(cfg.flags & FSE_FLAG_ORDERED)};
    pl.tune_key = fnv1a(dev_key, sizeof dev_key, tkey);
    return FSE_OK;
}

// Per-class constants of a launch (learned: the iterations after the network).
void set_classes(const fse_handle *h, DevParams &P, bool learned) {
    for (int c = 0; c < h->cfg.n_classes; ++c) {
        const fse_class &k = h->cfg.cls[c];
        fse::DevClass &D = P.cls[c];
        D.F = k.fft;
        D.b = k.block;
        D.d = k.border;
        D.M = k.block + 2 * k.border;
        D.off = (k.fft - D.M) / 2;
        D.iters = (learned && h->cfg.init_iters > 0) ? h->cfg.init_iters : k.iters;
        D.FT = k.frames > 1 ? 4 : 1;
        D.T = k.frames > 1 ? k.frames : 1;
        D.tc = (D.T - 1) / 2;
        D.toff = (D.FT - D.T) / 2;
        D.bpi = 4096 / (k.fft * k.fft * D.FT);
        D.gamma = k.gamma;
        D.wtab = h->d_wtab[c];
    }
}

// cuTensorMapEncodeTiled from the driver, through the runtime (no link
// against the driver library); nullptr when unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// TMA gather of the F = 64 windows (fse_device.cuh): tensor maps over the
// 8-bit images and the mask as [n_images * height rows, width columns], box
// (roundup16(M) + 16) columns x M rows.  Used when the batch runs the FFT-64
// kernel set and the buffers meet the tensor-map rules (16-byte aligned
// bases, row pitches multiples of 16 bytes); otherwise P.tma stays 0 and the
// kernel reads the windows with plain loads.
void setup_tma(const fse_handle *h, DevParams &P, int ks, int dtype, const void *images, const uint8_t *mask,
               int n_images, int height, int width, size_t pitch) {
    P.tma = 0;
    if ((ks != fse::kSetF64 && ks != fse::kSetFixW) || dtype != FSE_DTYPE_U8) return;
    if ((reinterpret_cast<uintptr_t>(images) & 15) || (reinterpret_cast<uintptr_t>(mask) & 15) || (pitch & 15) ||
        (width & 15) || (long long)n_images * height >= (1LL << 31))
        return;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return;
    int maxM = 0;
    for (int c = 0; c < h->cfg.n_classes; ++c)
        if (h->cfg.cls[c].fft == 64) maxM = std::max(maxM, h->cfg.cls[c].block + 2 * h->cfg.cls[c].border);
    const int bw = ((maxM + 15) & ~15) + 16, bh = maxM;
    if (2 * (((bw * bh) + 127) & ~127) > fse::kTmaStageMax) return;
    const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)n_images * height};
    const cuuint64_t istride[1] = {(cuuint64_t)pitch}, mstride[1] = {(cuuint64_t)width};
    const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh}, es[2] = {1, 1};
    if (enc(&P.tm_img, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(images), dims, istride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        enc(&P.tm_mask, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(mask), dims, mstride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return;
    P.tma = 1;
    P.tma_bw = bw;
    P.tma_bh = bh;
}

// The persistent concealment kernel of a handle: kernel set ks, 128 or 256
// threads per CTA.
cudaError_t launch_fse(const fse_handle *h, int ks, int nt, int grid, const DevParams &P, cudaStream_t s) {
    return fse::batch_kernel_launch(ks, nt, grid, h->smem_bytes, s, P);
}

int ctas_per_sm(const fse_handle *h, int ks, int nt) { return h->max_ctas[ks][nt == 256 ? 1 : 0]; }

template <typename T>
fse_status grow(fse_handle *h, T **ptr, size_t *cap, size_t need) {
    if (need <= *cap) return FSE_OK;
    const size_t n = std::max(need, *cap + *cap / 2);
    if (*ptr) fse::dev_free(*ptr);
    *ptr = nullptr;
    *cap = 0;
    cudaError_t e = fse::dev_malloc(reinterpret_cast<void **>(ptr), n * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc");
    *cap = n;
    return FSE_OK;
}

// CNN input of the blocks at sorted positions first .. first+count-1: per area
// sample (M x M, row-major) the pair (support sample / 255, support
// indicator); support = inside the image, not lost, not in the block's own B
// (the same test as the concealment kernel's gather).
__global__ void cnn_gather_kernel(const DevParams P, int first, int count, int M, int d, int b,
                                  __nv_bfloat162 *__restrict__ xin) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long MM = (long long)M * M;
    if (i >= count * MM) return;
    const int q = (int)(i / MM), r = (int)(i % MM), am = r / M, an = r % M;
    const BlockRec blk = P.blocks[first + q];
    const int yy = blk.y - d + am, xx = blk.x - d + an;
    const bool inB = am >= d && am < d + b && an >= d && an < d + b;
    float sv = 0.f, a = 0.f;
    if (!inB && yy >= 0 && yy < P.H && xx >= 0 && xx < P.W &&
        P.mask[((size_t)blk.image * P.H + yy) * P.W + xx] == 0) {
        const char *row = static_cast<const char *>(P.images) + ((long long)blk.image * P.H + yy) * P.pitch;
        sv = (P.dtype == 0 ? (float)reinterpret_cast<const uint8_t *>(row)[xx] : reinterpret_cast<const float *>(row)[xx]) *
             (1.f / 255.f);
        a = 1.f;
    }
    xin[i] = __floats2bfloat162_rn(sv, a);
}

// network output (estimate / 255) of those blocks -> per-block estimates in
// sample units, at the caller's block order.  The estimate is kept on B and
// zero on the rest of the area: the iterations then run on the unchanged
// support and the network supplies what they do not reach (the network is
// trained for exactly that; see train_init.py).
__global__ void est_scatter_kernel(const float *__restrict__ out, const BlockRec *__restrict__ blocks, int first,
                                   int count, int M, int d, int b, float *__restrict__ est, long long stride) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int MM = M * M;
    if (i >= (long long)count * MM) return;
    const int q = (int)(i / MM), r = (int)(i % MM), am = r / M, an = r % M;
    const bool inB = am >= d && am < d + b && an >= d && an < d + b;
    est[blocks[first + q].orig * stride + r] = inB ? 255.f * out[i] : 0.f;
}

// Model over the whole extrapolation area from the trace of the last launch:
// Re{g}[m, n] = Re{sum_i c_i exp(j 2 pi (u_i m + v_i n) / F)} at the area's
// grid positions (the IFFT of the accumulated model spectrum, Algorithm 1),
// evaluated with the same operation sequence and twiddle table as the
// kernel's own evaluation on B, so the B samples agree bit for bit.  One CTA
// per block (sorted order), 256 threads, up to 9 samples each (M <= 48).
__global__ void __launch_bounds__(256) area_model_kernel(const DevParams P, float *__restrict__ model,
                                                         long long mstride) {
    __shared__ float2 s_tw[64];
    if (threadIdx.x < 64) s_tw[threadIdx.x] = P.tw[threadIdx.x];
    __syncthreads();
    const int q = blockIdx.x;
    int sg = 0;
    while (sg + 1 < P.n_seg && q >= P.seg_block_start[sg] + P.seg_block_count[sg]) ++sg;
    const fse::DevClass &C = P.cls[P.seg_cls[sg]];
    const BlockRec blk = P.blocks[q];
    const int F = C.F, M = C.M, MM = M * M, step = 64 / F;
    constexpr int kPer = 9;
    float acc[kPer];
    int pm[kPer], pn[kPer];
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
        const int p = threadIdx.x + t * 256;
        acc[t] = 0.f;
        pm[t] = C.off + p / M;
        pn[t] = C.off + p % M;
    }
    const size_t o = (size_t)blk.orig * P.tr_stride;
    for (int i = 0; i < C.iters; ++i) {
        const int sel = P.tr_sel[o + i];
        const float2 c = P.tr_coef[o + i];
        const int u = sel / F, v = sel % F;
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
            const float2 tw = s_tw[((u * pm[t] + v * pn[t]) & (F - 1)) * step];
            acc[t] = fmaf(c.x, tw.x, fmaf(-c.y, tw.y, acc[t]));
        }
    }
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
        const int p = threadIdx.x + t * 256;
        if (p < MM) model[blk.orig * mstride + p] = acc[t];
    }
}

fse_status capture_graph(fse_handle *h, int ks, int nt, int grid, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    FSE_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    if (h->learned_launch && h->tc_net) {
        // learned initialisation on the tensor cores: the network's output on
        // B straight into h->d_est (zero elsewhere), one persistent launch
        const unsigned g = (unsigned)std::min(h->learned_n, h->sm_count);
        fse_tc::cnn_tc_kernel<DevParams, BlockRec><<<g, fse_tc::kThreads, fse_tc::kSmemBytes, h->cap_stream>>>(
            h->params, h->d_tc_w, h->d_cnn_params, h->d_est, (long long)h->cnn_M * h->cnn_M, h->learned_n,
            h->d_err);
    } else if (h->learned_launch) {
        // learned initialisation: CNN over all blocks in chunks, estimates
        // scattered to h->d_est, then the concealment from the residual
        const int M = h->cnn_M, MM = M * M;
        const fse::DevClass &C = h->params.cls[0];
        for (int first = 0; first < h->learned_n; first += h->cnn_chunk) {
            const int cnt = std::min(h->cnn_chunk, h->learned_n - first);
            const long long np = (long long)cnt * MM;
            cnn_gather_kernel<<<(unsigned)((np + 255) / 256), 256, 0, h->cap_stream>>>(
                h->params, first, cnt, M, C.d, C.b, reinterpret_cast<__nv_bfloat162 *>(h->d_cnn_x));
            const unsigned cg = (unsigned)((np + 127) / 128);
            fse_net::conv_fwd_kernel<0><<<cg, 128, 0, h->cap_stream>>>(h->d_cnn_x, h->d_cnn_wb, h->d_cnn_params,
                                                                       h->d_cnn_a0, cnt, M, M);
            fse_net::conv_fwd_kernel<1><<<cg, 128, 0, h->cap_stream>>>(h->d_cnn_a0, h->d_cnn_wb, h->d_cnn_params,
                                                                       h->d_cnn_a1, cnt, M, M);
            fse_net::conv_fwd_kernel<2><<<cg, 128, 0, h->cap_stream>>>(h->d_cnn_a1, h->d_cnn_wb, h->d_cnn_params,
                                                                       h->d_cnn_a0, cnt, M, M);
            fse_net::conv_fwd_kernel<3><<<cg, 128, 0, h->cap_stream>>>(h->d_cnn_a0, h->d_cnn_wb, h->d_cnn_params,
                                                                       h->d_cnn_out, cnt, M, M);
            est_scatter_kernel<<<(unsigned)((np + 255) / 256), 256, 0, h->cap_stream>>>(
                h->d_cnn_out, h->d_blocks, first, cnt, M, C.d, C.b, h->d_est, (long long)MM);
        }
    }
    if (h->params.ordered) cudaMemsetAsync(h->d_done, 0, (size_t)h->ordered_n * sizeof(int), h->cap_stream);
    cudaMemsetAsync(h->params.counter, 0, sizeof(int), h->cap_stream);
    cudaError_t le = launch_fse(h, ks, nt, grid, h->params, h->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(h, le, "fse_batch_kernel launch (capture)");
    }
    if (ce != cudaSuccess) return cuda_fail(h, ce, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return cuda_fail(h, ie, "cudaGraphInstantiate");
    return FSE_OK;
}

// Choices of the autotuner shared by every handle of the process: the same
// class mix (by class parameters and batch-size bucket) on the same kind of
// device with the same kernel set is not timed again by a new handle.
std::mutex g_tune_mu;
std::unordered_map<uint64_t, std::pair<int, int>> g_tuned;

// A launch the asynchronous autotuner times: the caller records e0 / e1 of
// session `s` around it (s < 0: no timing).
struct TuneTicket {
    int s = -1, i = -1;
};

void destroy_session(fse_handle::TuneSession &ss) {
    for (int i = 0; i < 4; ++i) {
        if (ss.e0[i]) cudaEventDestroy(ss.e0[i]);
        if (ss.e1[i]) cudaEventDestroy(ss.e1[i]);
        ss.e0[i] = ss.e1[i] = nullptr;
    }
}

void remember_choice(fse_handle *h, const Plan &pl, int nt, int cps, bool global) {
    // a choice closes any asynchronous session of the mix (one left open when
    // the mode changed): its launches no longer decide anything, and an open
    // session keeps the mix from replaying its captured graph
    for (size_t k = 0; k < h->sessions.size();)
        if (h->sessions[k].tune_key == pl.tune_key && h->sessions[k].mix_sig == pl.mix_sig) {
            destroy_session(h->sessions[k]);
            h->sessions.erase(h->sessions.begin() + k);
        } else {
            ++k;
        }
    h->tuned.emplace_back(pl.mix_sig, std::make_pair(nt, cps));
    if (global) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[pl.tune_key] = std::make_pair(nt, cps);
    }
}

// FSE_TUNE_ASYNC: poll the session's timed launches without waiting; once
// every candidate is timed, keep the fastest.  Otherwise hand out the next
// untimed candidate with a ticket, or (all launched, some still running)
// the fastest timed so far, else the first candidate.
fse_status autotune_async(fse_handle *h, const Plan &pl, int *best_nt, int *best_cps, TuneTicket *t) {
    int si = -1;
    for (int k = 0; k < (int)h->sessions.size(); ++k)
        if (h->sessions[k].tune_key == pl.tune_key && h->sessions[k].mix_sig == pl.mix_sig) si = k;
    if (si < 0) {
        fse_handle::TuneSession ss;
        ss.tune_key = pl.tune_key;
        ss.mix_sig = pl.mix_sig;
        for (int nt : {128, 256}) {
            const int maxc = ctas_per_sm(h, pl.ks, nt);
            for (int cps = std::max(1, maxc - 1); cps <= maxc && ss.n < 4; ++cps) {
                ss.nt[ss.n] = nt;
                ss.cps[ss.n] = cps;
                ++ss.n;
            }
        }
        h->sessions.push_back(ss);
        si = (int)h->sessions.size() - 1;
    }
    fse_handle::TuneSession &ss = h->sessions[si];
    int timed = 0, best = -1;
    for (int i = 0; i < ss.n; ++i) {
        if (ss.state[i] == 1) {
            const cudaError_t q = cudaEventQuery(ss.e1[i]);
            if (q == cudaSuccess) {
                FSE_CUDA(h, cudaEventElapsedTime(&ss.ms[i], ss.e0[i], ss.e1[i]));
                ss.state[i] = 2;
            } else if (q != cudaErrorNotReady) {
                return cuda_fail(h, q, "autotune event");
            }
        }
        if (ss.state[i] == 2) {
            ++timed;
            if (best < 0 || ss.ms[i] < ss.ms[best]) best = i;
        }
    }
    if (timed == ss.n) {
        *best_nt = ss.nt[best];
        *best_cps = ss.cps[best];
        remember_choice(h, pl, *best_nt, *best_cps, true);   // closes the session
        return FSE_OK;
    }
    for (int i = 0; i < ss.n; ++i)
        if (ss.state[i] == 0) {
            if (!ss.e0[i]) FSE_CUDA(h, cudaEventCreate(&ss.e0[i]));
            if (!ss.e1[i]) FSE_CUDA(h, cudaEventCreate(&ss.e1[i]));
            *best_nt = ss.nt[i];
            *best_cps = ss.cps[i];
            t->s = si;
            t->i = i;
            return FSE_OK;
        }
    const int c = best >= 0 ? best : 0;
    *best_nt = ss.nt[c];
    *best_cps = ss.cps[c];
    return FSE_OK;
}

// Records the ticket's start event (before the timed launch) or end event.
fse_status tune_mark(fse_handle *h, const TuneTicket &t, cudaStream_t stream, bool end) {
    if (t.s < 0) return FSE_OK;
    fse_handle::TuneSession &ss = h->sessions[t.s];
    FSE_CUDA(h, cudaEventRecord(end ? ss.e1[t.i] : ss.e0[t.i], stream));
    if (end) ss.state[t.i] = 1;
    return FSE_OK;
}

// Autotuner: time each candidate mapping -- 128 threads per CTA (32 bins per
// thread) or 256 (16 bins per thread), the two largest CTA counts per SM --
// on the actual batch (the outputs are identical for every candidate, so the
// runs are harmless) and keep the fastest per class mix, in the handle and
// in the process-wide cache.  FSE_TUNE_SYNC: the first call with a new class
// mix waits for its timing runs.  FSE_TUNE_ASYNC: no call waits; each call
// times one candidate on its own launch (ticket *t) until all are timed.
// FSE_TUNE_OFF: 128 threads per CTA at the largest CTA count (the measured
// choice for the FFT-64 classes), untimed.  Later calls (and, for measured
// choices, other handles) reuse the choice.
fse_status autotune(fse_handle *h, const Plan &pl, cudaStream_t stream, int *best_nt, int *best_cps,
                    TuneTicket *t = nullptr) {
    for (auto &kv : h->tuned)
        if (kv.first == pl.mix_sig) {
            *best_nt = kv.second.first;
            *best_cps = kv.second.second;
            return FSE_OK;
        }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(pl.tune_key);
        if (it != g_tuned.end()) {
            *best_nt = it->second.first;
            *best_cps = it->second.second;
        } else {
            *best_nt = 0;
        }
    }
    if (*best_nt > 0) {   // measured by another handle (or an earlier one)
        remember_choice(h, pl, *best_nt, *best_cps, false);
        return FSE_OK;
    }
    int bnt = 256, bcps = ctas_per_sm(h, pl.ks, 256);
    if (h->tune_mode == FSE_TUNE_OFF) {
        *best_nt = 128;
        *best_cps = ctas_per_sm(h, pl.ks, 128);
        remember_choice(h, pl, *best_nt, *best_cps, false);
        return FSE_OK;
    }
    if (h->tune_mode == FSE_TUNE_ASYNC && t && (long long)pl.total_items >= 2LL * h->sm_count)
        return autotune_async(h, pl, best_nt, best_cps, t);
    // small batches cannot fill the machine: no measurement needed
    if ((long long)pl.total_items >= 2LL * h->sm_count) {
        cudaEvent_t e0, e1;
        FSE_CUDA(h, cudaEventCreate(&e0));
        FSE_CUDA(h, cudaEventCreate(&e1));
        float best_ms = 1e30f;
        for (int nt : {128, 256}) {
            const int maxc = ctas_per_sm(h, pl.ks, nt);
            for (int cps = std::max(1, maxc - 1); cps <= maxc; ++cps) {
                const int grid = std::min(pl.total_items, cps * h->sm_count);
                cudaGraphExec_t ex = nullptr;
                fse_status st = capture_graph(h, pl.ks, nt, grid, &ex);
                if (st != FSE_OK) return st;
                cudaGraphLaunch(ex, stream);  // warm-up
                cudaEventRecord(e0, stream);
                cudaGraphLaunch(ex, stream);
                cudaEventRecord(e1, stream);
                cudaError_t se = cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                cudaGraphExecDestroy(ex);
                if (se != cudaSuccess) return cuda_fail(h, se, "autotune run");
                if (ms < best_ms) {
                    best_ms = ms;
                    bnt = nt;
                    bcps = cps;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    remember_choice(h, pl, bnt, bcps, true);
    *best_nt = bnt;
    *best_cps = bcps;
    return FSE_OK;
}

// Ordered concealment: for every block j (caller order), the earlier blocks
// i < j of the same image whose b x b block meets j's area
// [x - d, x + b + d) x [y - d, y + b + d): CSR lists, found through a grid of
// b x b cells.
void ordered_neighbours(const fse_block *blocks, int n, int b, int d, std::vector<int> &start,
                        std::vector<int> &list) {
    auto cell = [](int im, int cy, int cx) {
        return ((uint64_t)(uint32_t)im << 42) ^ ((uint64_t)(uint32_t)(cy + (1 << 20)) << 21) ^
               (uint64_t)(uint32_t)(cx + (1 << 20));
    };
    auto fdiv = [](int a, int q) { return a >= 0 ? a / q : -((-a + q - 1) / q); };
    std::unordered_map<uint64_t, std::vector<int>> grid;
    grid.reserve((size_t)n * 2);
    start.assign(n + 1, 0);
    list.clear();
    for (int j = 0; j < n; ++j) {
        const fse_block &bj = blocks[j];
        const int ax0 = bj.x - d, ax1 = bj.x + b + d, ay0 = bj.y - d, ay1 = bj.y + b + d;
        std::vector<int> cand;
        for (int cy = fdiv(ay0, b); cy <= fdiv(ay1 - 1, b); ++cy)
            for (int cx = fdiv(ax0, b); cx <= fdiv(ax1 - 1, b); ++cx) {
                auto it = grid.find(cell(bj.image, cy, cx));
                if (it == grid.end()) continue;
                for (int i : it->second) {
                    const fse_block &bi = blocks[i];
                    if (bi.x < ax1 && bi.x + b > ax0 && bi.y < ay1 && bi.y + b > ay0) cand.push_back(i);
                }
            }
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        list.insert(list.end(), cand.begin(), cand.end());
        start[j + 1] = (int)list.size();
        for (int cy = fdiv(bj.y, b); cy <= fdiv(bj.y + b - 1, b); ++cy)
            for (int cx = fdiv(bj.x, b); cx <= fdiv(bj.x + b - 1, b); ++cx) grid[cell(bj.image, cy, cx)].push_back(j);
    }
}

fse_status run_batch(fse_handle *h, const void *images, int dtype, int n_images, int height, int width,
                     size_t pitch, const uint8_t *mask, const fse_block *blocks, int n_blocks, float *out,
                     float *patches, cudaStream_t stream, const float *est = nullptr, long long est_stride = 0) {
    const bool learned = h->cfg.init == FSE_INIT_LEARNED && est == nullptr;
    const bool ordered = (h->cfg.flags & FSE_FLAG_ORDERED) != 0;
    if (ordered && n_blocks > 0 && (!out || est))
        return fail(h, FSE_ERR_INVALID_ARG, "ordered concealment needs the out image (and no warm start)");
    if (learned && n_blocks > 0 && !h->weights_loaded)
        return fail(h, FSE_ERR_NOT_TRAINED, "learned initialisation: no weights loaded (fse_load_init_weights)");
    if (n_blocks < 0) return fail(h, FSE_ERR_INVALID_ARG, "n_blocks %d < 0", n_blocks);
    if (n_blocks > 0 && !out && !patches) return fail(h, FSE_ERR_INVALID_ARG, "out and patches are both NULL");
    // plan key: every input of the captured launch (block list, pointers, geometry)
    uint64_t key = 0;
    if (n_blocks > 0 && blocks) {
        key = hash_words(blocks, (size_t)n_blocks * sizeof(fse_block), 0x51ed270b27a1f3c5ull);
        const uintptr_t ptrs[4] = {(uintptr_t)images, (uintptr_t)mask, (uintptr_t)out, (uintptr_t)patches};
        const long long geo[8] = {dtype, n_images, height, width, (long long)pitch, n_blocks,
                                  (long long)(uintptr_t)est, est_stride};
        key = fnv1a(ptrs, sizeof ptrs, key);
        key = fnv1a(geo, sizeof geo, key);
    }
    if (n_blocks > 0 && h->graph_valid && key == h->plan_key) {
        // same batch layout as the captured graph: validated when it was planned
        h->last_n_blocks = n_blocks;
        h->last_stream = stream;
        FSE_CUDA(h, cudaGraphLaunch(h->gexec, stream));
        return FSE_OK;
    }
    Plan pl;
    fse_status st = validate_and_plan(h, images, dtype, n_images, height, width, pitch, mask, blocks, n_blocks, pl);
    if (st != FSE_OK) return st;
    h->last_n_blocks = n_blocks;
    h->last_stream = stream;
    if (n_blocks == 0) return FSE_OK;
    const bool trace = (h->cfg.flags & FSE_FLAG_TRACE) != 0;
    int stride = 0;
    for (int c = 0; c < h->cfg.n_classes; ++c) stride = std::max(stride, h->cfg.cls[c].iters);
    if (learned && h->cfg.init_iters > 0) stride = h->cfg.init_iters;
    stride = std::max(stride, 1);

    if (h->graph_valid) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
        h->graph_valid = false;
    }
    // upload the sorted block list through pinned staging
    if (h->upload_done) cudaEventSynchronize(h->upload_done);
    if ((size_t)n_blocks > h->h_blocks_cap) {
        if (h->h_blocks) fse::host_free(h->h_blocks);
        h->h_blocks = nullptr;
        h->h_blocks_cap = 0;
        FSE_CUDA(h, fse::host_malloc(&h->h_blocks, (size_t)n_blocks * sizeof(BlockRec)));
        h->h_blocks_cap = n_blocks;
    }
    st = grow(h, &h->d_blocks, &h->blocks_cap, (size_t)n_blocks);
    if (st != FSE_OK) return st;
    std::memcpy(h->h_blocks, pl.sorted.data(), (size_t)n_blocks * sizeof(BlockRec));
    FSE_CUDA(h, cudaMemcpyAsync(h->d_blocks, h->h_blocks, (size_t)n_blocks * sizeof(BlockRec),
                                cudaMemcpyHostToDevice, stream));
    FSE_CUDA(h, cudaEventRecord(h->upload_done, stream));
    if (trace) {
        const size_t need = (size_t)n_blocks * stride;
        if (need > h->tr_cap) {
            fse::dev_free(h->d_tr_sel);
            fse::dev_free(h->d_tr_energy);
            fse::dev_free(h->d_tr_coef);
            fse::dev_free(h->d_tr_second);
            h->d_tr_sel = nullptr;
            h->d_tr_energy = nullptr;
            h->d_tr_coef = nullptr;
            h->d_tr_second = nullptr;
            h->tr_cap = 0;
            FSE_CUDA(h, fse::dev_malloc(&h->d_tr_sel, need * sizeof(int)));
            FSE_CUDA(h, fse::dev_malloc(&h->d_tr_energy, need * sizeof(float)));
            FSE_CUDA(h, fse::dev_malloc(&h->d_tr_coef, need * sizeof(float2)));
            FSE_CUDA(h, fse::dev_malloc(&h->d_tr_second, need * sizeof(float)));
            h->tr_cap = need;
        }
    }
    h->tr_stride = stride;
    DevParams &P = h->params;
    P = DevParams{};
    P.images = images;
    P.dtype = dtype;
    P.H = height;
    P.W = width;
    P.pitch = (long long)pitch;
    P.mask = mask;
    P.out = out;
    P.patches = patches;
    P.blocks = h->d_blocks;
    P.n_seg = pl.n_seg;
    for (int sg = 0; sg < pl.n_seg; ++sg) {
        P.seg_cls[sg] = pl.seg_cls[sg];
        P.seg_item_end[sg] = pl.seg_item_end[sg];
        P.seg_block_start[sg] = pl.seg_block_start[sg];
        P.seg_block_count[sg] = pl.seg_block_count[sg];
    }
    P.total_items = pl.total_items;
    set_classes(h, P, learned);
    P.n_images = n_images;
    setup_tma(h, P, pl.ks, dtype, images, mask, n_images, height, width, pitch);
    P.counter = h->d_counter;
    P.tr_sel = trace ? h->d_tr_sel : nullptr;
    P.tr_energy = trace ? h->d_tr_energy : nullptr;
    P.tr_coef = trace ? h->d_tr_coef : nullptr;
    P.tr_second = trace ? h->d_tr_second : nullptr;
    P.tr_stride = stride;
    P.tw = h->d_tw;
    h->learned_launch = learned;
    h->learned_n = n_blocks;
    if (learned) {
        const int MM = h->cnn_M * h->cnn_M;
        const size_t old_cap = h->est_cap;
        st = grow(h, &h->d_est, &h->est_cap, (size_t)n_blocks * MM);
        if (st != FSE_OK) return st;
        // the tensor-core network writes B only: the rest of every estimate stays 0
        if (h->est_cap != old_cap) FSE_CUDA(h, cudaMemset(h->d_est, 0, h->est_cap * sizeof(float)));
        if (!h->tc_net && !h->d_cnn_out) {
            // all four buffers or none: a failure frees the ones already made
            const size_t C = (size_t)h->cnn_chunk;
            cudaError_t e = fse::dev_malloc(&h->d_cnn_x, C * MM * 2 * sizeof(__nv_bfloat16));
            if (e == cudaSuccess) e = fse::dev_malloc(&h->d_cnn_a0, C * MM * 32 * sizeof(__nv_bfloat16));
            if (e == cudaSuccess) e = fse::dev_malloc(&h->d_cnn_a1, C * MM * 32 * sizeof(__nv_bfloat16));
            if (e == cudaSuccess) e = fse::dev_malloc(&h->d_cnn_out, C * MM * sizeof(float));
            if (e != cudaSuccess) {
                for (void **p : {reinterpret_cast<void **>(&h->d_cnn_x), reinterpret_cast<void **>(&h->d_cnn_a0),
                                 reinterpret_cast<void **>(&h->d_cnn_a1), reinterpret_cast<void **>(&h->d_cnn_out)}) {
                    fse::dev_free(*p);
                    *p = nullptr;
                }
                return cuda_fail(h, e, "network buffers");
            }
        }
        P.est = h->d_est;
        P.est_stride = MM;
    } else {
        P.est = est;
        P.est_stride = est_stride;
    }
    P.err = h->d_err;
    P.wait_ns = h->wait_ns;
    P.clamp_u8 = (h->cfg.flags & FSE_FLAG_CLAMP_U8) ? 1 : 0;
    P.fix_from = FSE_FIXED_W_FROM;   // read by the reduced-precision kernel set only
    P.ordered = ordered ? 1 : 0;
    if (ordered) {
        std::vector<int> nb_start, nb_list;
        ordered_neighbours(blocks, n_blocks, h->cfg.cls[0].block, h->cfg.cls[0].border, nb_start, nb_list);
        for (int i = 0; i < n_blocks; ++i)   // one class: the queue is the caller's order
            if (pl.sorted[i].orig != i) return fail(h, FSE_ERR_INVALID_ARG, "ordered concealment: queue order");
        st = grow(h, &h->d_nb_start, &h->nb_start_cap, nb_start.size());
        if (st != FSE_OK) return st;
        st = grow(h, &h->d_nb_list, &h->nb_list_cap, std::max<size_t>(nb_list.size(), 1));
        if (st != FSE_OK) return st;
        st = grow(h, &h->d_done, &h->done_cap, (size_t)n_blocks);
        if (st != FSE_OK) return st;
        FSE_CUDA(h, cudaMemcpy(h->d_nb_start, nb_start.data(), nb_start.size() * sizeof(int), cudaMemcpyHostToDevice));
        if (!nb_list.empty())
            FSE_CUDA(h, cudaMemcpy(h->d_nb_list, nb_list.data(), nb_list.size() * sizeof(int), cudaMemcpyHostToDevice));
        P.beta = h->cfg.reuse_weight;
        P.nb_start = h->d_nb_start;
        P.nb_list = h->d_nb_list;
        P.done = h->d_done;
        h->ordered_n = n_blocks;
    }
    int nt = 256, cps = ctas_per_sm(h, pl.ks, 256);
    TuneTicket ticket;
    st = autotune(h, pl, stream, &nt, &cps, &ticket);
    if (st != FSE_OK) return st;
    h->nt = nt;
    h->ks = pl.ks;
    h->grid = std::max(1, std::min(pl.total_items, cps * h->sm_count));
    st = capture_graph(h, pl.ks, nt, h->grid, &h->gexec);
    if (st != FSE_OK) return st;
    h->graph_valid = true;
    // while this class mix is still being tuned (FSE_TUNE_ASYNC), the next
    // call plans again instead of replaying this launch's configuration
    bool tuning = false;
    for (const auto &ss : h->sessions) tuning = tuning || ss.mix_sig == pl.mix_sig;
    h->plan_key = tuning ? 0 : key;
    st = tune_mark(h, ticket, stream, false);
    if (st != FSE_OK) return st;
    FSE_CUDA(h, cudaGraphLaunch(h->gexec, stream));
    return tune_mark(h, ticket, stream, true);
}

// Host-buffer batches over several images run as a pipeline of up to
// kHostChunks chunks: the images are uploaded in order on one stream while
// the chunks already resident are concealed on the caller's stream, and each
// chunk's patches are read back on a third stream as soon as its launch ends.
// A chunk is a contiguous range of the caller's block list and needs the
// images up to the last one its blocks read (the frames +-(T-1)/2 around a
// video volume's frame).  With blocks listed in image order the chunk sizes
// grow geometrically (1, 2, 4, 4, 4, 4, 4, 1 parts of 24): the first launch
// starts after 1/24 of the upload, each later chunk's upload is at most twice
// the previous chunk's work, so it stays hidden behind that launch unless the
// host-to-device copy is slower than twice the rate at which the kernel
// consumes frames, and only 1/24 of the patches are read back after the
// last launch; in any other order the pipeline is still correct, with less
// overlap.  Every block
// is concealed by the same code from the same inputs as in the one-launch
// path, so the patches are identical bit for bit.  The caller has validated
// the batch (image, class and position of every block).
fse_status run_host_chunked(fse_handle *h, const void *images, int dtype, int n_images, int height, int width,
                            size_t pitch, const uint8_t *loss_mask, const fse_block *blocks, int n_blocks,
                            float *patches, cudaStream_t stream) {
    if (!h->pipe_ready) {
        // each resource made once (a call that failed half-way resumes here)
        if (!h->h2d_stream) FSE_CUDA(h, cudaStreamCreateWithFlags(&h->h2d_stream, cudaStreamNonBlocking));
        if (!h->d2h_stream) FSE_CUDA(h, cudaStreamCreateWithFlags(&h->d2h_stream, cudaStreamNonBlocking));
        if (!h->ev_start) FSE_CUDA(h, cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming));
        if (!h->ev_out) FSE_CUDA(h, cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
        for (int c = 0; c < kHostChunks; ++c) {
            if (!h->ev_in[c]) FSE_CUDA(h, cudaEventCreateWithFlags(&h->ev_in[c], cudaEventDisableTiming));
            if (!h->ev_k[c]) FSE_CUDA(h, cudaEventCreateWithFlags(&h->ev_k[c], cudaEventDisableTiming));
        }
        if (!h->d_ccounter) FSE_CUDA(h, fse::dev_malloc(&h->d_ccounter, kHostChunks * sizeof(int)));
        h->pipe_ready = true;
    }
    const int K = std::min(kHostChunks, std::min(n_images, n_blocks));
    int halo = 0;
    for (int c = 0; c < h->cfg.n_classes; ++c)
        if (h->cfg.cls[c].frames > 1) halo = std::max(halo, (h->cfg.cls[c].frames - 1) / 2);
    // chunk c: blocks [cs[c], cs[c+1]), patches [po[c], po[c+1]), images [0, need[c]) resident
    int cs[kHostChunks + 1], need[kHostChunks];
    long long po[kHostChunks + 1];
    // a full pipeline has small first and last chunks (the GPU waits for the
    // first upload, the host for the last read-back) and chunks between that
    // at most double, so every upload after the first overlaps the launch
    // before it; small batches: equal chunks
    static const int kWeight[kHostChunks] = {1, 2, 4, 4, 4, 4, 4, 1};
    const bool weighted = K == kHostChunks && n_blocks >= 24 * 64;
    int wsum = 0, wacc = 0;
    for (int c = 0; c < K; ++c) wsum += weighted ? kWeight[c] : 1;
    for (int c = 0; c <= K; ++c) {
        cs[c] = (int)((long long)n_blocks * wacc / wsum);
        if (c < K) wacc += weighted ? kWeight[c] : 1;
    }
    long long acc = 0;
    int hi = 0;
    for (int c = 0; c < K; ++c) {
        po[c] = acc;
        for (int i = cs[c]; i < cs[c + 1]; ++i) {
            hi = std::max(hi, std::min(n_images, blocks[i].image + halo + 1));
            const long long b = h->cfg.cls[blocks[i].cls].block;
            acc += b * b;
        }
        need[c] = hi;
    }
    po[K] = acc;
    fse_status st = grow(h, &h->d_cblocks, &h->cblocks_cap, (size_t)n_blocks);
    if (st != FSE_OK) return st;
    if ((size_t)n_blocks > h->h_cblocks_cap) {
        if (h->h_cblocks) fse::host_free(h->h_cblocks);
        h->h_cblocks = nullptr;
        h->h_cblocks_cap = 0;
        FSE_CUDA(h, fse::host_malloc(&h->h_cblocks, (size_t)n_blocks * sizeof(BlockRec)));
        h->h_cblocks_cap = n_blocks;
    }
    // from here on, copies and launches may be queued: an error return first
    // waits for all three streams, so no queued copy still reads or writes
    // the staging buffers when the next call refills them
    auto drain = [&](fse_status st) {
        cudaStreamSynchronize(h->h2d_stream);
        cudaStreamSynchronize(stream);
        cudaStreamSynchronize(h->d2h_stream);
        return st;
    };
#define PIPE_CUDA(call)                                                 \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return drain(cuda_fail(h, e_, #call));   \
    } while (0)
    PIPE_CUDA(cudaEventRecord(h->ev_start, stream));
    PIPE_CUDA(cudaStreamWaitEvent(h->h2d_stream, h->ev_start, 0));
    PIPE_CUDA(cudaStreamWaitEvent(h->d2h_stream, h->ev_start, 0));
    DevParams P{};
    P.images = h->d_img;
    P.dtype = dtype;
    P.H = height;
    P.W = width;
    P.pitch = (long long)pitch;
    P.mask = h->d_mask;
    P.patches = h->d_patch;
    P.n_images = n_images;
    P.tr_stride = 1;
    P.tw = h->d_tw;
    P.err = h->d_err;
    P.wait_ns = h->wait_ns;
    P.clamp_u8 = (h->cfg.flags & FSE_FLAG_CLAMP_U8) ? 1 : 0;
    P.fix_from = FSE_FIXED_W_FROM;   // read by the reduced-precision kernel set only
    set_classes(h, P, false);
    const size_t img_frame = (size_t)height * pitch, mask_frame = (size_t)height * width;
    int copied = 0;
    for (int c = 0; c < K; ++c) {
        // upload what chunk c needs beyond the earlier chunks (issued before
        // the chunk is planned, so the copy engine starts at once; from
        // pageable memory the host waits here while chunk c-1 computes)
        if (need[c] > copied) {
            const size_t n = (size_t)(need[c] - copied);
            PIPE_CUDA(cudaMemcpyAsync(static_cast<char *>(h->d_img) + copied * img_frame,
                                        static_cast<const char *>(images) + copied * img_frame, n * img_frame,
                                        cudaMemcpyHostToDevice, h->h2d_stream));
            PIPE_CUDA(cudaMemcpyAsync(h->d_mask + copied * mask_frame, loss_mask + copied * mask_frame,
                                        n * mask_frame, cudaMemcpyHostToDevice, h->h2d_stream));
            copied = need[c];
        }
        const int n = cs[c + 1] - cs[c];
        Plan pc;
        st = validate_and_plan(h, h->d_img, dtype, n_images, height, width, pitch, h->d_mask, blocks + cs[c], n, pc);
        if (st != FSE_OK) return drain(st);
        for (BlockRec &r : pc.sorted) {
            r.orig += cs[c];
            r.patch_off += po[c];
        }
        // the sorted list travels on the upload stream too: a copy on the
        // compute stream would queue behind the next chunk's upload
        std::memcpy(h->h_cblocks + cs[c], pc.sorted.data(), (size_t)n * sizeof(BlockRec));
        PIPE_CUDA(cudaMemcpyAsync(h->d_cblocks + cs[c], h->h_cblocks + cs[c], (size_t)n * sizeof(BlockRec),
                                    cudaMemcpyHostToDevice, h->h2d_stream));
        PIPE_CUDA(cudaEventRecord(h->ev_in[c], h->h2d_stream));
        P.blocks = h->d_cblocks + cs[c];
        P.n_seg = pc.n_seg;
        for (int sg = 0; sg < pc.n_seg; ++sg) {
            P.seg_cls[sg] = pc.seg_cls[sg];
            P.seg_item_end[sg] = pc.seg_item_end[sg];
            P.seg_block_start[sg] = pc.seg_block_start[sg];
            P.seg_block_count[sg] = pc.seg_block_count[sg];
        }
        P.total_items = pc.total_items;
        P.counter = h->d_ccounter + c;
        setup_tma(h, P, pc.ks, dtype, h->d_img, h->d_mask, n_images, height, width, pitch);
        PIPE_CUDA(cudaStreamWaitEvent(stream, h->ev_in[c], 0));
        int nt = 256, cps = ctas_per_sm(h, pc.ks, 256);
        TuneTicket ticket;
        {   // the autotuner times graph replays of h->params: lend it this chunk's
            const DevParams saved = h->params;
            h->params = P;
            st = autotune(h, pc, stream, &nt, &cps, &ticket);
            h->params = saved;
            if (st != FSE_OK) return drain(st);
        }
        const int grid = std::max(1, std::min(pc.total_items, cps * h->sm_count));
        PIPE_CUDA(cudaMemsetAsync(P.counter, 0, sizeof(int), stream));
        st = tune_mark(h, ticket, stream, false);
        if (st != FSE_OK) return drain(st);
        PIPE_CUDA(launch_fse(h, pc.ks, nt, grid, P, stream));
        st = tune_mark(h, ticket, stream, true);
        if (st != FSE_OK) return drain(st);
        PIPE_CUDA(cudaEventRecord(h->ev_k[c], stream));
    }
    // read-backs after every launch is queued (a copy to pageable memory
    // returns only when it is done)
    for (int c = 0; c < K; ++c) {
        PIPE_CUDA(cudaStreamWaitEvent(h->d2h_stream, h->ev_k[c], 0));
        PIPE_CUDA(cudaMemcpyAsync(patches + po[c], h->d_patch + po[c], (size_t)(po[c + 1] - po[c]) * sizeof(float),
                                    cudaMemcpyDeviceToHost, h->d2h_stream));
    }
    PIPE_CUDA(cudaEventRecord(h->ev_out, h->d2h_stream));
    PIPE_CUDA(cudaStreamWaitEvent(stream, h->ev_out, 0));
#undef PIPE_CUDA
    h->last_n_blocks = n_blocks;
    h->last_stream = stream;
    FSE_CUDA(h, cudaStreamSynchronize(stream));
    return FSE_OK;
}

// A block list in device memory is copied to the handle's host staging on
// the caller's stream (after the work that may have produced it) and *blocks
// is pointed there; a host (pageable, pinned or managed) list is used as is.
fse_status host_block_list(fse_handle *h, const fse_block **blocks, int n_blocks, cudaStream_t stream) {
    if (n_blocks <= 0 || !*blocks) return FSE_OK;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, *blocks) != cudaSuccess) {
        cudaGetLastError();   // an unregistered host pointer on older drivers: host memory
        return FSE_OK;
    }
    if (a.type != cudaMemoryTypeDevice) return FSE_OK;
    if (a.device != h->device) return fail(h, FSE_ERR_INVALID_ARG, "blocks live on device %d, not %d", a.device, h->device);
    h->hb_stage.resize((size_t)n_blocks);
    FSE_CUDA(h, cudaMemcpyAsync(h->hb_stage.data(), *blocks, (size_t)n_blocks * sizeof(fse_block),
                                cudaMemcpyDeviceToHost, stream));
    FSE_CUDA(h, cudaStreamSynchronize(stream));
    *blocks = h->hb_stage.data();
    return FSE_OK;
}

}  // namespace

extern "C" {

fse_status fse_create(fse_handle **out, const fse_config *cfg) {
    if (!out) return fail(nullptr, FSE_ERR_INVALID_ARG, "out is NULL");
    fse_status st = validate_config(cfg);
    if (st != FSE_OK) return st;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) return fail(nullptr, FSE_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    if (cfg->device < 0 || cfg->device >= ndev)
        return fail(nullptr, FSE_ERR_INVALID_ARG, "device %d not in [0, %d)", cfg->device, ndev);
    DeviceGuard guard(cfg->device);
    fse_handle *h = new fse_handle();
    h->cfg = *cfg;
    h->device = cfg->device;
    h->cnn_M = cfg->cls[0].block + 2 * cfg->cls[0].border;
    auto bail = [&](fse_status s) {
        g_create_error = h->err;
        fse_destroy(h);
        return s;
    };
#define CREATE_CUDA(call)                                    \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return bail(cuda_fail(h, e_, #call)); \
    } while (0)
    cudaDeviceProp prop;
    CREATE_CUDA(cudaGetDeviceProperties(&prop, h->device));
    h->sm_count = prop.multiProcessorCount;
    h->cc = prop.major * 10 + prop.minor;
    // dynamic smem: the largest per-item region over the configured classes
    size_t smem = 0;
    for (int c = 0; c < cfg->n_classes; ++c) {
        const int F = cfg->cls[c].fft;
        smem = std::max(smem, (size_t)fse::cta_region_bytes(F, cfg->cls[c].frames > 1 ? 4 : 1));
    }
    h->smem_bytes = smem;
    h->ext = (cfg->flags & FSE_FLAG_ORDERED) != 0;
    for (int c = 0; c < cfg->n_classes; ++c) h->ext = h->ext || cfg->cls[c].frames > 1;
    // the kernel sets this handle's batches can run: the reduced-precision
    // set, the traced set, the extended set, or the image set and (with an
    // FFT-64 class) the FFT-64 set
    bool any64 = false;
    for (int c = 0; c < cfg->n_classes; ++c) any64 = any64 || cfg->cls[c].fft == 64;
    const bool traced = (cfg->flags & FSE_FLAG_TRACE) != 0;
    const bool fixw = (cfg->flags & FSE_FLAG_FIXED_W) != 0;
    for (int ks : {fse::kSetImage, fse::kSetExt, fse::kSetF64, fse::kSetTrace, fse::kSetFixW}) {
        if (fixw != (ks == fse::kSetFixW)) continue;
        if (!fixw && traced != (ks == fse::kSetTrace)) continue;
        if (!fixw && !traced && ((ks == fse::kSetExt) != h->ext || (ks == fse::kSetF64 && !any64))) continue;
        for (int t = 0; t < 2; ++t) {
            int occ = 0;
            CREATE_CUDA(fse::batch_kernel_prepare(ks, t ? 256 : 128, smem, &occ));
            if (occ < 1) return bail(fail(h, FSE_ERR_UNSUPPORTED, "kernel does not fit on an SM"));
            h->max_ctas[ks][t] = occ;
        }
    }
    h->tc_net = cfg->init == FSE_INIT_LEARNED && cfg->cls[0].block == 16 && cfg->cls[0].border == 16;
    if (h->tc_net) {
        if (prop.major < 10) return bail(fail(h, FSE_ERR_UNSUPPORTED, "learned initialisation needs sm_100 or later"));
        CREATE_CUDA(cudaFuncSetAttribute(fse_tc::cnn_tc_kernel<DevParams, BlockRec>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, fse_tc::kSmemBytes));
    }
    CREATE_CUDA(fse::dev_malloc(&h->d_err, sizeof(int)));
    CREATE_CUDA(cudaMemset(h->d_err, 0, sizeof(int)));
    CREATE_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CREATE_CUDA(cudaEventCreateWithFlags(&h->upload_done, cudaEventDisableTiming));
    CREATE_CUDA(fse::dev_malloc(&h->d_counter, sizeof(int)));
    CREATE_CUDA(fse::dev_malloc(&h->d_tw, 64 * sizeof(float2)));
    fse::twiddle_kernel<<<1, 64, 0, h->cap_stream>>>(h->d_tw);
    CREATE_CUDA(cudaGetLastError());
    for (int c = 0; c < cfg->n_classes; ++c) {
        const int M = cfg->cls[c].block + 2 * cfg->cls[c].border;
        const int T = cfg->cls[c].frames > 1 ? cfg->cls[c].frames : 1;
        CREATE_CUDA(fse::dev_malloc(&h->d_wtab[c], (size_t)T * M * M * sizeof(float)));
        fse::weight_table_kernel<<<(T * M * M + 255) / 256, 256, 0, h->cap_stream>>>(h->d_wtab[c], M, T,
                                                                                    (double)cfg->cls[c].rho);
        CREATE_CUDA(cudaGetLastError());
    }
    CREATE_CUDA(cudaStreamSynchronize(h->cap_stream));
#undef CREATE_CUDA
    *out = h;
    return FSE_OK;
}

fse_status fse_extrapolate_batch(fse_handle *h, const void *images, int dtype, int n_images, int height, int width,
                                 size_t pitch_bytes, const uint8_t *loss_mask, const fse_block *blocks, int n_blocks,
                                 float *out, float *patches, void *cuda_stream) {
    if (!h) return fail(nullptr, FSE_ERR_INVALID_ARG, "handle is NULL");
    DeviceGuard guard(h->device);
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    fse_status st = host_block_list(h, &blocks, n_blocks, stream);
    if (st != FSE_OK) return st;
    return run_batch(h, images, dtype, n_images, height, width, pitch_bytes, loss_mask, blocks, n_blocks, out,
                     patches, stream);
}

fse_status fse_extrapolate_batch_init(fse_handle *h, const void *images, int dtype, int n_images, int height,
                                      int width, size_t pitch_bytes, const uint8_t *loss_mask,
                                      const fse_block *blocks, int n_blocks, const float *init_estimate,
                                      size_t est_stride, float *out, float *patches, void *cuda_stream) {
    if (!h) return fail(nullptr, FSE_ERR_INVALID_ARG, "handle is NULL");
    if (n_blocks > 0 && !init_estimate) return fail(h, FSE_ERR_INVALID_ARG, "init_estimate is NULL");
    for (int c = 0; c < h->cfg.n_classes; ++c)
        if (h->cfg.cls[c].frames > 1) return fail(h, FSE_ERR_UNSUPPORTED, "the warm start is for image classes");
    long long maxMM = 0;
    for (int c = 0; c < h->cfg.n_classes; ++c) {
        const long long M = h->cfg.cls[c].block + 2 * h->cfg.cls[c].border;
        maxMM = std::max(maxMM, M * M);
    }
    if ((long long)est_stride < maxMM)
        return fail(h, FSE_ERR_INVALID_ARG, "est_stride %zu < largest area %lld", est_stride, maxMM);
    DeviceGuard guard(h->device);
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    fse_status st = host_block_list(h, &blocks, n_blocks, stream);
    if (st != FSE_OK) return st;
    return run_batch(h, images, dtype, n_images, height, width, pitch_bytes, loss_mask, blocks, n_blocks, out,
                     patches, stream, init_estimate, (long long)est_stride);
}

fse_status fse_load_init_weights(fse_handle *h, const float *params, size_t n) {
    if (!h) return fail(nullptr, FSE_ERR_INVALID_ARG, "handle is NULL");
    if (h->cfg.init != FSE_INIT_LEARNED)
        return fail(h, FSE_ERR_INVALID_ARG, "handle was not created with FSE_INIT_LEARNED");
    if (!params || n != (size_t)fse_net::kParams)
        return fail(h, FSE_ERR_INVALID_ARG, "need %d parameters", fse_net::kParams);
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(params[i])) return fail(h, FSE_ERR_INVALID_ARG, "parameter %zu is not finite", i);
    DeviceGuard guard(h->device);
    if (!h->d_cnn_params) FSE_CUDA(h, fse::dev_malloc(&h->d_cnn_params, fse_net::kParams * sizeof(float)));
    if (!h->d_cnn_wb) FSE_CUDA(h, fse::dev_malloc(&h->d_cnn_wb, fse_net::kWbTotal * sizeof(__nv_bfloat16)));
    if (!h->d_cnn_wt) FSE_CUDA(h, fse::dev_malloc(&h->d_cnn_wt, fse_net::kWtTotal * sizeof(float)));
    FSE_CUDA(h, cudaDeviceSynchronize());
    FSE_CUDA(h, cudaMemcpy(h->d_cnn_params, params, n * sizeof(float), cudaMemcpyHostToDevice));
    const int m = std::max(fse_net::kWbTotal, fse_net::kWtTotal);
    fse_net::pack_weights_kernel<<<(m + 255) / 256, 256>>>(h->d_cnn_params, h->d_cnn_wb, h->d_cnn_wt);
    FSE_CUDA(h, cudaGetLastError());
    if (h->tc_net) {
        if (!h->d_tc_w) FSE_CUDA(h, fse::dev_malloc(&h->d_tc_w, fse_tc::kWBytes));
        fse_tc::pack_tc_weights_kernel<<<(fse_tc::kWBytes / 2 + 255) / 256, 256>>>(
            h->d_cnn_params, reinterpret_cast<__nv_bfloat16 *>(h->d_tc_w));
        FSE_CUDA(h, cudaGetLastError());
    }
    FSE_CUDA(h, cudaDeviceSynchronize());
    h->weights_loaded = true;
    h->graph_valid = false;   // the captured launch reads the new weights anyway; re-plan to be safe
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    return FSE_OK;
}

fse_status fse_extrapolate_batch_host(fse_handle *h, const void *images, int dtype, int n_images, int height,
                                      int width, size_t pitch_bytes, const uint8_t *loss_mask,
                                      const fse_block *blocks, int n_blocks, float *patches, void *cuda_stream) {
    if (!h) return fail(nullptr, FSE_ERR_INVALID_ARG, "handle is NULL");
    DeviceGuard guard(h->device);
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    if (n_blocks < 0) return fail(h, FSE_ERR_INVALID_ARG, "n_blocks %d < 0", n_blocks);
    if (n_blocks == 0) {
        h->last_n_blocks = 0;
        return FSE_OK;
    }
    if (!patches) return fail(h, FSE_ERR_INVALID_ARG, "patches is NULL");
    // validate before any copy (the geometry is checked again by run_batch)
    long long patch_total = 0;
    fse_status st = validate_batch(h, images, dtype, n_images, height, width, pitch_bytes, loss_mask, blocks,
                                   n_blocks, &patch_total);
    if (st != FSE_OK) return st;
    const size_t img_bytes = (size_t)n_images * height * pitch_bytes;
    const size_t mask_bytes = (size_t)n_images * height * width;
    st = grow(h, reinterpret_cast<unsigned char **>(&h->d_img), &h->img_cap, img_bytes);
    if (st != FSE_OK) return st;
    st = grow(h, &h->d_mask, &h->mask_cap, mask_bytes);
    if (st != FSE_OK) return st;
    st = grow(h, &h->d_patch, &h->patch_cap, (size_t)patch_total);
    if (st != FSE_OK) return st;
    const bool plain = h->cfg.init == FSE_INIT_ZERO && !(h->cfg.flags & (FSE_FLAG_TRACE | FSE_FLAG_ORDERED));
    if (plain && n_images >= 2 && n_blocks >= 2)
        return run_host_chunked(h, images, dtype, n_images, height, width, pitch_bytes, loss_mask, blocks, n_blocks,
                                patches, stream);
    FSE_CUDA(h, cudaMemcpyAsync(h->d_img, images, img_bytes, cudaMemcpyHostToDevice, stream));
    FSE_CUDA(h, cudaMemcpyAsync(h->d_mask, loss_mask, mask_bytes, cudaMemcpyHostToDevice, stream));
    st = run_batch(h, h->d_img, dtype, n_images, height, width, pitch_bytes, h->d_mask, blocks, n_blocks, nullptr,
                   h->d_patch, stream);
    if (st != FSE_OK) return st;
    FSE_CUDA(h, cudaMemcpyAsync(patches, h->d_patch, (size_t)patch_total * sizeof(float), cudaMemcpyDeviceToHost,
                                stream));
    FSE_CUDA(h, cudaStreamSynchronize(stream));
    return FSE_OK;
}

fse_status fse_get_trace(fse_handle *h, int32_t *sel, float *energy, float *coef, size_t cap, int *stride_out) {
    if (!h) return fail(nullptr, FSE_ERR_INVALID_ARG, "handle is NULL");
    if (!(h->cfg.flags & FSE_FLAG_TRACE)) return fail(h, FSE_ERR_INVALID_ARG, "handle was created without FSE_FLAG_TRACE");
    DeviceGuard guard(h->device);
    const size_t n = (size_t)h->last_n_blocks * h->tr_stride;
    if (stride_out) *stride_out = h->tr_stride;
    if (n == 0 || (!sel && !energy && !coef)) return FSE_OK;   // stride query
    if (cap < n) return fail(h, FSE_ERR_INVALID_ARG, "cap %zu < n_blocks * stride = %zu", cap, n);
    FSE_CUDA(h, cudaStreamSynchronize(h->last_stream));
    if (sel) FSE_CUDA(h, cudaMemcpy(sel, h->d_tr_sel, n * sizeof(int), cudaMemcpyDeviceToHost));
    if (energy) FSE_CUDA(h, cudaMemcpy(energy, h->d_tr_energy, n * sizeof(float), cudaMemcpyDeviceToHost));
    if (coef) FSE_CUDA(h, cudaMemcpy(coef, h->d_tr_coef, n * sizeof(float2), cudaMemcpyDeviceToHost));
    return FSE_OK;
}

fse_status fse_get_trace_gap(fse_handle *h, float *gap2, size_t cap) {
    if (!h) return fail(nullptr, FSE_ERR_INVALID_ARG, "handle is NULL");
    if (!(h->cfg.flags & FSE_FLAG_TRACE)) return fail(h, FSE_ERR_INVALID_ARG, "handle was created without FSE_FLAG_TRACE");
    if (h->cfg.flags & FSE_FLAG_FIXED_W)
        return fail(h, FSE_ERR_UNSUPPORTED, "the top-two gap is not recorded with FSE_FLAG_FIXED_W");
    DeviceGuard guard(h->device);
    const size_t n = (size_t)h->last_n_blocks * h->tr_stride;
    if (n == 0) return FSE_OK;
    if (!gap2) return fail(h, FSE_ERR_INVALID_ARG, "gap2 is NULL");
    if (cap < n) return fail(h, FSE_ERR_INVALID_ARG, "cap %zu < n_blocks * stride = %zu", cap, n);
    FSE_CUDA(h, cudaStreamSynchronize(h->last_stream));
    std::vector<float> e1(n), e2(n);
    FSE_CUDA(h, cudaMemcpy(e1.data(), h->d_tr_energy, n * sizeof(float), cudaMemcpyDeviceToHost));
    FSE_CUDA(h, cudaMemcpy(e2.data(), h->d_tr_second, n * sizeof(float), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i)
        gap2[i] = e1[i] > 0.f ? (float)(((double)e1[i] - (double)e2[i]) / (double)e1[i]) : 0.f;
    return FSE_OK;
}

fse_status fse_get_area_model(fse_handle *h, float *model, size_t model_stride, void *cuda_stream) {
    if (!h) return fail(nullptr, FSE_ERR_INVALID_ARG, "handle is NULL");
    if (!(h->cfg.flags & FSE_FLAG_TRACE)) return fail(h, FSE_ERR_INVALID_ARG, "handle was created without FSE_FLAG_TRACE");
    size_t maxMM = 0;
    for (int c = 0; c < h->cfg.n_classes; ++c) {
        const size_t M = (size_t)(h->cfg.cls[c].block + 2 * h->cfg.cls[c].border);
        maxMM = std::max(maxMM, M * M);
    }
    if (model_stride < maxMM) return fail(h, FSE_ERR_INVALID_ARG, "model_stride %zu < largest area %zu", model_stride, maxMM);
    for (int c = 0; c < h->cfg.n_classes; ++c)
        if (h->cfg.cls[c].frames > 1) return fail(h, FSE_ERR_UNSUPPORTED, "the area model is for image classes");
    if (h->last_n_blocks == 0) return FSE_OK;
    if (!model) return fail(h, FSE_ERR_INVALID_ARG, "model is NULL");
    DeviceGuard guard(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (st != h->last_stream) FSE_CUDA(h, cudaStreamSynchronize(h->last_stream));
    area_model_kernel<<<h->last_n_blocks, 256, 0, st>>>(h->params, model, (long long)model_stride);
    FSE_CUDA(h, cudaGetLastError());
    return FSE_OK;
}

fse_status fse_sync(fse_handle *h) {
    if (!h) return fail(nullptr, FSE_ERR_INVALID_ARG, "handle is NULL");
    DeviceGuard guard(h->device);
    FSE_CUDA(h, cudaStreamSynchronize(h->last_stream));
    int e = 0;
    FSE_CUDA(h, cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != 0) {
        FSE_CUDA(h, cudaMemset(h->d_err, 0, sizeof(int)));
        if (e & fse::kErrBounds)
            return fail(h, FSE_ERR_CUDA, "device bounds check: an index left its buffer (access skipped)");
        if (e & fse::kErrTimeout)
            return fail(h, FSE_ERR_TIMEOUT, "a bounded device wait ran out (limit %llu ns)", h->wait_ns);
        return fail(h, FSE_ERR_INVALID_ARG, "a lost block's loss area is not marked lost in the loss mask");
    }
    return FSE_OK;
}

fse_status fse_set_wait_limit(fse_handle *h, unsigned long long ns) {
    if (!h) return fail(nullptr, FSE_ERR_INVALID_ARG, "handle is NULL");
    if (ns > 60000000000ull) return fail(h, FSE_ERR_INVALID_ARG, "wait limit %llu ns above 60 s", ns);
    if (ns != h->wait_ns && h->gexec) {   // the captured launch holds the old limit
        DeviceGuard guard(h->device);
        if (h->last_stream) cudaStreamSynchronize(h->last_stream);
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
        h->graph_valid = false;
    }
    h->wait_ns = ns;
    return FSE_OK;
}

fse_status fse_set_tuning(fse_handle *h, int mode) {
    if (!h) return fail(nullptr, FSE_ERR_INVALID_ARG, "handle is NULL");
    if (mode != FSE_TUNE_SYNC && mode != FSE_TUNE_ASYNC && mode != FSE_TUNE_OFF)
        return fail(h, FSE_ERR_INVALID_ARG, "tuning mode %d unknown", mode);
    h->tune_mode = mode;
    return FSE_OK;
}

fse_status fse_get_tuning(const fse_handle *h, int *mode, int *pending) {
    if (!h) return fail(nullptr, FSE_ERR_INVALID_ARG, "handle is NULL");
    if (mode) *mode = h->tune_mode;
    if (pending) *pending = (int)h->sessions.size();
    return FSE_OK;
}

void fse_test_clear_tuning_cache(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
}

const char *fse_last_error(const fse_handle *h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void fse_destroy(fse_handle *h) {
    if (!h) return;
    {
        DeviceGuard guard(h->device);
        if (h->last_stream || h->cap_stream) cudaDeviceSynchronize();
        if (h->gexec) cudaGraphExecDestroy(h->gexec);
        for (auto &p : h->d_wtab) fse::dev_free(p);
        fse::dev_free(h->d_tw);
        fse::dev_free(h->d_counter);
        fse::dev_free(h->d_blocks);
        if (h->h_blocks) fse::host_free(h->h_blocks);
        fse::dev_free(h->d_tr_sel);
        fse::dev_free(h->d_tr_energy);
        fse::dev_free(h->d_tr_coef);
        fse::dev_free(h->d_tr_second);
        fse::dev_free(h->d_img);
        fse::dev_free(h->d_mask);
        fse::dev_free(h->d_patch);
        fse::dev_free(h->d_cnn_params);
        fse::dev_free(h->d_cnn_wb);
        fse::dev_free(h->d_cnn_wt);
        fse::dev_free(h->d_cnn_x);
        fse::dev_free(h->d_tc_w);
        fse::dev_free(h->d_err);
        fse::dev_free(h->d_nb_start);
        fse::dev_free(h->d_nb_list);
        fse::dev_free(h->d_done);
        fse::dev_free(h->d_cnn_a0);
        fse::dev_free(h->d_cnn_a1);
        fse::dev_free(h->d_cnn_out);
        fse::dev_free(h->d_est);
        if (h->upload_done) cudaEventDestroy(h->upload_done);
        fse::dev_free(h->d_cblocks);
        if (h->h_cblocks) fse::host_free(h->h_cblocks);
        fse::dev_free(h->d_ccounter);
        for (int c = 0; c < kHostChunks; ++c) {
            if (h->ev_in[c]) cudaEventDestroy(h->ev_in[c]);
            if (h->ev_k[c]) cudaEventDestroy(h->ev_k[c]);
        }
        for (auto &ss : h->sessions) destroy_session(ss);
        if (h->ev_start) cudaEventDestroy(h->ev_start);
        if (h->ev_out) cudaEventDestroy(h->ev_out);
        if (h->h2d_stream) cudaStreamDestroy(h->h2d_stream);
        if (h->d2h_stream) cudaStreamDestroy(h->d2h_stream);
        if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    }
    delete h;
}

}  // extern "C"
