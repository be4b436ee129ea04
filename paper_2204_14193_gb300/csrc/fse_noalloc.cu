// fse_noalloc.cu -- fse_extrapolate_batch_noalloc: the batch concealment
// without any device allocation, for callers that may not call cudaMalloc.
//
// Some host programs cannot let a library allocate device memory once they
// are running: cudaMalloc / cudaFree may synchronise the whole device (a
// stall a real-time video pipeline cannot afford), some applications hand
// all device memory to their own pool allocator at start-up and cap what
// anything else may take, and some certified or embedded processes forbid
// any allocation after initialisation.  This entry point serves them: it
// takes the same inputs and output image as fse_extrapolate_batch but no
// handle, and keeps everything the persistent kernel needs beyond its inputs
// and outputs (work-queue head, bucketed block list, Eq. (3) weight tables,
// DFT twiddles) in one fixed, file-scope __device__ array.
//
// That array is g_scratch below, kNoallocScratchBytes bytes; every GPU that
// loads the library holds it until the process exits.  All calls on one
// device share it and it keeps the last call's contents, so calls whose work
// overlaps on the GPU (other streams, other host threads) race on it and must
// be serialised by the caller.  Each call rewrites every part it reads and
// zeroes the work-queue head before the kernel starts.  The persistent kernel
// itself is the library's (fse_kernels.cuh); the table kernels are a private
// copy (fse_tables.cuh, internal linkage).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "fse.h"
#include "fse_kernels.cuh"
#include "fse_tables.cuh"

void fse_internal_set_global_error(const char *msg);   // fse_api.cu: text of fse_last_error(NULL)

namespace {

constexpr int kNoallocMaxBlocks = 65536;
constexpr int kNoallocSmem = fse::cta_region_bytes(64);   // the largest per-CTA region
constexpr int kMaxM = 64;   // largest window edge M = b + 2d <= F <= 64

// layout of the scratch array (byte offsets, each 256-byte aligned)
constexpr size_t kOffCounter = 0;
constexpr size_t kOffTw = 256;
constexpr size_t kOffWtab = kOffTw + 64 * sizeof(float2);                           // 768
constexpr size_t kOffRaw = kOffWtab + FSE_MAX_CLASSES * kMaxM * kMaxM * sizeof(float);  // 66304
constexpr size_t kOffRec = (kOffRaw + kNoallocMaxBlocks * sizeof(fse_block) + 255) / 256 * 256;
constexpr size_t kNoallocScratchBytes = kOffRec + kNoallocMaxBlocks * sizeof(fse::BlockRec);
static_assert(kOffWtab % 256 == 0 && kOffRaw % 256 == 0 && kOffRec % 256 == 0, "scratch alignment");

// The scratch of every call on a device (3.1 MB).  In host code this name is
// only a host-side stand-in: kernels get its device address from
// cudaGetSymbolAddress, looked up once per device.
static __device__ __align__(256) unsigned char g_scratch[kNoallocScratchBytes];

struct DeviceScratch {
    unsigned char *ptr = nullptr;
    int sm_count = 0;
    int ctas_per_sm[3] = {};   // per kernel set (fse_device.cuh), 128 threads per CTA
};
constexpr int kMaxDevices = 64;
DeviceScratch g_dev[kMaxDevices];
std::mutex g_mu;

fse_status fail(fse_status st, const char *msg) {
    fse_internal_set_global_error(msg);
    return st;
}

// First queue position of each class's blocks, passed to the bucketing
// kernel by value.
struct Starts {
    int v[FSE_MAX_CLASSES];
};

// Bucket the caller's blocks by class into the queue order of the plan:
// warp c walks the list 32 blocks at a time and appends the blocks of class c
// (ballot + popcount keeps the caller's order inside the class).
__global__ void noalloc_bucket_kernel(const fse_block *raw, int n, fse::BlockRec *rec, const Starts starts,
                                      int n_classes) {
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (c >= n_classes) return;
    int pos = starts.v[c];
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        fse_block b = {0, 0, 0, -1};
        if (i < n) b = raw[i];
        const unsigned hit = __ballot_sync(0xffffffffu, b.cls == c);
        if (b.cls == c) {
            fse::BlockRec r;
            r.image = b.image;
            r.x = b.x;
            r.y = b.y;
            r.orig = i;
            r.patch_off = 0;
            r.pad = 0;
            rec[pos + __popc(hit & ((1u << lane) - 1u))] = r;
        }
        pos += __popc(hit);
    }
}

__global__ void noalloc_setup_kernel(int *counter) { *counter = 0; }

}  // namespace

extern "C" fse_status fse_extrapolate_batch_noalloc(const fse_class *classes, int n_classes, const void *images,
                                                    int dtype, int n_images, int height, int width,
                                                    size_t pitch_bytes, const uint8_t *loss_mask,
                                                    const fse_block *blocks, int n_blocks, float *out,
                                                    void *cuda_stream) {
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    // ---- validation (host only, nothing enqueued on failure) ----
    if (!classes || n_classes < 1 || n_classes > FSE_MAX_CLASSES)
        return fail(FSE_ERR_INVALID_ARG, "noalloc: classes NULL or n_classes not in [1, 4]");
    for (int c = 0; c < n_classes; ++c) {
        const fse_class &k = classes[c];
        if (k.fft != 16 && k.fft != 32 && k.fft != 64)
            return fail(FSE_ERR_INVALID_ARG, "noalloc: fft must be 16, 32 or 64");
        if (k.block < 1 || 2 * k.block > k.fft || k.border < 1 || k.block + 2 * k.border > k.fft)
            return fail(FSE_ERR_INVALID_ARG, "noalloc: need 1 <= b <= fft/2, d >= 1, b + 2d <= fft");
        if (!(k.rho > 0.f && k.rho <= 1.f) || !(k.gamma > 0.f && k.gamma < 2.f) || k.iters < 0 || k.iters > 4096)
            return fail(FSE_ERR_INVALID_ARG, "noalloc: rho, gamma or iters out of range");
        if (k.frames > 1) return fail(FSE_ERR_UNSUPPORTED, "noalloc: video volumes need fse_extrapolate_batch");
    }
    if (n_blocks < 0) return fail(FSE_ERR_INVALID_ARG, "noalloc: n_blocks < 0");
    if (n_blocks > kNoallocMaxBlocks)
        return fail(FSE_ERR_INVALID_ARG,
                    "noalloc: n_blocks exceeds the fixed scratch maximum of 65536 blocks per call; "
                    "split the batch or use fse_extrapolate_batch");
    if (dtype != FSE_DTYPE_U8 && dtype != FSE_DTYPE_F32) return fail(FSE_ERR_INVALID_ARG, "noalloc: dtype unknown");
    if (n_blocks == 0) return FSE_OK;
    if (!images || !loss_mask || !blocks || !out)
        return fail(FSE_ERR_INVALID_ARG, "noalloc: images, loss_mask, blocks and out must be non-NULL");
    if (n_images < 1 || height < 1 || width < 1) return fail(FSE_ERR_INVALID_ARG, "noalloc: bad geometry");
    const size_t es = dtype == FSE_DTYPE_U8 ? 1 : 4;
    if (pitch_bytes < (size_t)width * es) return fail(FSE_ERR_INVALID_ARG, "noalloc: pitch < width * element size");
    if (dtype == FSE_DTYPE_F32 && (pitch_bytes % 4 != 0 || (reinterpret_cast<uintptr_t>(images) & 3)))
        return fail(FSE_ERR_INVALID_ARG, "noalloc: FP32 images need 4-byte aligned base and pitch");
    int cnt[FSE_MAX_CLASSES] = {0, 0, 0, 0};
    for (int i = 0; i < n_blocks; ++i) {
        const fse_block &b = blocks[i];
        if (b.cls < 0 || b.cls >= n_classes) return fail(FSE_ERR_INVALID_ARG, "noalloc: block class out of range");
        const int e = classes[b.cls].block;
        if (b.image < 0 || b.image >= n_images || b.x < 0 || b.y < 0 || b.x + e > width || b.y + e > height)
            return fail(FSE_ERR_INVALID_ARG, "noalloc: a block is not inside its image");
        cnt[b.cls]++;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(FSE_ERR_CUDA, "noalloc: no current CUDA device");

    // ---- once per device: scratch address, kernel attribute, occupancy ----
    DeviceScratch ds;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        DeviceScratch &d = g_dev[dev];
        if (!d.ptr) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p) return fail(FSE_ERR_CUDA, "noalloc: cudaGetSymbolAddress(g_scratch) failed");
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return fail(FSE_ERR_CUDA, "noalloc: device query failed");
            for (int ks : {fse::kSetImage, fse::kSetF64}) {
                int occ = 0;
                if (fse::batch_kernel_prepare(ks, 128, kNoallocSmem, &occ) != cudaSuccess || occ < 1)
                    return fail(FSE_ERR_CUDA, "noalloc: cannot set the kernel's shared-memory size or occupancy");
                d.ctas_per_sm[ks] = occ;
            }
            d.sm_count = sms;
            d.ptr = static_cast<unsigned char *>(p);
        }
        ds = d;
    }
    unsigned char *S = ds.ptr;
    int *d_counter = reinterpret_cast<int *>(S + kOffCounter);
    float2 *d_tw = reinterpret_cast<float2 *>(S + kOffTw);
    float *d_wtab = reinterpret_cast<float *>(S + kOffWtab);
    fse_block *d_raw = reinterpret_cast<fse_block *>(S + kOffRaw);
    fse::BlockRec *d_rec = reinterpret_cast<fse::BlockRec *>(S + kOffRec);

    // ---- plan (host, fixed-size arrays only) ----
    int order[FSE_MAX_CLASSES];
    for (int i = 0; i < n_classes; ++i) order[i] = i;
    std::stable_sort(order, order + n_classes, [&](int a, int b) { return classes[a].fft > classes[b].fft; });
    fse::DevParams P{};
    int seg_start_by_cls[FSE_MAX_CLASSES] = {0, 0, 0, 0};
    int pos = 0, items = 0;
    for (int oi = 0; oi < n_classes; ++oi) {
        const int c = order[oi];
        seg_start_by_cls[c] = pos;
        if (cnt[c] == 0) continue;
        const int F = classes[c].fft, bpi = 4096 / (F * F);
        items += (cnt[c] + bpi - 1) / bpi;
        P.seg_cls[P.n_seg] = c;
        P.seg_item_end[P.n_seg] = items;
        P.seg_block_start[P.n_seg] = pos;
        P.seg_block_count[P.n_seg] = cnt[c];
        P.n_seg++;
        pos += cnt[c];
    }
    P.total_items = items;
    bool all_f64 = true;
    for (int sg = 0; sg < P.n_seg; ++sg) all_f64 = all_f64 && classes[P.seg_cls[sg]].fft == 64;
    const int ks = fse::kernel_set_for(false, all_f64);
    P.images = images;
    P.dtype = dtype;
    P.n_images = n_images;
    P.H = height;
    P.W = width;
    P.pitch = (long long)pitch_bytes;
    P.mask = loss_mask;
    P.out = out;
    P.patches = nullptr;
    P.blocks = d_rec;
    for (int c = 0; c < n_classes; ++c) {
        fse::DevClass &D = P.cls[c];
        D.F = classes[c].fft;
        D.b = classes[c].block;
        D.d = classes[c].border;
        D.M = D.b + 2 * D.d;
        D.off = (D.F - D.M) / 2;
        D.iters = classes[c].iters;
        D.bpi = 4096 / (D.F * D.F);
        D.gamma = classes[c].gamma;
        D.wtab = d_wtab + (size_t)c * kMaxM * kMaxM;
    }
    P.counter = d_counter;
    P.tr_sel = nullptr;
    P.tr_energy = nullptr;
    P.tr_coef = nullptr;
    P.tr_stride = 1;
    P.tw = d_tw;
    P.wait_ns = fse::kDrainNs;   // no bounded wait runs here (no TMA gather, no ordering)

    // ---- enqueue: tables, block list, queue head, persistent kernel ----
    fse::twiddle_kernel<<<1, 64, 0, stream>>>(d_tw);
    for (int c = 0; c < n_classes; ++c) {
        const int M = P.cls[c].M;
        fse::weight_table_kernel<<<(M * M + 255) / 256, 256, 0, stream>>>(d_wtab + (size_t)c * kMaxM * kMaxM, M, 1,
                                                                          (double)classes[c].rho);
    }
    if (cudaMemcpyAsync(d_raw, blocks, (size_t)n_blocks * sizeof(fse_block), cudaMemcpyHostToDevice, stream) !=
        cudaSuccess)
        return fail(FSE_ERR_CUDA, "noalloc: block-list copy failed");
    // class -> segment start travels in the kernel argument (by value)
    Starts st;
    for (int c = 0; c < FSE_MAX_CLASSES; ++c) st.v[c] = seg_start_by_cls[c];
    noalloc_bucket_kernel<<<1, 32 * FSE_MAX_CLASSES, 0, stream>>>(d_raw, n_blocks, d_rec, st, n_classes);
    noalloc_setup_kernel<<<1, 1, 0, stream>>>(d_counter);
    const int grid = std::max(1, std::min(items, ds.ctas_per_sm[ks] * ds.sm_count));
    if (fse::batch_kernel_launch(ks, 128, grid, kNoallocSmem, stream, P) != cudaSuccess)
        return fail(FSE_ERR_CUDA, "noalloc: kernel launch failed");
    return FSE_OK;
}
