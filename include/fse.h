/*
 * fse.h -- C ABI of the GB300 (sm_103a) complex-valued Frequency Selective
 * Extrapolation library (cFSE, Seiler & Kaup, arXiv 2204.14193).
 *
 * The library conceals lost b x b blocks of 8-bit or FP32 images.  For every
 * lost block it builds the extrapolation area L = A u B of Fig. 1 (an
 * M x M window, M = b + 2d, centred on the loss area B), weights the support
 * area A with Eq. (3), runs the I iterations of Algorithm 1 in the Fourier
 * domain on an F x F grid and writes Re{g} on B (the last loop of
 * Algorithm 1).
 *
 * Conventions shared by every entry point:
 *   - Nothing is thrown across the ABI; every call returns an fse_status.
 *     fse_last_error() gives a one-line reason for the last failure.
 *   - Arguments are validated on the host before anything is enqueued; a
 *     rejected call launches nothing and leaves all outputs untouched.
 *   - Device-pointer calls are asynchronous on the given CUDA stream (NULL =
 *     the legacy default stream) and return after enqueueing.  One handle
 *     serves one stream at a time; calls on one handle must not overlap.
 *   - Results are deterministic: the same inputs give bit-identical outputs.
 *   - Image geometry: n_images images of height x width samples.  Image i,
 *     row y starts at byte (i * height + y) * pitch_bytes of `images`.  The
 *     loss mask is n_images x height x width bytes, tightly packed (row pitch
 *     = width).  The output image, when given, is n_images x height x width
 *     FP32 values, tightly packed; only the samples of B are written.
 *   - Every sample of a window that lies outside its image, is marked lost in
 *     the mask (mask != 0), or belongs to the block's own B has weight 0.
 *     Blocks are concealed independently of each other from the original
 *     mask (concealed values of one block are never support of another).
 */
#ifndef FSE_H
#define FSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FSE_MAX_CLASSES 4

typedef enum {
    FSE_OK = 0,
    FSE_ERR_INVALID_ARG = 1, /* a bad argument; nothing was enqueued          */
    FSE_ERR_UNSUPPORTED = 2, /* valid but not implemented (e.g. F = 128)       */
    FSE_ERR_CUDA = 3,        /* a CUDA runtime call failed                     */
    FSE_ERR_OOM = 4,         /* device or pinned host allocation failed        */
    FSE_ERR_TIMEOUT = 5,     /* a bounded device wait ran out                  */
    FSE_ERR_NOT_TRAINED = 6  /* learned initialisation without loaded weights  */
} fse_status;

typedef enum { FSE_DTYPE_U8 = 0, FSE_DTYPE_F32 = 1 } fse_dtype;

typedef enum {
    FSE_INIT_ZERO = 0,    /* Algorithm 1 as printed: the model starts at zero */
    FSE_INIT_LEARNED = 1  /* a CNN estimate e of the area seeds the model     */
} fse_init_mode;

/* fse_config.flags */
#define FSE_FLAG_TRACE 1u /* record every selection (see fse_get_trace) */
/* Ordered concealment (no counterpart in the paper, which conceals every block
 * from the original support): blocks are concealed in the caller's order and
 * the samples of blocks concealed before a block, where they fall in its
 * area, join its support at their concealed values with weight
 * reuse_weight x Eq. (3).  One image class of fft 32 or 64, zero
 * initialisation, the `out`
 * image of fse_extrapolate_batch required (the concealed values are read
 * from it); not with the host-buffer or allocation-free entry points.  On
 * the GPU a block waits (bounded by the handle's wait limit, see
 * fse_set_wait_limit) for the blocks it reuses. */
#define FSE_FLAG_ORDERED 2u
/* Outputs as 8-bit sample values: every concealed sample is clamped to
 * [0, 255] and rounded to the nearest integer, ties to even (still written
 * as FP32).  Without it the output is the unclamped model Re{g} (Algorithm 1
 * produces real values; the paper does not round). */
#define FSE_FLAG_CLAMP_U8 4u
/* Reduced-precision residual storage (the Conclusion's remark that the method
 * suits fixed-point arithmetic).  After the first FSE_FIXED_W_FROM residual
 * updates of a block, the spectrum W that every update re-reads (Eq. (18))
 * is held as 16-bit fixed-point codes q = round(W / W[0,0] * 32767) (round
 * to nearest, ties to even, decided in FP32; |W| <= W[0,0] for a
 * non-negative weight), half the shared-memory bytes per update; the
 * residual R_w, c-hat and the model stay FP32.  The first updates carry the
 * large coefficients and keep FP32 W: codes from the first update move the
 * concealed samples by more than 1e-2, from the switch on they stay within
 * 1e-2 of Algorithm 1 along the same selections.  Image classes of fft 64
 * only, not with FSE_FLAG_ORDERED (FSE_ERR_UNSUPPORTED at fse_create);
 * FSE_FLAG_TRACE records the selections but not the top-two gap
 * (fse_get_trace_gap returns FSE_ERR_UNSUPPORTED). */
#define FSE_FLAG_FIXED_W 8u
#define FSE_FIXED_W_FROM 20   /* FP32 updates before the switch */

/*
 * One block-size class.
 *   block  b, edge of the lost block (loss area B), 1 <= b <= fft/2
 *   border d, width of the support frame around B, d >= 1, b + 2d <= fft
 *   fft    F, FFT size and DFT period: 16, 32 or 64 (Section IV uses 64x64)
 *   rho    rho-hat of Eq. (3), 0 < rho <= 1
 *   gamma  orthogonality-deficiency compensation factor of Eq. (13),
 *          0 < gamma < 2 (the paper uses values in (0, 1])
 *   iters  I, number of selected basis functions (Algorithm 1), 0 <= I <= 4096
 *   frames 0 or 1 for image areas.  3 for video volumes (Section II and the
 *          Conclusion: the method extends to higher-dimensional data such as
 *          video): the extrapolation volume is the M x M area in the block's
 *          frame and in the frames before and after it (images[] is then a
 *          sequence of frames; frames outside it are not support), the
 *          weighting function's distance includes the frame offset, and
 *          Algorithm 1 runs on a 4 x F x F transform grid (the volume in
 *          planes 0..2) with 3-D basis functions and circular shifts.  Volume
 *          classes need fft 16 or 32; they are not available with the learned
 *          initialisation, the warm start, fse_get_area_model or the
 *          allocation-free entry.
 */
typedef struct {
    int block;
    int border;
    int fft;
    float rho;
    float gamma;
    int iters;
    int frames;   /* 0 or 1: image areas; 3: video volumes (see below) */
} fse_class;

/*
 * Handle configuration.
 *   n_classes   number of valid entries of cls (1..FSE_MAX_CLASSES)
 *   init        fse_init_mode
 *   init_iters  iterations run after a learned initialisation (0 = iters)
 *   device      CUDA device ordinal
 *   flags       FSE_FLAG_* bits
 */
typedef struct {
    int n_classes;
    fse_class cls[FSE_MAX_CLASSES];
    int init;
    int init_iters;
    int device;
    unsigned flags;
    float reuse_weight;   /* FSE_FLAG_ORDERED: weight factor of reused samples, (0, 1] */
} fse_config;

/* A lost block: image index, top-left sample (x = column, y = row) of B, and
 * the index of its class in fse_config.cls.  B must lie inside the image. */
typedef struct {
    int32_t image;
    int32_t x;
    int32_t y;
    int32_t cls;
} fse_block;

typedef struct fse_handle fse_handle;

/*
 * Create a handle on cfg->device: validates the configuration, computes the
 * Eq. (3) weight tables and the DFT twiddle table on the device, and
 * allocates the work-queue state.  *out is set only on success.  The handle
 * owns all its device memory, CUDA graphs and streams.
 */
fse_status fse_create(fse_handle **out, const fse_config *cfg);

/*
 * Conceal a batch of lost blocks (Algorithm 1 once per block), device
 * buffers.
 *   images       device, dtype FSE_DTYPE_U8 or FSE_DTYPE_F32, geometry above
 *   loss_mask    device, uint8, 1 = lost sample, geometry above
 *   blocks       n_blocks descriptors in host memory (read during the call)
 *                or in device memory of the handle's device (copied to the
 *                host on cuda_stream first, after the stream's earlier work:
 *                the call then waits for the stream)
 *   out          device FP32 image (geometry above) or NULL; only B samples
 *                of each block are written
 *   patches      device FP32 array or NULL: block i's b x b result (row-major)
 *                at offset sum_{j<i} b_j^2, in the order of `blocks`
 *   cuda_stream  cudaStream_t to enqueue on
 * At least one of out, patches must be non-NULL when n_blocks > 0.
 * n_blocks == 0 is valid and enqueues nothing.  The batch runs as one
 * persistent, graph-captured launch; the graph is rebuilt only when the block
 * list or a pointer changes.  The launch shape (threads per CTA, CTAs per SM)
 * is chosen by timing the candidates on the batch itself the first time a
 * class mix of that size appears in the process; by default that first call
 * waits for its timing runs (see fse_set_tuning for a mode that never waits);
 * later calls and other handles reuse the choice.
 */
fse_status fse_extrapolate_batch(fse_handle *h, const void *images, int dtype, int n_images,
                                 int height, int width, size_t pitch_bytes,
                                 const uint8_t *loss_mask, const fse_block *blocks,
                                 int n_blocks, float *out, float *patches, void *cuda_stream);

/*
 * Warm start (no counterpart in the paper): Algorithm 1 on the residual of a
 * caller-supplied estimate e of every block's extrapolation area.  The
 * support samples become s - e, the model starts at zero, and B receives
 * e + Re{g}.  init_estimate: device FP32; block i (order of `blocks`) has its
 * M x M estimate (row-major, sample units, M = b + 2d of its class) at offset
 * i * est_stride, est_stride >= the largest M*M.  Other arguments as
 * fse_extrapolate_batch.  The learned initialisation (FSE_INIT_LEARNED) is
 * this call with e produced on the GPU by the network.
 */
fse_status fse_extrapolate_batch_init(fse_handle *h, const void *images, int dtype, int n_images,
                                      int height, int width, size_t pitch_bytes,
                                      const uint8_t *loss_mask, const fse_block *blocks,
                                      int n_blocks, const float *init_estimate, size_t est_stride,
                                      float *out, float *patches, void *cuda_stream);

/*
 * Load the learned-initialisation network (FSE_CNN_PARAMS FP32 values, the
 * layout of fse_cnn_set_params) into a handle created with init =
 * FSE_INIT_LEARNED (one block class).  fse_extrapolate_batch then, inside its
 * captured launch, evaluates the network on every block's area (input as
 * described for the fse_cnn_* calls), takes its output on B as the estimate
 * e (zero on the rest of the area, so the support is unchanged), runs
 * Algorithm 1 for init_iters (or iters when 0) iterations, and writes
 * e + Re{g} on B: the network is trained to supply what iterations beyond
 * init_iters would add.
 * Without loaded weights it returns FSE_ERR_NOT_TRAINED.  Synchronous.
 */
fse_status fse_load_init_weights(fse_handle *h, const float *params, size_t n);

/*
 * The same computation with HOST buffers (pageable or pinned): copies images
 * and mask to the handle's device staging buffers, runs the batch, copies the
 * patches (layout as above) back, and synchronises the stream before it
 * returns.  `patches` is a host FP32 array of sum_i b_i^2 values.
 * With two or more images (zero initialisation, no trace, not ordered) the
 * call is a pipeline: the block list is cut into up to 8 contiguous chunks
 * (1, 2, 4, 4, 4, 4, 4 and 1 parts of 24 of a large batch: each upload after
 * the first is at most twice the work of the launch it overlaps), the images
 * are uploaded in order
 * on a second stream while the chunks whose images (and, for video volumes,
 * neighbouring frames) are resident are concealed on `cuda_stream`, and each
 * chunk's patches are read back on a third stream once its launch ends.
 * Blocks listed in image order give the most overlap; any order gives the
 * same patches, bit for bit.
 */
fse_status fse_extrapolate_batch_host(fse_handle *h, const void *images, int dtype,
                                      int n_images, int height, int width, size_t pitch_bytes,
                                      const uint8_t *loss_mask, const fse_block *blocks,
                                      int n_blocks, float *patches, void *cuda_stream);

/*
 * Copy the selection trace of the last batch (FSE_FLAG_TRACE only) to host
 * memory, synchronising the handle's last stream first.  For block i (order
 * of `blocks`) and iteration nu < I of its class, entry i * stride + nu holds
 *   sel    linear index u * F + v of the selected bin,
 *   energy |R_w[u,v]|^2 (FP32) at selection,
 *   coef   c-hat as (re, im).
 * stride is written to *stride_out (the maximum I over the classes).  Each
 * output pointer may be NULL (all NULL = query the stride only); cap is the
 * number of entries each non-NULL array holds and must be >= n_blocks * stride.
 */
fse_status fse_get_trace(fse_handle *h, int32_t *sel, float *energy, float *coef,
                         size_t cap, int *stride_out);

/* The top-two gap of every selection of the last batch (FSE_FLAG_TRACE
 * only), in the layout of fse_get_trace: (e1 - e2) / e1, e1 the selected
 * bin's FP32 energy |R_w[u,v]|^2 and e2 the largest FP32 energy of the other
 * bins at that selection (0 where e1 = 0).  It tells how close each pick was
 * to a tie in the kernel's own precision: Section III selects the maximum,
 * and a pick whose gap is below the arithmetic's resolution could have gone
 * to the runner-up.  cap as fse_get_trace.  Synchronises the last stream. */
fse_status fse_get_trace_gap(fse_handle *h, float *gap2, size_t cap);

/* The model over every lost block's whole extrapolation area, for the last
 * batch of a handle created with FSE_FLAG_TRACE: Re{g}[m][n] for the M x M
 * area, the inverse transform of the accumulated model spectrum G of
 * Algorithm 1 (Section III: the model g is defined on the whole area L)
 * evaluated at the area's positions in the F x F grid.  Only the model: a
 * warm start's estimate is not added.  model: device, block i (caller order)
 * at model + i * model_stride, row-major, model_stride >= the largest M * M.
 * Enqueued on cuda_stream (after the last launch's stream has finished when
 * the two differ); the B samples equal the concealed output bit for bit.
 * Errors: FSE_ERR_INVALID_ARG (no trace flag, NULL model, short stride). */
fse_status fse_get_area_model(fse_handle *h, float *model, size_t model_stride, void *cuda_stream);

/* Wait for the handle's last launch and report what the kernels recorded on
 * the device (no counterpart in the paper), then clear the record:
 *   FSE_ERR_TIMEOUT      a bounded device wait ran out: the TMA gather of a
 *                        window, an ordered block's wait for the blocks it
 *                        reuses, or the learned-initialisation network's wait
 *                        for its tensor-core work.  The kernel records it,
 *                        waits at most 1 s more for its own copies or MMAs in
 *                        flight, frees its tensor memory and carries on or
 *                        stops; the outputs of that launch are not valid.
 *   FSE_ERR_INVALID_ARG  a block's loss area B is not marked lost in the
 *                        loss mask (the blocks must be lost samples); that
 *                        block was concealed as if B were lost.
 *   FSE_ERR_CUDA         (bounds-checked library only) an index into a
 *                        shared-memory spectrum, the output image or the
 *                        block list left its buffer; the kernel skipped the
 *                        access (or the block) and carried on.
 * The handle stays usable after any of them.
 * The library is also built bounds-checked (libfse_checked.so, compiled with
 * FSE_BOUNDS_CHECK; the Python binding loads it when the environment sets
 * FSE_BOUNDS_CHECK=1): same interface and results, with the kernels' W-chunk
 * loads and stores, output stores and block descriptors checked against
 * their buffers.  It stands in for a memory checker where none can run. */
fse_status fse_sync(fse_handle *h);

/* Limit of every bounded device wait of the handle's launches, in
 * nanoseconds of the GPU's global timer (default 1e9 = 1 s, at most 60 s).
 * 0 lets a wait expire as soon as its first poll fails, which tests use to
 * exercise the timeout path.  Takes effect from the next call (a captured
 * launch is re-captured).  No counterpart in the paper. */
fse_status fse_set_wait_limit(fse_handle *h, unsigned long long ns);

/* How the handle chooses the launch shape (threads per CTA: 128 or 256, CTAs
 * per SM: the two largest counts) of a class mix it has not seen (no
 * counterpart in the paper).  Every shape gives the same outputs bit for
 * bit; only the speed differs.
 *   FSE_TUNE_SYNC  (default) the first call with the mix times the four
 *                  shapes on the batch itself (two launches each) and waits
 *                  for them before it enqueues its own launch;
 *   FSE_TUNE_ASYNC no call waits: each call with an untuned mix runs its own
 *                  launch with the next untimed shape, bracketed by events
 *                  that later calls poll without blocking; once all four
 *                  are timed the fastest is kept (so the first four or five
 *                  calls run at the candidates' speeds, and re-plan instead
 *                  of replaying a captured launch);
 *   FSE_TUNE_OFF   128 threads per CTA at the largest CTA count, untimed.
 * Measured choices (SYNC, ASYNC) go to the process-wide cache that other
 * handles read; choices the handle already holds are kept.
 * fse_get_tuning reports the mode and how many class mixes are still being
 * timed asynchronously (either pointer may be NULL). */
#define FSE_TUNE_SYNC 0
#define FSE_TUNE_ASYNC 1
#define FSE_TUNE_OFF 2
fse_status fse_set_tuning(fse_handle *h, int mode);
fse_status fse_get_tuning(const fse_handle *h, int *mode, int *pending);

/* ------------------------------------------------------------------------
 * Learned initialisation network (no counterpart in the paper).
 *
 * A small CNN estimates the whole extrapolation area from its support so
 * that Algorithm 1 can start from the residual (fse_config.init =
 * FSE_INIT_LEARNED).  Four 3x3 convolutions with "same" zero padding and
 * dilations 1, 2, 4, 8, channels 2 -> 32 -> 32 -> 32 -> 1, ReLU after the
 * first three; bfloat16 weights and activations, FP32 accumulation (tensor
 * cores); FP32 gradients; Adam (beta 0.9 / 0.999, eps 1e-8) on FP32 master
 * weights.  Input of one area (H x W, row-major, FP32): channel 0 = support
 * sample / 255 on the support area and 0 elsewhere, channel 1 = 1 on the
 * support area and 0 elsewhere.  Output: the estimate / 255.
 * Parameters: one flat FP32 vector, per layer W[co][ci][ky][kx] then b[co].
 * ------------------------------------------------------------------------ */
#define FSE_CNN_PARAMS 19393
typedef struct fse_cnn fse_cnn;

/* Number of parameters (FSE_CNN_PARAMS). */
size_t fse_cnn_param_count(void);

/* Network state for areas of height x width on `device`, with buffers for up
 * to max_batch areas per call; parameters start at zero. */
fse_status fse_cnn_create(fse_cnn **out, int device, int height, int width, int max_batch);

/* Copy n = FSE_CNN_PARAMS host FP32 parameters in (resets the Adam moments
 * and step count) or out.  Synchronous. */
fse_status fse_cnn_set_params(fse_cnn *c, const float *params, size_t n);
fse_status fse_cnn_get_params(fse_cnn *c, float *params, size_t n);

/* The whole training state, for checkpoints: the FP32 master parameters,
 * Adam's first and second moments (FSE_CNN_PARAMS host FP32 values each)
 * and the number of Adam steps taken (which sets the bias corrections).
 * Setting it and training on continues bit for bit where the state was
 * taken (the gradients are reduced in a fixed order).  Synchronous. */
fse_status fse_cnn_get_state(fse_cnn *c, float *params, float *m, float *v, long long *step);
fse_status fse_cnn_set_state(fse_cnn *c, const float *params, const float *m, const float *v,
                             long long step);

/* Inference on n areas: x device [n][2][H][W] FP32, y device [n][H][W] FP32.
 * Asynchronous on cuda_stream. */
fse_status fse_cnn_forward(fse_cnn *c, const float *x, int n, float *y, void *cuda_stream);

/* Mean weighted squared error L = sum lam (y - target)^2 / (n H W) and its
 * gradient with respect to every parameter.  target, lam: device [n][H][W]
 * (lam NULL = all ones).  grad_host (FSE_CNN_PARAMS floats) and loss_host may
 * be NULL.  Synchronises the stream. */
fse_status fse_cnn_loss_grad(fse_cnn *c, const float *x, const float *target, const float *lam, int n,
                             float *grad_host, float *loss_host, void *cuda_stream);

/* One Adam step with learning rate lr on the loss above.  loss_host (the loss
 * before the step) may be NULL, which keeps the call asynchronous. */
fse_status fse_cnn_train_step(fse_cnn *c, const float *x, const float *target, const float *lam, int n,
                              float lr, float *loss_host, void *cuda_stream);

/* Reason for the last failure on c (or of fse_cnn_create when c is NULL). */
const char *fse_cnn_last_error(const fse_cnn *c);

/* Free the network state.  NULL is a no-op. */
void fse_cnn_destroy(fse_cnn *c);

/*
 * Batch concealment that allocates nothing, for callers that may not call
 * cudaMalloc (the paper has no counterpart: this is a deployment variant).
 * Some programs cannot let a library allocate device memory once they run:
 * cudaMalloc / cudaFree can synchronise the whole device, which a real-time
 * video pipeline cannot afford; some applications give all device memory to
 * their own pool allocator at start-up; some certified or embedded processes
 * forbid allocation after initialisation.  This entry point needs no handle:
 * the work-queue head, bucketed block list and weight / twiddle tables live
 * in one fixed file-scope device array of about 3.1 MB that every GPU which
 * loads the library holds until the process exits.
 *   classes, n_classes   the size classes (as fse_config.cls), 1..4
 *   images, dtype, n_images, height, width, pitch_bytes, loss_mask
 *                        device buffers, as fse_extrapolate_batch
 *   blocks               HOST array of n_blocks descriptors, n_blocks <= 65536
 *                        (larger batches are rejected with
 *                        FSE_ERR_INVALID_ARG; split them)
 *   out                  device FP32 image; only B samples are written
 *   cuda_stream          stream to enqueue on; the current device is used
 * The first call on a device looks up the array's device address and the
 * kernel's occupancy (once per device); make that first call before any
 * stream capture.  That set-up belongs to the device's context: after
 * cudaDeviceReset on a device, do not call this entry point on it again in
 * the same process.  All calls on a device share the array and it keeps the
 * last call's contents: each call rewrites what it reads and zeroes the
 * queue head, but calls whose GPU work overlaps (other streams or threads)
 * race on it and must be serialised by the caller.  The block list is copied
 * to the device on the stream: from pageable host memory the call returns
 * once the list has been staged, from pinned (page-locked) memory the copy
 * is asynchronous and the array must stay valid and unchanged until the
 * stream has reached the call.  Errors: fse_last_error(NULL).
 */
fse_status fse_extrapolate_batch_noalloc(const fse_class *classes, int n_classes, const void *images,
                                         int dtype, int n_images, int height, int width,
                                         size_t pitch_bytes, const uint8_t *loss_mask,
                                         const fse_block *blocks, int n_blocks, float *out,
                                         void *cuda_stream);

/* Measurement helper (no counterpart in the paper): the shared-memory load
 * bandwidth of `device` in GB/s (1e9 bytes/s), measured as a stream of
 * conflict-free 16-byte shared-memory loads on every SM (one CTA of 1024
 * threads per SM), best of five event-timed launches.  This is the peak the
 * concealment kernel's iterations, which read one 16-byte W chunk per
 * register pair from shared memory, are reported against.  Synchronous;
 * allocates a few bytes of device memory.  Errors: fse_last_error(NULL). */
fse_status fse_measure_smem_bandwidth(int device, double *gbytes_per_s);

/* Test hooks for fault injection (no counterpart in the paper).
 * fse_test_fail_allocation(n): the n-th device or pinned-host allocation the
 * library makes from now on fails as if memory were exhausted (the call that
 * made it returns FSE_ERR_OOM); n = 0 disarms.  Process-wide.
 * fse_test_live_allocations(): device and pinned-host allocations the
 * library holds now (handles, networks, staging), to check for leaks. */
void fse_test_fail_allocation(int n);
long long fse_test_live_allocations(void);
/* Forgets the process-wide tuning cache (every handle's own choices stay),
 * so a test can watch a class mix being tuned again. */
void fse_test_clear_tuning_cache(void);

/* Reason for the last failure on h (or, when h is NULL, of fse_create or
 * fse_extrapolate_batch_noalloc); never NULL; valid until the next call. */
const char *fse_last_error(const fse_handle *h);

/* Free everything the handle owns (synchronises its streams).  NULL is a no-op. */
void fse_destroy(fse_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* FSE_H */
