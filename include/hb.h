/*
 * hb.h -- C ABI of the GB300 haemoglobin estimator (libhb.so).
 *
 * The method ("Fast Estimation of Haemoglobin Concentration in Tissue Via
 * Wavelet Decomposition", Section 2) turns one RGB frame into oxy- and
 * deoxy-haemoglobin concentration maps:
 *   1. log-attenuation y = -ln(max(I, eps)) of every channel (Eq. 8's -log);
 *   2. n levels of the 2x2-window Haar transform (Eq. 1-2);
 *   3. the Tikhonov operator M = (A^T A + gamma I)^-1 A^T on every directional
 *      (detail) coefficient, 3 colour values in, 2 concentrations out (Eq. 5);
 *   4. a Bayesian estimate on the low-pass band: the posterior mean of
 *      c = (HbO2, Hb) over a discretised concentration grid with a flat prior
 *      and Gaussian likelihood exp(-|ybar - A c|^2 / (2 sigma^2));
 *   5. the inverse transform (Eq. 4, H = H*);
 *   6. THb = HbO2 + Hb and SO2 = HbO2 / THb (Section 3, Fig. 1-2).
 *
 * Conventions for every entry point:
 *   - every function returns hb_status; nothing throws across the ABI;
 *   - "_dev" pointers are CUDA device pointers on the device current when the
 *     context was created; "_host" pointers are host memory (pinned is faster);
 *   - the caller owns every frame and output buffer; the context owns the
 *     operator, the grid constants, its scratch and its own streams/events;
 *   - work is enqueued on the caller's stream (a cudaStream_t passed as void*,
 *     NULL = legacy default stream) and is asynchronous: a fault inside a
 *     kernel surfaces as HB_ERR_CUDA from a later call or synchronisation;
 *   - a context is not thread-safe and its scratch is shared by all calls made
 *     with it: calls with the same context must not overlap on different
 *     streams;
 *   - the host side of the calls is marked with NVTX ranges (hb_estimate,
 *     hb_estimate_host, hb_estimate_host_async, and hb.frame, hb.analysis,
 *     hb.lowpass, hb.synthesis around each launch; hb_serve.batch around each
 *     serving batch's enqueue), which cost nothing unless a profiler is attached.
 */
#ifndef HB_H
#define HB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hb_ctx hb_ctx;

typedef enum {
    HB_OK = 0,
    HB_ERR_ARG = 1,     /* NULL pointer, bad enum, misaligned or too-small stride */
    HB_ERR_SHAPE = 2,   /* non-positive size, levels outside 0..6, grid < 1 node */
    HB_ERR_CUDA = 3,    /* a CUDA runtime call or kernel launch failed */
    HB_ERR_OOM = 4,     /* device or pinned-host allocation failed */
    HB_ERR_BUDGET = 5,  /* admission refused: the request does not fit the memory budget */
    HB_ERR_TIMEOUT = 6, /* a bounded wait ran out */
    HB_ERR_STATE = 7,   /* call not valid in the object's current state */
    HB_ERR_IO = 8       /* a file could not be read or written, or is not of the expected kind */
} hb_status;

/* Mixing model: A[c][j] is the attenuation of colour channel c (R, G, B) per
 * unit concentration (uM) of chromophore j (HbO2, Hb), so y = A c for a
 * noiseless pixel (Beer-Lambert, Section 2). */
typedef struct {
    double A[3][2];
} hb_mixing;

/* Concentration grid of the Bayesian low-pass estimate: n0 x n1 nodes, inclusive
 * linear spacing c0 = lo0 + i (hi0 - lo0) / (n0 - 1), c1 = lo1 + j (hi1 - lo1) / (n1 - 1)
 * (a single node sits at lo when n = 1); sigma_l is the likelihood standard
 * deviation in log-attenuation units. */
typedef struct {
    int n0, n1;
    double lo0, hi0, lo1, hi1;
    double sigma_l;
} hb_grid;

/* Input pixel formats: interleaved RGB, channel fastest, rows row_stride_bytes apart. */
enum {
    HB_IN_F32_HWC = 0, /* float intensities; eps = 1e-6 */
    HB_IN_U8_HWC = 1   /* 8-bit codes k meaning k / 255; eps = 1 / 255 */
};

/* Flags of hb_create. */
enum {
    HB_LAMBDA_ABSOLUTE = 1u << 0,  /* gamma = lambda; default gamma = lambda * trace(A^T A) / 2 */
    HB_LOWPASS_TIKHONOV = 1u << 1, /* low pass through M as well (the all-Tikhonov comparison) */
    HB_FULL_GRID = 1u << 2,        /* posterior enumerates every grid node; by default, per low-pass
                                      pixel, only the nodes within 2^-(30 + log2(n0 n1)) of the reference
                                      node's weight (which is exactly 1) are, so that the nodes left out
                                      carry together less than 2^-30 of the posterior mass */
    HB_ILLUMINATION = 1u << 5,     /* the constant term of Eq. 8 (global illumination): the Tikhonov
                                      operator solves over xi = [A | 1] and keeps the HbO2 and Hb rows;
                                      the posterior integrates a per-pixel offset kappa (1,1,1) out
                                      under a flat prior.  Not with the learned low pass. */
    HB_LOWPASS_INTENSITY = 1u << 6, /* Eq. 3-8 literally for the low pass: the posterior sees
                                      -log(block mean of the intensities) instead of the block mean of
                                      -log I (directional bands unchanged).  Levels 0..4; not with
                                      HB_LOWPASS_TIKHONOV nor the learned low pass. */
    HB_LOWPASS_LS = 1u << 7,        /* the low pass by least squares instead of the posterior: the fit
                                      of the maximisation step in Section 2 (Eq. 9, read as the ordinary
                                      least-squares solution), c = (xi^T xi)^-1 xi^T ybar with xi = A, or
                                      [A | 1] with HB_ILLUMINATION, on the low pass of -log I or, with
                                      HB_LOWPASS_INTENSITY, -log of the block mean of I; directional
                                      bands through M as always.  Not with HB_LOWPASS_TIKHONOV nor the
                                      learned low pass. */
    HB_NODE_SUMS = 1u << 8          /* the posterior's grid rows summed node by node (an exact ratio
                                      recurrence of the weights along the row) instead of in closed
                                      form.  By default a row is summed in closed form wherever the grid
                                      allows it: over all integer columns a row's weights are a sampled
                                      Gaussian whose sum and mean column follow from its peak (Poisson
                                      summation, error below 2e-13 relative where used), and a row the
                                      box edge cuts off on one side takes the one-sided sum from a table
                                      of FP64 sums built at hb_create (cubic pieces, checked there);
                                      both agree with the node-by-node sums far inside the tolerance */
};

/* Per-stage timing slots reported by hb_timing_read. */
/* HB_STAGE_FRAME: the single-pass frame kernel (all steps in one launch: the default for the
 * plain posterior at 1..3 levels where the rows are summed in closed form). */
enum { HB_STAGE_ANALYSIS = 0, HB_STAGE_LOWPASS = 1, HB_STAGE_SYNTHESIS = 2, HB_STAGE_FRAME = 3, HB_NUM_STAGES = 4 };

/* Create a context for frames of width x height pixels.
 *   mix, grid  : copied; grid must have n0, n1 >= 1, hi >= lo, sigma_l > 0.
 *   levels     : Haar levels n, 0..6.  0 = no decomposition (Bayesian estimate on
 *                every pixel, the full-resolution comparison).  Sizes that are not
 *                multiples of 2^n are edge-replicated internally and cropped on output.
 *   lambda     : Tikhonov constant (Eq. 5, Gamma = gamma I); see HB_LAMBDA_ABSOLUTE.
 *   in_format  : HB_IN_F32_HWC or HB_IN_U8_HWC.
 * Precomputes M, the grid constants and the log table in FP64 on the host,
 * uploads them and allocates the context's scratch (the low-pass band and its
 * concentration estimate).  *out is NULL on failure. */
hb_status hb_create(const hb_mixing *mix, const hb_grid *grid, int levels, double lambda, int width, int height,
                    int in_format, unsigned flags, hb_ctx **out);

/* Release the context and everything it owns; NULL is a no-op.  Synchronises
 * the device work the context enqueued. */
void hb_destroy(hb_ctx *ctx);

/* One frame -> THb and SO2 maps (the proposed method, steps 1-6).
 *   frame_dev        : height rows of width*3 values (u8 or f32 per in_format),
 *                      row_stride_bytes apart (>= width*3*element size).
 *   thb_dev, so2_dev : height*width floats each, row-major, contiguous.  THb in
 *                      the units of 1/A (uM); SO2 as a fraction, 0 where THb <= 0.
 * Asynchronous on `stream`.  With the plain posterior at 1-3 levels and a grid whose
 * rows are summed in closed form, the frame is one kernel launch (every step of a
 * strip of the frame in one warp); otherwise two or three launches (HB_NODE_SUMS: low
 * pass and synthesis; other configurations: analysis, posterior, synthesis).  The
 * first launch may start, under programmatic dependent launch, before the kernel ahead
 * of it on `stream` has finished: it waits for that kernel before reading the frame. */
hb_status hb_estimate(hb_ctx *ctx, const void *frame_dev, size_t row_stride_bytes, float *thb_dev, float *so2_dev,
                      void *stream);

/* Same computation on host buffers: copies the frame host->device, runs
 * hb_estimate into context-owned device buffers, copies THb and SO2
 * device->host, and synchronises `stream` before returning.  The frame is taken in
 * bands of whole 2^n-row superblock bands (a band's pixels depend on no other band), so
 * a band's input copy, its kernels (on `stream` and a context-owned stream, alternately)
 * and the previous band's output copy overlap; the copies use two more context-owned
 * streams.  Results equal hb_estimate's.
 * Pinned host buffers let the copies run asynchronously.  A second call with the same
 * buffers and the same (non-default) stream captures the sequence as a CUDA graph, which
 * later calls with those buffers replay; other buffers or stage timing run it directly. */
hb_status hb_estimate_host(hb_ctx *ctx, const void *frame_host, size_t row_stride_bytes, float *thb_host,
                           float *so2_host, void *stream);

/* hb_estimate_host without the final synchronisation, for streams of frames: the call
 * queues the copies and kernels and returns; THb and SO2 are in the host buffers once
 * `stream` has reached the point of the call (cudaStreamSynchronize or an event on it).
 * Successive calls overlap: the context alternates two staging sets, so one frame's input
 * copy and kernels run while the previous frame's results are copied back.  Nothing waits
 * for work queued on `stream` before the call, so the host frame must be complete when the
 * call is made, and it and the output buffers must stay untouched until the stream has
 * passed the call.  Results equal hb_estimate_host's (the same bands and kernels).  Every
 * other call on the context that launches work or reads its device state (hb_estimate*,
 * hb_posterior_mean, hb_lowpass_*, hb_mlp_* except get_params, hb_set_lowpass_mode,
 * hb_timing_start) first waits for asynchronous calls still in flight.
 * Returns HB_ERR_STATE while per-stage timing is armed (hb_timing_start); otherwise as
 * hb_estimate_host. */
hb_status hb_estimate_host_async(hb_ctx *ctx, const void *frame_host, size_t row_stride_bytes, float *thb_host,
                                 float *so2_host, void *stream);

/* Intermediate results of the same pipeline, for testing.  Any output may be NULL.
 *   ybar_dev  : hl*wl*3 doubles, low-pass band divided by 2^n (block mean of y).
 *   conc_dev  : hl*wl*2 floats, concentration low-pass coefficients 2^n * estimate.
 *   hbo2_dev, hb_dev : height*width floats each.
 * hl = ceil(height / 2^n), wl = ceil(width / 2^n). */
hb_status hb_estimate_debug(hb_ctx *ctx, const void *frame_dev, size_t row_stride_bytes, double *ybar_dev,
                            float *conc_dev, float *hbo2_dev, float *hb_dev, void *stream);

/* The low-pass Bayesian step alone on caller-supplied block means: for each of
 * npix rows of ybar_dev (3 doubles each) writes the posterior mean (HbO2, Hb)
 * over the context's grid to conc_dev (2 floats each). */
hb_status hb_posterior_mean(hb_ctx *ctx, const double *ybar_dev, long npix, float *conc_dev, void *stream);

/* Low-pass band size of the context (hl, wl as above). */
hb_status hb_lowpass_shape(const hb_ctx *ctx, int *hl, int *wl);

/* Kernel launches the context has made since creation (all entry points). */
long hb_launch_count(const hb_ctx *ctx);

/* Optional per-stage timing with CUDA events recorded on the launch stream.
 * hb_timing_start(ctx, max_launches) arms up to max_launches event pairs and zeroes the
 * node counter; hb_timing_read synchronises them and writes, per stage (HB_STAGE_*), the
 * summed milliseconds and the number of timed launches, then disarms.
 * hb_timing_nodes (while armed, before hb_timing_read) synchronises the device and writes
 * the number of grid nodes the posterior launches since hb_timing_start enumerated
 * (rows x n1 per pixel; see HB_FULL_GRID), the work the posterior's roofline counts. */
hb_status hb_timing_start(hb_ctx *ctx, int max_launches);
hb_status hb_timing_read(hb_ctx *ctx, double ms[HB_NUM_STAGES], long launches[HB_NUM_STAGES]);
hb_status hb_timing_nodes(hb_ctx *ctx, unsigned long long *nodes);
/* Like hb_timing_nodes for the grid rows the posterior launches summed in closed form (see
 * HB_NODE_SUMS): rows[0] all of them, rows[1] those the box edge cuts off (one-sided sums from
 * the table).  Their nodes are not in hb_timing_nodes' count. */
hb_status hb_timing_rows(hb_ctx *ctx, unsigned long long rows[2]);

/* Static description of a status code. */
const char *hb_strerror(hb_status s);

/* ------------------------------------------------------------------------------------
 * Learned stand-in for the low-pass posterior (not part of the paper's method).
 * A 3 -> 64 -> 64 -> 2 multilayer perceptron with exact GELU, BF16 weights and hidden
 * activations (FP32 input) and FP32 accumulation maps a low-pass pixel's block-mean
 * log-attenuation to a correction, in posterior standard deviations, of a baseline: the
 * least-squares concentration moved by each edge of the grid box as the mean of the
 * Gaussian likelihood cut by that edge alone (inverse Mills ratio); it is trained on the
 * GPU on pairs produced by the posterior step.  The grid needs at least 2 nodes and an
 * extent on both axes (else hb_mlp_init and hb_mlp_set_params return HB_ERR_STATE).
 * Parameters (FP32 masters, HB_MLP_NPARAMS floats): W1[64][3], b1[64], W2[64][64]
 * (row = output unit), b2[64], W3[2][64], b3[2].
 * ------------------------------------------------------------------------------------ */
#define HB_MLP_NPARAMS 4546
enum { HB_MODE_BAYES = 0, HB_MODE_MLP = 1, HB_MODE_MLP_MEAN_GATE = 2 };

/* Random initialisation (Glorot-uniform from a seeded splitmix64 stream, biases 0)
 * and zeroed Adam state.  The input normalisation and the least-squares baseline are
 * fixed by the context's mixing matrix and grid box. */
hb_status hb_mlp_init(hb_ctx *ctx, unsigned seed);

/* Copy the FP32 master parameters in / out (host arrays of HB_MLP_NPARAMS floats);
 * set_params also refreshes the BF16 copies and zeroes the Adam state. */
hb_status hb_mlp_set_params(hb_ctx *ctx, const float *params_host);
hb_status hb_mlp_get_params(hb_ctx *ctx, float *params_host);

/* Save the network to a file: the FP32 master parameters (not the Adam state) and the
 * model they were trained for -- the mixing matrix, the grid box and sigma_l, which fix
 * the network's input transform, least-squares baseline and output scale.  Layout, all
 * little-endian: 8 bytes "HBMLPv1\n"; uint32 HB_MLP_NPARAMS; uint32 0; 11 doubles A[0][0],
 * A[0][1], A[1][0], ..., A[2][1], lo0, hi0, lo1, hi1, sigma_l; HB_MLP_NPARAMS floats in the
 * order of hb_mlp_set_params; uint32 FNV-1a hash of every preceding byte (18,292 bytes in
 * all).  HB_ERR_STATE if the context has no network; HB_ERR_IO if the file cannot be
 * written completely. */
hb_status hb_mlp_save(hb_ctx *ctx, const char *path);

/* Load a network written by hb_mlp_save, as hb_mlp_set_params would.  HB_ERR_IO if the
 * file cannot be read or is not such a file (length, header, parameter count, hash, or a
 * non-finite value); HB_ERR_STATE if it was trained for another mixing matrix, grid box
 * or sigma_l than the context's (compared exactly); the context is then unchanged. */
hb_status hb_mlp_load(hb_ctx *ctx, const char *path);

/* Training pairs from one frame: the block means of the low-pass band (npix x 3
 * floats) and the posterior means the exact step gives for them (npix x 2 floats, uM),
 * npix = hl * wl of the context. */
hb_status hb_lowpass_pairs(hb_ctx *ctx, const void *frame_dev, size_t row_stride_bytes, float *ybar_dev,
                           float *conc_dev, void *stream);

/* `steps` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on minibatches
 * of `batch` samples drawn with replacement from the n pairs (ybar_dev n x 3, target_dev
 * n x 2 posterior means in uM) by a hash of (seed, step, position).  loss_host, if not
 * NULL, receives the minibatch loss of every step (steps floats); the call then
 * synchronises `stream`.  batch <= 65536. */
hb_status hb_mlp_train(hb_ctx *ctx, const float *ybar_dev, const float *target_dev, long n, int steps, int batch,
                       double lr, unsigned seed, float *loss_host, void *stream);

/* Gradient of the mean loss over all n pairs (n <= 65536) with respect to the master
 * parameters (grad_dev: HB_MLP_NPARAMS floats) and the loss itself (loss_dev: 1 float);
 * the parameters are not changed. */
hb_status hb_mlp_gradient(hb_ctx *ctx, const float *ybar_dev, const float *target_dev, long n, float *grad_dev,
                          float *loss_dev, void *stream);

/* Network estimate of the posterior mean for n block means (conc_dev: n x 2 floats). */
hb_status hb_mlp_forward(hb_ctx *ctx, const float *ybar_dev, long n, float *conc_dev, void *stream);

/* Low-pass mode of hb_estimate.  HB_MODE_MLP: the network replaces the posterior; on
 * every frame the exact posterior is also evaluated on nsample seeded low-pass pixels
 * (1 <= nsample <= 2^24, else HB_ERR_ARG), and if the largest of their errors exceeds tol
 * -- a pixel's error being the larger of |dHbO2| / (hi0 - lo0) and |dHb| / (hi1 - lo1) --
 * or any is NaN, the whole low pass of that frame is recomputed exactly (all on the
 * device, no host round trip).  HB_MODE_MLP_MEAN_GATE: the same with the mean of the
 * sampled errors in place of the largest (a weaker guard, kept for comparison).  After
 * hb_mlp_certify, the pixels of cells the certification did not trust are computed by the
 * exact posterior in every frame (and count as error 0 in the check). */
hb_status hb_set_lowpass_mode(hb_ctx *ctx, int mode, double tol, int nsample);

/* Frames estimated in a learned mode, how many of them fell back to the exact posterior,
 * and (routed_pixels, may be NULL) how many low-pass pixels of the others the
 * certification's route sent to the exact posterior (synchronises the context's work). */
hb_status hb_lowpass_stats(hb_ctx *ctx, long *mlp_frames, long *fallbacks, long *routed_pixels);

/* Certify the current network against the exact posterior.  Over a 128 x 128 map of cells
 * of least-squares concentrations covering the grid box widened by 3 posterior standard
 * deviations on every side, the network and the exact posterior step are evaluated at
 * every cell corner and centre, each for three values (-1.5, 0, 1.5 sigma_l) of the
 * component of ybar outside the range of A; a cell is trusted when every one of its points
 * is within tol (error as in hb_set_lowpass_mode).  From then on the learned modes send
 * the low-pass pixels whose least-squares point falls in an untrusted cell, or outside the
 * map, to the exact posterior (one gated launch per frame).  Any change of the parameters
 * (init, set, load, train) ends the certification.  trusted_fraction (may be NULL)
 * receives the share of trusted cells.  Synchronises `stream`; allocates and frees
 * temporary device memory (a few MB). */
hb_status hb_mlp_certify(hb_ctx *ctx, double tol, double *trusted_fraction, void *stream);

/* ------------------------------------------------------------------------------------
 * Serving: continuous batching of frames from many concurrent streams (an extension; the
 * paper processes single frames).  A request-loop thread inside the library packs the
 * frames waiting from all streams -- any mix of sizes and of 0..4 levels -- into batches
 * that run as one launch per stage, four batches in flight on separate CUDA streams;
 * frames that arrive while a batch runs join the next one.  Each stream owns `slots`
 * frame slots (pinned host + device buffers) admitted against the server's budget.
 * The mixing model, grid and lambda are shared by all streams.
 * ------------------------------------------------------------------------------------ */
typedef struct hb_server hb_server;

/* One completed frame.  thb_host / so2_host (width*height floats each) stay valid until
 * hb_release(stream_id, slot); latency_ms runs from the hb_submit call to the moment the
 * results were in host memory. */
typedef struct {
    int stream_id;
    int slot;
    uint64_t tag;
    double latency_ms;
    const float *thb_host;
    const float *so2_host;
} hb_result;

typedef struct {
    long batches, frames, max_batch_frames, queued;
    double mean_batch_frames;
    size_t bytes_in_use, budget_bytes;
} hb_server_info;

enum { HB_SERVE_SEQUENTIAL = 1u << 4 }; /* one frame at a time, one batch in flight (baseline) */

/* Create a server.  flags: HB_LAMBDA_ABSOLUTE, HB_FULL_GRID, HB_ILLUMINATION, HB_LOWPASS_INTENSITY,
 * HB_SERVE_SEQUENTIAL.  budget_bytes bounds
 * the device memory of all stream slots plus the four batches' scratch (sized for
 * batch_lowpass_pixels low-pass pixels each); max_batch (1..64) bounds frames per batch.
 * HB_ERR_BUDGET if the scratch alone exceeds the budget.  Starts the request loop. */
hb_status hb_server_create(const hb_mixing *mix, const hb_grid *grid, double lambda, unsigned flags, int in_format,
                           size_t budget_bytes, int max_batch, long batch_lowpass_pixels, hb_server **out);

/* Stop the loop (frames not yet enqueued are dropped), wait for the GPU, free everything. */
void hb_server_destroy(hb_server *srv);

/* Admit a stream of width x height frames at `levels` (0..4) with `slots` frame slots.
 * HB_ERR_BUDGET when its slots do not fit the remaining budget (nothing is allocated);
 * HB_ERR_SHAPE when one frame's low pass exceeds a batch. */
hb_status hb_stream_open(hb_server *srv, int width, int height, int levels, int slots, int *stream_id);

/* Close a stream and return its memory to the budget.  HB_ERR_STATE while any of its
 * frames is being submitted, queued, running, or completed but not yet released. */
hb_status hb_stream_close(hb_server *srv, int stream_id);

/* Queue one frame (host memory, copied before the call returns) with a caller tag.
 * HB_ERR_STATE when all of the stream's slots are busy (poll, release and retry). */
hb_status hb_submit(hb_server *srv, int stream_id, const void *frame_host, size_t row_stride_bytes, uint64_t tag);

/* Up to max_results completed frames, waiting up to wait_us microseconds for the first.
 * Returns HB_ERR_CUDA (with any results) if a batch failed to launch. */
hb_status hb_poll(hb_server *srv, hb_result *out, int max_results, int *n_out, int wait_us);

/* Hand a completed slot back to its stream. */
hb_status hb_release(hb_server *srv, int stream_id, int slot);

/* Hold (paused != 0) or resume the start of new batches; frames keep queueing while held
 * and batches in flight finish.  Lets a caller release a burst of frames at once. */
hb_status hb_server_pause(hb_server *srv, int paused);

/* Block until every frame submitted so far has completed (is ready for hb_poll or
 * already polled), e.g. before hb_server_destroy or before a configuration change.
 * Waits at most timeout_ms milliseconds (0: only test) and then returns
 * HB_ERR_TIMEOUT, leaving every frame where it is; a paused server with queued
 * frames therefore times out.  Returns HB_ERR_CUDA if a batch failed since start. */
hb_status hb_server_drain(hb_server *srv, int timeout_ms);

/* Counters of the server so far. */
hb_status hb_server_stats(hb_server *srv, hb_server_info *out);

/* Measurement helper (the paper has no counterpart): the MUFU ex2 throughput of the
 * current device, the denominator of the grid posterior's roofline (one ex2 per grid node
 * it evaluates).  A throughput kernel fills every SM with independent ex2 chains and reads
 * the SMs' cycle counters around its loop, so the figure is in ex2 results per SM clock
 * per SM, independent of the clock frequency.  Synchronous (about a millisecond of GPU
 * time); allocates and frees a few KB of device memory.  Writes the SM count too. */
hb_status hb_measure_ex2_rate(double *ex2_per_clock_per_sm, int *sm_count);

/* Largest npix that hb_posterior_mean_static accepts. */
#define HB_STATIC_MAX_PIXELS 65536

/* The low-pass posterior step without any memory allocation.  The paper has no
 * counterpart to this entry point; it exists for callers that cannot call
 * cudaMalloc: real-time frame loops that may not block on the device allocator
 * (an allocation can synchronise the device and stall every stream), plug-ins
 * whose host application owns all device memory through its own pool, and
 * embedded deployments that must know their whole device footprint up front.
 *
 * Computes what hb_posterior_mean computes for a context created with HB_NODE_SUMS (any
 * lambda: the posterior does not use it) -- the posterior mean of (HbO2, Hb) for each
 * of npix rows of ybar_dev, 3 doubles each, written as 2 floats each to conc_dev, every
 * grid row summed node by node -- up to the order of FP32 additions, but takes the mixing
 * model and grid directly instead of a context.  A context created with flags 0 sums the
 * rows in closed form where the grid allows it; the two agree to a few FP32 roundings
 * (about 1e-5 relative).  The flags that change the posterior (HB_ILLUMINATION,
 * HB_FULL_GRID) have no counterpart here.  Its working memory is one fixed array
 * compiled into libhb.so (about 4.3 MiB per GPU, held from library load until process
 * exit).
 *   - npix > HB_STATIC_MAX_PIXELS returns HB_ERR_SHAPE and launches nothing;
 *     npix == 0 returns HB_OK; ybar_dev and conc_dev must be 8-byte aligned.
 *   - The first call on each device looks up that array's device address
 *     (cudaGetSymbolAddress, with the device current); make that first call
 *     before any stream capture starts.  The address is kept for the life of the
 *     process: after a cudaDeviceReset of a device this entry point must not be
 *     called on that device again.
 *   - Every call on a device shares the one array and leaves its contents
 *     behind; the call clears the part it needs before use.  Calls whose work
 *     overlaps on the GPU (different streams, or threads without ordering)
 *     race on the array and give wrong results: order them on one stream.
 *   - Asynchronous on `stream`, like the other entry points. */
hb_status hb_posterior_mean_static(const hb_mixing *mix, const hb_grid *grid, const double *ybar_dev, long npix,
                                   float *conc_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HB_H */
