/*
 * pa_hodmas.h -- C ABI of the GB300 (sm_103a) higher-order delay-multiply-
 * and-sum photoacoustic beamformer.
 *
 * Method: Mulani, Paul, Singh, "Higher-order correlation based real-time
 * beamforming in photoacoustic imaging" (arXiv 2203.14906).
 *   - DAS                         Eq. 1   (Section 2.1)
 *   - DMAS, real-time O(N) form   Eqs. 2, 3 (Section 2.2)
 *   - DMAS-k, k = 3, 4, 5         Eqs. 4-6, O(N) forms Eqs. 7-9
 *                                 (Section 2.3); any k <= 8 by the same
 *                                 Newton-identity recursion (Section 6 notes
 *                                 higher orders are possible)
 *   - band-pass, Hilbert envelope, log compression   (Section 3)
 *   - delays precomputed into GPU global memory        (Section 5)
 *
 * Conventions the paper leaves open (stated once here, used everywhere):
 *   geometry  element i at x_i = (i - (N-1)/2) * pitch, z = 0; pixel (j, l)
 *             centre x = x0 + (j + 1/2)(x1 - x0)/nx, z = z0 + (l + 1/2)(z1 - z0)/nz
 *   delay     one-way time of flight, tau = fs (r / c - t0) samples
 *   sample    linear interpolation s = r[n] + a (r[n+1] - r[n]), n = floor(tau);
 *             s = 0 when n < 0 or n + 1 > Ns - 1 (the channel drops out)
 *   apodise   f_number > 0: element active iff |x_i - x| <= z / (2F),
 *             weight cos^2(pi (x_i - x) F / z), applied to s before the root
 *   root      x_i = sgn(s_i) |s_i|^(1/k) (signed even roots as in Eqs. 2, 5;
 *             real odd roots as in Eqs. 4, 6)
 *   combine   e_k of the x_i by Newton's identities from power sums, in FP64
 *             (for k = 4, 5 the term p2^2 - 2 p4 enters as one FP32 value
 *             formed with an error-free square, as DMAS is)
 *   post      per depth column: zero-pad to M = 2^ceil(log2 nz), FFT, multiply
 *             by a raised-cosine band (f0 +- f0/2 for DAS and odd orders,
 *             2 f0 +- f0/2 for even orders, roll-off f0/4, clipped at the
 *             axial Nyquist c / (2 dz)) times the analytic-signal mask,
 *             inverse FFT, modulus; log = 20 log10(env / image max),
 *             clipped to [-dyn_range_db, 0].
 *
 * Threading: a plan is not thread-safe; use one plan per host thread or
 * lock around it.  Functions never throw; failures return a status and
 * pa_last_error() gives a thread-local message.
 */
#ifndef PA_HODMAS_H
#define PA_HODMAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PA_OK = 0,
  PA_EINVAL = 1,        /* bad argument: sizes, order, null pointer       */
  PA_ENOMEM = 2,        /* device allocation failed or budget exceeded    */
  PA_ECUDA = 3,         /* CUDA runtime error (pa_last_error has detail)  */
  PA_ETIMEOUT = 4,      /* a bounded wait ran out                         */
  PA_EUNSUPPORTED = 5,  /* valid request outside what the library handles */
  PA_EBUSY = 6          /* resource in use (e.g. server queue full)       */
} pa_status;

typedef enum { PA_RF_F32 = 0, PA_RF_BF16 = 1, PA_RF_F16 = 2 } pa_rf_dtype;

/* Sampling of the delayed signal.  LINEAR interpolates between the two
 * samples around the delay; NEAREST takes the sample at the rounded delay,
 * s_i[k + Delta_i] with an integer index exactly as Eq. 1 writes it (valid
 * iff 0 <= round(tau) <= Ns-1, rounding halves up). */
typedef enum { PA_INTERP_LINEAR = 0, PA_INTERP_NEAREST = 1 } pa_interp;

/* Form of the resident delay / apodisation table (Section 5 precomputes the
 * delay of every pixel and element into GPU memory).
 *   LATTICE  the delay depends on the pixel and the element only through
 *            their lateral offset and the depth; when the element pitch is
 *            an integer multiple m (1..32) of the lateral pixel pitch those
 *            offsets lie on a lattice of about nx + m N values, and one
 *            table row per lattice offset serves every pair on it (a few MB,
 *            resident in L2).
 *   FULL     one entry per pixel and element (nx x N x nz; 8 bytes, plus 4
 *            with apodisation): any lateral grid, finer or coarser than the
 *            pitch or incommensurate with it.
 *   AUTO     LATTICE when the grid allows it, else FULL.
 * Both forms hold the same FP64-computed delays, so images agree to FP32
 * rounding of the sums. */
typedef enum { PA_TABLE_AUTO = 0, PA_TABLE_LATTICE = 1, PA_TABLE_FULL = 2 } pa_delay_table;
/* Largest FULL table pa_plan builds (bytes). */
#define PA_FULL_TABLE_MAX_BYTES ((size_t)16 << 30)

/* Output images (bit mask).  Planes of one frame are ordered DAS, DMAS,
 * HODMAS, keeping only the requested ones. */
enum { PA_OUT_DAS = 1u, PA_OUT_DMAS = 2u, PA_OUT_HODMAS = 4u };
/* Stages written (bit mask), ordered RAW, ENV, LOG. */
enum { PA_STAGE_RAW = 1u, PA_STAGE_ENV = 2u, PA_STAGE_LOG = 4u };

/* Plan descriptor.  All lengths in metres, times in seconds. */
typedef struct {
  int32_t n_elem;        /* N >= 1 array elements                           */
  double pitch_m;        /* element pitch > 0                               */
  double c_m_s;          /* speed of sound > 0                              */
  double fs_hz;          /* RF sample rate > 0                              */
  double t0_s;           /* time of RF sample 0 after the laser shot        */
  int32_t n_samples;     /* Ns >= 2 samples per channel                     */
  int32_t nx, nz;        /* image grid >= 1                                 */
  double x0_m, x1_m;     /* lateral extent, x1 > x0 (any lateral pitch dx;
                            pitch / dx an integer 1..32 allows the lattice
                            delay table)                                    */
  double z0_m, z1_m;     /* depth extent, 0 <= z0 < z1                      */
  int32_t order_k;       /* 1..8; 1 = DAS only, 2 = DMAS                    */
  uint32_t outputs;      /* PA_OUT_* mask, non-zero                         */
  pa_rf_dtype rf_dtype;  /* RF storage type; arithmetic is FP32 regardless  */
  int32_t max_batch;     /* frames per launch; <= 0 means 1                 */
  double f_number;       /* 0 = full aperture; > 0 dynamic aperture + Hann  */
  double f0_hz;          /* pulse centre frequency (post-filter band)       */
  double band_lo_hz;     /* both > 0: explicit band for every output;
                            otherwise the order-dependent default band      */
  double band_hi_hz;     /* < 0: band-pass off (analytic mask only)         */
  double dyn_range_db;   /* log-compression range; <= 0 means 60 dB        */
  int32_t compensated;   /* 1: Kahan-compensated FP32 power sums (totals
                            and compensation terms kept in tensor memory) */
  pa_interp interp;      /* sampling of the delayed signal                  */
  pa_delay_table delay_table; /* table form; PA_TABLE_AUTO picks            */
} pa_plan_desc;

typedef struct pa_plan_s* pa_plan_t;

/* Read-only facts about a plan (for tests, benchmarks and admission). */
typedef struct {
  int32_t lattice_m;          /* pitch / lateral pixel pitch (lattice table;
                                 0 with the full table)                    */
  int32_t tile_x, tile_z;     /* pixel tile of one thread block            */
  int32_t window;             /* RF samples staged per channel per tile    */
  int32_t n_tiles;            /* tiles per frame                           */
  int32_t threads;            /* threads per beamforming block             */
  int32_t blocks_per_sm;      /* resident beamforming blocks per SM        */
  int32_t fft_size;           /* M                                         */
  int32_t n_outputs;          /* popcount(outputs)                         */
  uint32_t warnings;          /* bit k set: output plane k's band lies above
                                 the axial Nyquist rate (DC removal only)  */
  int64_t nominal_pairs;      /* nx * nz * N per frame                     */
  int64_t active_pairs;       /* pairs with non-zero apodisation weight    */
  int64_t executed_pairs;     /* pairs the kernel evaluates per frame      */
  size_t device_bytes;        /* device memory owned by the plan now       */
  int32_t tma_staging;        /* 1: RF windows staged by TMA boxes,
                                 0: by vectorised loads                   */
  uint32_t device_error_flags; /* bounds-check flags raised by device code
                                  since the plan was built (0 = none): 1, 2
                                  index checks (checked builds only), 8 a
                                  TMA wait that ran out (the kernel stopped
                                  early).  Reading it synchronises the
                                  device.                                  */
  int32_t chunk_steps;        /* channel steps staged per shared-memory
                                 chunk of the fused kernel                 */
  int32_t lane_rows;          /* depth rows per lane group of the fused
                                 kernel (32, 16 or 8; a warp covers
                                 32 / lane_rows neighbouring slots)        */
  int32_t tmem_columns;       /* tensor-memory columns each fused-kernel
                                 block allocates for the Kahan totals of
                                 compensated sums (0: plain sums); resident
                                 blocks per SM x tmem_columns <= 512       */
  int32_t delay_table;        /* PA_TABLE_LATTICE or PA_TABLE_FULL         */
  size_t table_bytes;         /* bytes of the delay (+ apodisation) table  */
  int32_t tmem_dense;         /* 1: a fused-kernel block holds more TMEM
                                 columns than its share of the SM's 512 by
                                 registers (blocks of <= 3 warps), so blocks
                                 of another compensated kernel on the same
                                 SM could wait for columns; the server never
                                 overlaps such a plan with another
                                 compensated batch                         */
} pa_plan_info;

/*
 * pa_plan -- validate the descriptor, build the resident delay /
 * apodisation table on the device (Section 5 computes every pixel/element
 * delay before the beamforming launch and keeps it in GPU global memory),
 * the per-tile RF
 * windows and the post-filter masks.  Work is issued on cuda_stream (a
 * cudaStream_t, NULL = legacy default stream) and the call synchronises it
 * once before returning.  On success *out owns all device memory it
 * allocated until pa_destroy.
 * Errors: PA_EINVAL (null pointer, sizes, order outside 1..8, N < k, z0 < 0,
 * PA_TABLE_LATTICE asked for a grid whose pitch / dx is not an integer in
 * 1..32), PA_EUNSUPPORTED (full table above PA_FULL_TABLE_MAX_BYTES, RF
 * window too large for shared memory), PA_ENOMEM, PA_ECUDA.
 * Environment, read here (for measurements and tests; results do not depend
 * on the first three): PA_STAGING=tma|loads picks the RF staging path (TMA
 * boxes need Ns to be a multiple of the window alignment), PA_CHUNK_STEPS=n
 * caps the channel steps per staged chunk, PA_LANE_ROWS=32|16|8 sets the
 * depth rows per lane group of the fused kernel.  In the checked build only
 * (device bounds checks, PA_CHECK_BOUNDS), PA_INJECT_TMA_SHORTFALL makes
 * every TMA chunk expect 16 bytes more than it receives, so each block's
 * bounded wait runs out (failure-detection tests); the release build ignores
 * it.  After a PA_ETIMEOUT that was not injected (a copy that never
 * arrived), copies may still be in flight into the stopped blocks' shared
 * memory: destroy the plan and treat the CUDA context as suspect.
 */
pa_status pa_plan(const pa_plan_desc* desc, void* cuda_stream, pa_plan_t* out);

/* Bytes of device memory a plan for desc holds, plus the RF and output
 * buffers of n_frames frames with all stages (for admission control). */
pa_status pa_plan_footprint(const pa_plan_desc* desc, int32_t n_frames,
                            size_t* bytes);

pa_status pa_plan_get_info(pa_plan_t plan, pa_plan_info* info);

/*
 * pa_beamform -- the hot path (Sections 2-3 and 5) on n_frames frames that
 * are already in device memory.
 *   rf_dev   [n_frames][N][Ns] RF, contiguous, in desc->rf_dtype; device
 *            pointer aligned to 16 bytes.  Caller-owned, read only.
 *   out_dev  [n_frames][n_stages][n_outputs][nx][nz] FP32, z fastest;
 *            n_stages = popcount(stages), n_outputs = popcount(outputs);
 *            device pointer aligned to 16 bytes.  Caller-owned.
 *   stages   PA_STAGE_* mask, non-zero.
 * Asynchronous on cuda_stream (no host synchronisation); RF and output
 * buffers must stay valid until the stream reaches this point.  Frames
 * beyond max_batch are processed in consecutive launches.  n_frames == 0
 * is a no-op.  Per-pixel channel order is fixed, so a frame's result does
 * not depend on which other frames share its launch.
 * Errors: PA_EINVAL (null plan / pointer, n_frames < 0, bad stages),
 * PA_ECUDA (launch failure; the stream may hold earlier work).
 */
pa_status pa_beamform(pa_plan_t plan, const void* rf_dev, int32_t n_frames,
                      float* out_dev, uint32_t stages, void* cuda_stream);

/*
 * pa_beamform_host -- same computation on HOST buffers (same layouts): the
 * call copies RF host->device, runs the hot path and copies the output
 * device->host, then synchronises cuda_stream, so out_host is complete on
 * return.  Copies overlap with compute across frames.  Pinned (page-locked)
 * host memory gives the full copy rate.  Device staging buffers are
 * allocated on first use and owned by the plan.
 * Frames are processed in chunks rotating over three device buffer sets and
 * streams; the launch sequence of a chunk starts after the previous chunk's
 * (neighbouring launches do not share the GPU), while uploads and downloads
 * overlap them.  The chunk schedule per (n_frames, stages) is tuned over the
 * first calls of that shape (pa_plan_host_schedule).  With both host buffers
 * pinned (and graph launch enabled, kernel timing off) the whole call is one
 * CUDA graph launched on cuda_stream: the plan keeps one per (n_frames,
 * stages, schedule), at most 64, and rewrites only its host addresses when
 * the caller's buffers change.
 * Errors: as pa_beamform, plus PA_ETIMEOUT when a thread block of the fused
 * kernel gave up waiting for its TMA staging copies (a bounded wait of about
 * a second; the block stops early, so the output is incomplete;
 * pa_plan_info.device_error_flags has bit 8 set) in this call, or in an
 * earlier launch of the plan that no call has reported yet.
 */
pa_status pa_beamform_host(pa_plan_t plan, const void* rf_host,
                           int32_t n_frames, float* out_host, uint32_t stages,
                           void* cuda_stream);

/*
 * Host-path chunk schedules.  pa_beamform_host splits its frames into chunks
 * (see the pipeline model below).  For each (n_frames, stages) the plan first
 * tries a few candidate schedules, each on two calls, timing every call on
 * the host, and then keeps the fastest; results are identical whatever the
 * schedule.  pa_plan_set_host_schedule fixes the schedule of one
 * (n_frames, stages) instead: chunks[0..n_chunks) are frame counts, each in
 * 1..max_batch, summing to n_frames (n_chunks = 0 returns that shape to
 * tuning).  pa_plan_host_schedule reports the schedule the next call of that
 * shape will use in chunks[0..*n_chunks) (max_chunks entries of room) and
 * *state: 1 still trying candidates, 2 tuned, 3 set by the caller.
 * Tuning: every candidate is timed once, then the three fastest once more;
 * a call that had to build a CUDA graph or grow the plan's staging buffers
 * is not counted, and its candidate runs again.
 * Errors: PA_EINVAL for null pointers, n_frames < 1, an invalid stages mask
 * or an invalid schedule, or too little room.
 */
pa_status pa_plan_set_host_schedule(pa_plan_t plan, int32_t n_frames, uint32_t stages,
                                    const int32_t* chunks, int32_t n_chunks);
pa_status pa_plan_host_schedule(pa_plan_t plan, int32_t n_frames, uint32_t stages,
                                int32_t* chunks, int32_t max_chunks, int32_t* n_chunks,
                                int32_t* state);

/*
 * Pipeline model of the host path (host logic; no GPU involved).  Per chunk
 * of f frames: an upload of f * upload_us, the launch sequence taking
 * f * kernel_us * ((1 - wave_share) + wave_share * ceil(w) / w) + launch_us
 * with w = f * items_per_frame / resident (the waves of the persistent fused
 * kernel; wave_share = 1 when every work item costs the same, less when
 * cheaper items fill the last wave), and a download of f * download_us.  Uploads,
 * launch sequences and downloads each run one at a time in chunk order; the
 * chunks rotate over n_sets buffer sets, and a chunk's upload waits for the
 * download that last used its set.  pa_pipe_time gives the makespan (us) of
 * a schedule; pa_pipe_schedule writes the schedule of least makespan among a
 * searched family (a short first chunk, equal middle chunks, a tail of
 * shrinking chunks; chunks of at most max_chunk frames) to
 * chunks[0..*n_chunks), max_chunks entries of room.  pa_beamform_host draws
 * its candidate schedules from it over a range of kernel_us, launch_us and
 * wave_share.
 * Errors: PA_EINVAL for null pointers, items_per_frame or resident < 1,
 * n_sets outside 1..8, chunks of < 1 frame, n_frames or max_chunk < 1, or
 * too little room.
 */
typedef struct pa_pipe_model {
  int32_t items_per_frame;  /* work items of the fused kernel per frame */
  int32_t resident;         /* thread blocks of the fused kernel resident at once */
  int32_t n_sets;           /* device buffer sets (streams), 1..8 */
  int32_t reserved;         /* 0 */
  double upload_us;         /* per frame */
  double kernel_us;         /* per frame, at whole waves */
  double download_us;       /* per frame */
  double launch_us;         /* per chunk */
  double wave_share;        /* share of kernel_us that runs in whole waves, 0..1 */
} pa_pipe_model;
pa_status pa_pipe_time(const pa_pipe_model* model, const int32_t* chunks, int32_t n_chunks,
                       double* us);
pa_status pa_pipe_schedule(const pa_pipe_model* model, int32_t n_frames, int32_t max_chunk,
                           int32_t* chunks, int32_t max_chunks, int32_t* n_chunks);

/*
 * Launch mode.  By default (enable = 1) each pa_beamform launch sequence
 * (clear, fused beamforming kernel, post-filter, log) runs as one CUDA graph;
 * the plan keeps one executable graph per (frames per launch, stages) and
 * only rewrites its buffer pointers on later calls.  enable = 0 launches the
 * kernels one by one.  Results are identical either way.  Kernel timing
 * (pa_plan_profile) works in both modes: in graph mode the timed launches
 * run a graph of their own with an event-record node before and after each
 * kernel.
 */
pa_status pa_plan_use_graph(pa_plan_t plan, int32_t enable);

/*
 * Kernel timing.  While enabled, every launch of the plan's kernels is
 * bracketed by CUDA events recorded on the stream it runs on (kernel kinds:
 * 0 fused beamforming, 1 post-filter/envelope, 2 log compression).
 * enable: 0 off, 1 every kernel, 2 the fused beamforming kernel only (each
 * timed kernel adds two event records, which stop the next launch from
 * overlapping the previous kernel's tail); other values: PA_EINVAL.
 * pa_plan_profile_read waits for the recorded events, returns the summed
 * milliseconds and launch counts per kind and clears them.
 */
pa_status pa_plan_profile(pa_plan_t plan, int32_t enable);
pa_status pa_plan_profile_read(pa_plan_t plan, double ms[3], int64_t launches[3]);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of beamforming requests (not in the paper;
 * it serves the paper's real-time use, Section 5, with many concurrent
 * frames of different geometries and orders).
 *
 * A server owns a scheduler thread, a plan-builder thread, a cache of
 * resident plans (delay tables stay on the device between requests) and
 * `slots` CUDA streams.  Each request brings one RF frame in host memory and
 * receives its output images in host memory.  Whenever a slot is free the
 * scheduler takes the oldest request that has arrived and whose plan is
 * resident, adds up to max_batch - 1 later arrivals with the same
 * descriptor, and runs them as one batch: RF copies, pa_beamform (kernel by
 * kernel), output copies, all on the slot's stream, so batches of different
 * requests overlap on the device.  A request with a new descriptor has its
 * plan built on the builder thread (its own stream) while other requests go
 * on; the plan's tables are admitted against the budget when the build
 * starts.  A batch is admitted only when its RF and output buffers fit in
 * device_budget_bytes next to what is in flight; otherwise it waits.  A
 * compensated plan whose blocks could hold more tensor memory than their
 * register share of an SM (pa_plan_info.tmem_dense) never runs together with
 * another compensated batch.  Frames are independent and each pixel's
 * arithmetic is fixed, so a result is the same whichever batch it ran in.
 * ---------------------------------------------------------------------- */
typedef struct pa_server_s* pa_server_t;

typedef struct {
  size_t device_budget_bytes; /* admission limit: plans + in-flight buffers   */
  int32_t slots;              /* concurrent batches (streams), >= 1           */
  int32_t max_batch;          /* frames per batch, >= 1                       */
  int32_t max_plans;          /* resident plans kept (least recently used
                                 idle plans are destroyed beyond this)        */
  uint32_t stages;            /* PA_STAGE_* written for every request         */
} pa_server_config;

typedef struct {
  uint64_t ticket;
  pa_status status;           /* PA_OK, or why the request failed            */
  double arrival_s;           /* request arrival, seconds on the server clock */
  double start_s;             /* its batch was issued                          */
  double done_s;              /* the scheduler saw its batch complete          */
  double latency_ms;          /* done_s - arrival_s                            */
  int32_t batch_frames;       /* frames in its batch                           */
  float device_ms;            /* device time of its batch's stream work, from
                                 before the RF upload to after the download
                                 (CUDA events); 0 if the batch failed          */
} pa_request_result;

typedef struct {
  uint64_t submitted, completed, failed, batches;
  size_t bytes_in_use, bytes_peak;   /* admission accounting                 */
  int32_t plans_resident;
} pa_server_stats;

/* Starts the scheduler thread on the current CUDA device.  The server clock
 * (seconds) starts at 0 here. */
pa_status pa_server_create(const pa_server_config* cfg, pa_server_t* out);
/* Current server-clock time in seconds. */
double pa_server_now(pa_server_t srv);
/*
 * Queue one frame.  rf_host: [N][Ns] in desc->rf_dtype; out_host: [n_stages]
 * [n_outputs][nx][nz] FP32; both stay caller-owned and must stay valid until
 * the request completes (pinned memory gives full copy speed).  arrival_s:
 * server-clock time at which the request becomes visible to the scheduler
 * (<= now: immediately; later values replay a recorded arrival trace).
 * desc->max_batch is ignored (the server's max_batch applies).
 * Errors: PA_EINVAL (descriptor or pointers), PA_ENOMEM (one frame alone
 * needs more than the budget).  The call never blocks on the device.  A
 * request whose batch hit a timed-out staging wait in the fused kernel
 * completes with status PA_ETIMEOUT.
 */
pa_status pa_server_submit(pa_server_t srv, const pa_plan_desc* desc, const void* rf_host,
                           float* out_host, double arrival_s, uint64_t* ticket);
/* Wait up to timeout_ms (< 0: forever) for a request; PA_ETIMEOUT if it is
 * still pending.  A finished request's result can be read once. */
pa_status pa_server_wait(pa_server_t srv, uint64_t ticket, int32_t timeout_ms,
                         pa_request_result* result);
pa_status pa_server_get_stats(pa_server_t srv, pa_server_stats* stats);
/* Waits for in-flight batches, stops the thread and frees every plan and
 * buffer.  Pending requests that never ran complete with PA_EBUSY. */
pa_status pa_server_destroy(pa_server_t srv);

/* ------------------------------------------------------------------------
 * Image-quality metrics of Section 3 on images already in device memory:
 * SNR (Eq. 10), CR (Eq. 11), gCNR (Eq. 12) and the lateral FWHM of a
 * target's main lobe.  Meant for envelope images (the ENV stage, linear
 * amplitude), which is what the paper's PA signal amplitudes are.
 *
 * Definitions (where the paper leaves a choice, the reading is stated):
 *   regions   a pixel belongs to a region when its centre
 *             (x0 + (j + 1/2) dx, z0 + (l + 1/2) dz) lies inside it, tested
 *             in FP64 without fused multiply-adds: RECT |x - xc| <= a and
 *             |z - zc| <= b; DISC d^2 <= a^2; ANNULUS a^2 < d^2 <= b^2,
 *             d^2 = (x - xc)^2 + (z - zc)^2 (a disc and an annulus with the
 *             same a partition the plane around the centre).
 *   mu_in, mu_out   means over the target / background pixels; sigma_out the
 *             background's population standard deviation (divides by n_out).
 *   snr_db = 20 log10(mu_in / sigma_out), cr_db = 20 log10(mu_in / mu_out).
 *   gcnr      1 - sum_b min(h_in[b], h_out[b]) over 256 bins of the
 *             normalised amplitude v / vmax, vmax the largest value in the
 *             two regions; bin = min(255, floor((v * 256) / vmax)) in FP32
 *             with an IEEE-rounded division (values <= 0, or vmax <= 0,
 *             fall in bin 0); h = bin count / region pixel count.
 *   fwhm_m    on the image row (fixed depth) of the target's maximum
 *             (first in x-major order on ties): walk left and right from it
 *             while the value stays >= max / 2; each side's crossing is
 *             linearly interpolated between the last pixel >= max / 2 and
 *             the first one below; fwhm = x_right - x_left.  NaN when a side
 *             reaches the image edge without crossing.
 *   Undefined quantities (an empty region, 0 / 0) are NaN or +-inf as IEEE
 *   arithmetic gives them; peak_j = peak_l = -1 for an empty target.
 * ---------------------------------------------------------------------- */
typedef enum { PA_REGION_RECT = 0, PA_REGION_DISC = 1, PA_REGION_ANNULUS = 2 } pa_region_shape;

typedef struct {
  int32_t shape;         /* pa_region_shape                                */
  double xc_m, zc_m;     /* centre                                         */
  double a_m, b_m;       /* RECT half-widths in x, z; DISC radius a;
                            ANNULUS inner radius a, outer radius b         */
} pa_region;

typedef struct {
  pa_region target;      /* "in" region of Eqs. 10-12                      */
  pa_region background;  /* "out" region                                   */
} pa_roi;

typedef struct {
  int32_t nx, nz;          /* image grid, the same as the plan's            */
  double x0_m, x1_m;
  double z0_m, z1_m;
} pa_grid;

typedef struct {
  double mu_in, mu_out, sigma_out;
  double snr_db, cr_db, gcnr, fwhm_m;
  double peak;             /* largest target value                         */
  int64_t n_in, n_out;     /* pixels in the target / background            */
  int32_t peak_j, peak_l;  /* where the target maximum is                  */
} pa_metrics;

#define PA_METRICS_MAX_ROIS 4096
/*
 * pa_image_metrics -- every ROI pair on every image.
 *   images_dev  [n_images][nx][nz] FP32, z fastest, device memory (e.g. the
 *               ENV planes of pa_beamform called with stages = PA_STAGE_ENV:
 *               n_images = frames x outputs).  Caller-owned, read only.
 *   rois        host array of n_roi pairs (1 <= n_roi <= PA_METRICS_MAX_ROIS),
 *               read before the call returns.
 *   out_dev     [n_images][n_roi] pa_metrics in device memory, caller-owned.
 * Asynchronous on cuda_stream; its scratch memory is taken from and given
 * back to the device's default memory pool in stream order.  The result is
 * deterministic (fixed reduction order).  n_images == 0 is a no-op.
 * Errors: PA_EINVAL (null pointers, bad grid, n_roi out of range, unknown
 * region shape, negative extents), PA_ENOMEM, PA_ECUDA.
 */
pa_status pa_image_metrics(const pa_grid* grid, const float* images_dev, int32_t n_images,
                           const pa_roi* rois, int32_t n_roi, pa_metrics* out_dev,
                           void* cuda_stream);

/* Frees everything the plan owns after synchronising the streams it used.
 * NULL is accepted (no-op). */
pa_status pa_destroy(pa_plan_t plan);

/*
 * pa_log_compress_noalloc -- log compression (20 log10(env / image max),
 * clipped to [-dyn_range_db, 0]; -dyn_range_db where env or the max is 0)
 * of n_images envelope images that allocates no memory.  The paper has no
 * counterpart: this is a deployment variant of the log stage for callers
 * that cannot call cudaMalloc once streaming (e.g. a real-time acquisition
 * loop that must not stall the device, or a host framework that owns all
 * device memory); it needs no plan.
 *   env_dev   [n_images][image_elems] FP32 envelopes (>= 0; negative values
 *             count as 0), device memory, caller-owned, read only.
 *   log_dev   [n_images][image_elems] FP32 output, caller-owned; may equal
 *             env_dev (in place).
 *   dyn_range_db  clipping range in dB; not positive (or NaN) means 60 dB,
 *             as in pa_plan_desc.
 * The per-image maxima live in a fixed device array of PA_NOALLOC_MAX_IMAGES
 * ints inside this library (16 KiB held on every GPU that loads it until the
 * process exits); n_images > PA_NOALLOC_MAX_IMAGES returns PA_EINVAL.  The
 * first call on a device looks up that array's device address (once per
 * device and CUDA context: a new context on the device, e.g. after
 * cudaDeviceReset, is looked up again on its first call), so make the first
 * call before any stream capture.  Every call
 * reuses the same array and clears the slots it needs on cuda_stream before
 * use: calls whose work overlaps on the GPU (other streams, other threads)
 * race on it and must be serialised by the caller.  Asynchronous on
 * cuda_stream.  No cudaMalloc, cudaFree or allocating library call is made.
 * Errors: PA_EINVAL (sizes, null buffer), PA_ECUDA; pa_last_error() has the
 * detail.
 */
#define PA_NOALLOC_MAX_IMAGES 4096
pa_status pa_log_compress_noalloc(const float* env_dev, int32_t n_images,
                                  int64_t image_elems, float dyn_range_db,
                                  float* log_dev, void* cuda_stream);

/*
 * pa_lanes_raw -- the other thread mapping of the fused pass, kept for
 * measurement (not the product path): channels on lanes, lanes_per_pixel
 * (4, 8 or 32) lanes per pixel, each lane's DAS / DMAS / DMAS-3 sums added
 * across the pixel's lanes by warp shuffles before the epilogue (Eq. 3,
 * Eq. 7).  Writes the RAW planes of n_frames frames (layout of pa_beamform
 * with stages = PA_STAGE_RAW) for a plan in the plain FP32 lattice form at
 * k = 3 (else PA_EUNSUPPORTED); n_frames <= the plan's max_batch.  Results
 * agree with pa_beamform's RAW planes to FP32 rounding (channel sums are
 * added in another order).  Asynchronous on cuda_stream.
 */
pa_status pa_lanes_raw(pa_plan_t plan, const void* rf_dev, int32_t n_frames, float* out_dev,
                       int32_t lanes_per_pixel, void* cuda_stream);

const char* pa_status_str(pa_status status);
/* Thread-local description of the last failure on this thread ("" if none). */
const char* pa_last_error(void);
/* ABI version (major * 100 + minor). */
int32_t pa_version(void);  /* 105: kernel timing inside CUDA graphs, fused-kernel-only mode */

#ifdef __cplusplus
}
#endif
#endif /* PA_HODMAS_H */
