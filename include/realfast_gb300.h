/*
 * realfast_gb300.h -- C ABI of the GB300 engine for the realfast transient
 * search hot path (Law et al. 2018, arXiv:1802.03084).
 *
 * The engine takes one segment of fast-sampled visibilities and, for every
 * DM trial, every boxcar width dt and every output integration t', forms a
 * Stokes-I dirty image by integer-sample dedispersion, boxcar resampling,
 * nearest-neighbour uv gridding and a 2D inverse FFT, and thresholds the
 * image peak against the image noise (Sec. 3.1 "Algorithm": a Stokes I image
 * per DM and time width, thresholded for point sources; Fig. 2: loops over
 * dispersion and sampling time).  The plan is the immutable "state" of
 * Sec. 3.2: it is fixed by the metadata (antenna positions, channels,
 * integration time) and the preferences (image size, DM and dt lists,
 * threshold), so any candidate can be reproduced from it.
 *
 * Conventions used by every entry point:
 *   - All pointers are plain host or device pointers; sizes are element
 *     counts unless stated.  No call keeps a pointer it was given after it
 *     returns, except the plan handle itself.
 *   - Every call returns an rf_status; no call aborts, prints or throws.
 *     On failure rf_last_error() gives a thread-local message.
 *   - A plan is used by one caller at a time: a call made while another call
 *     on the same plan is in progress returns RF_ERR_BUSY.
 *   - Device work is issued on the caller's CUDA stream (a cudaStream_t
 *     passed as void*; NULL means the legacy default stream).  Calls that
 *     return results on the host synchronise that stream before returning.
 */
#ifndef REALFAST_GB300_H
#define REALFAST_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rf_status {
  RF_OK = 0,
  RF_ERR_INVALID_ARG = 1, /* a NULL pointer, a size out of range, a bad flag */
  RF_ERR_NO_MEMORY = 2,   /* a device or host allocation failed            */
  RF_ERR_CUDA = 3,        /* a CUDA runtime error (message has the detail) */
  RF_ERR_SHAPE = 4,       /* nint out of range for the plan                */
  RF_ERR_CAPACITY = 5,    /* the caller's output array is too small        */
  RF_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up            */
  RF_ERR_BUSY = 7,        /* the plan is in use by another call            */
  RF_ERR_NO_DEVICE = 8    /* no usable CUDA device                         */
} rf_status;

/* ---- plan flags (rf_plan_desc.flags) ---------------------------------- */
/* Store the Stokes-I visibilities on the device as FP16 (round to nearest)
 * instead of FP32; dedispersion sums, gridding and FFT stay FP32.  The
 * boxcar sums over dt > 1 integrations are formed in FP32 and stored as
 * FP32, so only the visibilities themselves are rounded to FP16. */
#define RF_STORE_FP16 0x1u
/* PARTIAL edge rule: search t' < floor(nint/dt) for every DM; samples past
 * the end of the segment get weight 0.  Default (FULL): only t' whose whole
 * dispersed sweep lies in the segment, t' < floor((nint - max_c delay)/dt). */
#define RF_EDGE_PARTIAL 0x2u
/* Mean-visibility subtraction (Sec. 3.1): before dedispersion, every
 * (baseline, channel) loses its mean over the segment's nint integrations,
 * which removes sources that are constant over the segment.  The mean is
 * summed in FP64 over the stored Stokes-I values. */
#define RF_MEAN_SUBTRACT 0x4u
/* Clipped noise (Sec. 3.1 asks only for an S/N above a threshold; this is
 * the one-pass robust variant): with mu0 and sigma0 the mean and population
 * standard deviation of all N^2 pixels, mean and sigma are recomputed over
 * the pixels with |I - mu0| <= 5 sigma0.  The peak stays the maximum of all
 * pixels and snr = peak / sigma.  The search reads each image once as
 * without it (the kept-pixel sums are taken in the row FFT's registers,
 * around mu0 and sigma0 obtained from the grid by Parseval's identity). */
#define RF_NOISE_CLIPPED 0x8u
/* Build the host tables only; no device memory is touched.  Such a plan
 * answers the table queries (rf_plan_info, rf_plan_delays, rf_plan_cells,
 * rf_count_images) and rejects searches with RF_ERR_INVALID_ARG. */
#define RF_HOST_ONLY 0x100u

/* ---- search forms (rf_plan_set_form) --------------------------------- */
#define RF_FORM_BATCHED 0 /* all trials in waves of fused launches (a CUDA graph) */
#define RF_FORM_PLAIN 1   /* one unfused launch set per (DM, dt) trial     */

/*
 * Plan description.  Everything is copied by rf_plan_create; the caller keeps
 * ownership of the arrays.
 *
 * ant_uvw_m  [nant][3] antenna (u, v, w) in metres, row major.  Baseline b
 *            runs over antenna pairs (i, j), i < j, i outer, and has
 *            uvw_b = uvw_j - uvw_i (Sec. 2.2: N_bl = N_ant (N_ant - 1)/2).
 *            w is not used (w-term ignored).
 * freq_hz    [nchan] channel centre frequencies, any order; the highest is
 *            the dispersion reference f_top.
 * npol       1 or 2; with 2 the input is Stokes-I formed as the mean of the
 *            two polarisations (Sec. 3.1).
 * inttime_s  integration time in seconds (> 0).
 * npix       image side N, a power of two in [16, 8192].
 * cell_rad   pixel size in radians (> 0); the uv cell is 1/(N cell_rad).
 * dm_list    [ndm] dispersion measures in pc cm^-3, each >= 0.
 * dt_list    [ndt] boxcar widths in integrations, each in [1, 1024].
 * threshold_sigma  candidate threshold on peak / sigma (> 0).
 * flags      RF_STORE_FP16 | RF_EDGE_PARTIAL | RF_MEAN_SUBTRACT | RF_NOISE_CLIPPED |
 *            RF_HOST_ONLY.
 * max_nint   largest segment length (integrations) this plan will search;
 *            sizes the device buffers.
 * device     CUDA device ordinal the plan lives on.
 */
typedef struct rf_plan_desc {
  int32_t nant;
  const double* ant_uvw_m;
  int32_t nchan;
  const double* freq_hz;
  int32_t npol;
  double inttime_s;
  int32_t npix;
  double cell_rad;
  int32_t ndm;
  const double* dm_list;
  int32_t ndt;
  const int32_t* dt_list;
  double threshold_sigma;
  uint32_t flags;
  int32_t max_nint;
  int32_t device;
} rf_plan_desc;

/*
 * One candidate: the peak of the image of trial (dm_idx, dt_idx, t_idx)
 * whose peak / sigma reached the threshold (Sec. 3.1; at most one per image).
 * x, y     peak pixel; l_rad = (x - N/2) cell, m_rad = (y - N/2) cell.
 * peak     peak pixel value (units of the visibilities, a weighted mean).
 * sigma    population standard deviation of all N^2 pixels (of the kept
 *          pixels with RF_NOISE_CLIPPED).
 * snr      peak / sigma.
 * t_idx    output integration t' (start integration t' * dt at f_top).
 */
typedef struct rf_candidate {
  int32_t dm_idx;
  int32_t dt_idx;
  int32_t t_idx;
  int32_t x;
  int32_t y;
  float snr;
  float peak;
  float sigma;
  double dm;
  double l_rad;
  double m_rad;
} rf_candidate;

/* Statistics of one searched image (whether or not it became a candidate). */
typedef struct rf_image_stat {
  int32_t dm_idx;
  int32_t dt_idx;
  int32_t t_idx;
  int32_t x;
  int32_t y;
  float peak;
  float sigma;
  float snr;
  double mean;
  double weight; /* W: samples summed over on-grid (baseline, channel) */
} rf_image_stat;

/* Derived plan facts. */
typedef struct rf_plan_info {
  int32_t nbl;
  int32_t nchan;
  int32_t npix;
  int32_t ndm;
  int32_t ndt;
  int32_t iu_max;        /* largest |u| cell of an on-grid visibility      */
  int32_t iv_max;        /* largest |v| cell of an on-grid visibility      */
  int32_t n_offgrid;     /* (baseline, channel) pairs off the grid         */
  int32_t n_cells;       /* occupied cells of the half plane               */
  int32_t n_entries;     /* gridding entries (iu = 0 pairs count twice)    */
  int32_t max_delay;     /* largest delay in integrations over all trials  */
  int32_t images_per_group; /* consecutive t' imaged together              */
  uint64_t device_bytes; /* device memory held by the plan                 */
} rf_plan_info;

/*
 * rf_plan_create: validate `desc`, build the FP64 host tables (baselines,
 * delay table of Sec. 2.1's dispersion law rounded to integrations, nearest
 * uv cells), upload them and allocate the device buffers for segments of up
 * to max_nint integrations.  On success *out owns all device state.
 * Errors: RF_ERR_INVALID_ARG (bad desc; also a uv layout whose busiest
 * column, or whose number of columns, does not fit the imaging kernels' shared
 * memory at this npix: possible only for very large npix with many channels
 * on fine cells), RF_ERR_NO_DEVICE, RF_ERR_NO_MEMORY, RF_ERR_CUDA.  *out is set
 * to NULL on failure.
 */
rf_status rf_plan_create(const rf_plan_desc* desc, struct rf_plan** out);

/*
 * rf_plan_estimate_bytes: the device memory rf_plan_create(desc) would
 * allocate, with column-FFT scratch for `wave_images` images per wave
 * (0 = the default), without touching the device.  Used for admission by
 * memory.  Errors: as rf_plan_create's validation.
 */
rf_status rf_plan_estimate_bytes(const rf_plan_desc* desc, int64_t wave_images, uint64_t* bytes);

/* rf_plan_destroy: free everything the plan owns.  NULL is accepted.  The
 * caller must not have work in flight on the plan. */
rf_status rf_plan_destroy(struct rf_plan* plan);

/* Thread-local message for the last failing call on this thread ("" if none). */
const char* rf_last_error(void);

/*
 * rf_search_segment: search one segment (Sec. 3.1-3.2).
 * vis      [nint][nbl][nchan][npol] complex64 (interleaved float re, im),
 *          host memory (pinned or pageable) or device memory on the plan's
 *          device; the kind is detected.  Device memory and page-locked host
 *          memory the device can address (cudaHostAlloc, cudaHostRegister)
 *          are read in place by the ingest kernel, the latter over the
 *          host link; other host data is copied in chunks through a staging
 *          buffer.  Host data must stay unchanged until the call returns.
 * nint     integrations in the segment, 1 <= nint <= max_nint.
 * stream   cudaStream_t to run on (NULL = default stream).
 * out      host array of `cap` candidates; receives the candidates sorted by
 *          (dm_idx, dt_idx, t_idx).
 * n_out    receives the number of candidates.  If it exceeds cap, the first
 *          cap are written and RF_ERR_CAPACITY is returned.
 * Returns after the stream has finished the segment.
 * Errors: RF_ERR_INVALID_ARG, RF_ERR_SHAPE (nint out of range), RF_ERR_BUSY,
 * RF_ERR_CAPACITY, RF_ERR_CUDA, RF_ERR_TIMEOUT.
 */
rf_status rf_search_segment(struct rf_plan* plan, const void* vis, int32_t nint, void* stream,
                            rf_candidate* out, size_t cap, size_t* n_out);

/*
 * rf_search_segment_stats: as rf_search_segment, and also returns the
 * statistics of every searched image in (dm_idx, dt_idx, t_idx) order in the
 * host array `stats` of `stats_cap` entries (*n_stats = images searched).
 * Candidates go to `out` exactly as in rf_search_segment (out may be NULL
 * when cap is 0).  Meant for verification; it is slower than the search.
 */
rf_status rf_search_segment_stats(struct rf_plan* plan, const void* vis, int32_t nint, void* stream,
                                  rf_candidate* out, size_t cap, size_t* n_out,
                                  rf_image_stat* stats, size_t stats_cap, size_t* n_stats);

/*
 * rf_render_images: compute the full dirty images I[y][x] (float32, N x N,
 * row major, y = v axis) of `n` listed trials.  trials is a host array of n
 * triples (dm_idx, dt_idx, t_idx); images is a host array of n * N * N floats.
 * A trial outside the searched set (t_idx beyond the edge rule) or with
 * weight 0 is rejected with RF_ERR_INVALID_ARG.
 */
rf_status rf_render_images(struct rf_plan* plan, const void* vis, int32_t nint, void* stream,
                           const int32_t* trials, int32_t n, float* images);

/* Select the search form: RF_FORM_BATCHED (default) or RF_FORM_PLAIN. */
rf_status rf_plan_set_form(struct rf_plan* plan, int32_t form);

/*
 * Tuning knobs (used by the autotuner; results do not depend on them).
 * RF_TUNE_WAVE_IMAGES  images imaged per wave.  A wave's column-FFT
 *                      intermediate is images x (iu_max + 1) x npix x 8 bytes;
 *                      waves small enough to stay in L2 avoid an HBM round
 *                      trip.  Range [images_per_group, 32768].  Reallocates
 *                      the plan's scratch.
 * Errors: RF_ERR_INVALID_ARG (unknown key or value out of range),
 * RF_ERR_NO_MEMORY, RF_ERR_BUSY.
 */
#define RF_TUNE_WAVE_IMAGES 1
/* RF_TUNE_GRAPHS       1 (default): the batched form records its per-wave
 *                      launches once per segment length as a CUDA graph and
 *                      replays it; 0: direct launches. */
#define RF_TUNE_GRAPHS 2
/* RF_TUNE_WIDE_INDEX   0 (default): gridding addresses a resampled series
 *                      with 32-bit sample offsets whenever every index fits,
 *                      64-bit ones otherwise; 1: always 64-bit.  Both give
 *                      the same images; the knob lets a test run the 64-bit
 *                      variant on a small plan. */
#define RF_TUNE_WIDE_INDEX 3
/* RF_TUNE_FUSED        1: for npix 1024 .. 4096 the search runs
 *                      each wave's column and row FFTs as one persistent
 *                      launch whose column-FFT output passes through a small
 *                      ring of chunk slots (RF_TUNE_RING of them, each one
 *                      round of column transforms: 8 images at 1024^2, 4 at
 *                      2048^2, 2 at 4096^2) that stays in L2; 0 (default):
 *                      separate column and row launches through a wave-sized
 *                      buffer (always so for other sizes, with
 *                      RF_NOISE_CLIPPED and for rendered images).  The
 *                      autotuner times both. */
#define RF_TUNE_FUSED 4
/* RF_TUNE_RING         chunk slots of the fused pass's ring, 2 .. 8
 *                      (default 3). */
#define RF_TUNE_RING 5
/* RF_TUNE_OVERLAP      1: waves hold at most half of RF_TUNE_WAVE_IMAGES
 *                      images and alternate between the two halves of the
 *                      scratch, so that one wave's gridding and column pass
 *                      run on the caller's stream while the previous wave's
 *                      row pass and finalize run on a second stream of the
 *                      plan (the column pass at the higher priority, at most
 *                      one of its blocks per SM, the row pass in short
 *                      blocks that take the rest); the caller's stream waits
 *                      for both before the call returns.  0 (default): one
 *                      wave after another on the caller's stream.  Without
 *                      effect with RF_TUNE_FUSED, RF_NOISE_CLIPPED and for
 *                      rendered images.  The autotuner times both. */
#define RF_TUNE_OVERLAP 6
rf_status rf_plan_set_tuning(struct rf_plan* plan, int32_t key, int64_t value);
rf_status rf_plan_get_tuning(const struct rf_plan* plan, int32_t key, int64_t* value);

/*
 * rf_plan_autotune: pick the tuning that searches `vis` fastest and apply
 * it.  Candidates: where the fused pass exists (npix 1024 .. 4096, no
 * clipped noise), RF_TUNE_FUSED on with RF_TUNE_RING 2, 3 and 4, and off with
 * RF_TUNE_OVERLAP off and on, at waves of 2048 and 8192 images, graphs on;
 * elsewhere a ladder of wave sizes (256 .. 8192 images) with RF_TUNE_GRAPHS
 * on and off, and from 2048 images RF_TUNE_OVERLAP on.  Before either, waves
 * of one, two and four image groups (below 256 images) whose column-FFT
 * buffer fits the device's L2 cache, separate passes, graphs on.  Wave sizes whose
 * column-FFT buffer would not fit in half the free device memory are
 * skipped.  Each candidate is timed with CUDA events on `stream`, after one
 * warm-up, on a search of the segment in which every (DM, dt) is limited to
 * its first nint/4 integrations (the full search for short segments).  vis
 * and nint as for rf_search_segment.  `report` (may be NULL) receives what
 * was tried (at most 16 entries).  Results of the search do not depend on
 * the tuning.  Errors: as rf_search_segment.
 */
typedef struct rf_tune_report {
  int32_t best_wave_images;
  int32_t best_graphs;
  int32_t ntried;
  int32_t tried_wave_images[16];
  int32_t tried_graphs[16];
  float tried_ms[16];
  int32_t best_fused;
  int32_t best_ring;
  int32_t tried_fused[16];
  int32_t tried_ring[16];
  int32_t best_overlap;
  int32_t tried_overlap[16];
} rf_tune_report;
rf_status rf_plan_autotune(struct rf_plan* plan, const void* vis, int32_t nint, void* stream,
                           rf_tune_report* report);

/* Derived facts of a plan (see rf_plan_info). */
rf_status rf_plan_get_info(const struct rf_plan* plan, rf_plan_info* info);

/* Copy the delay table, [ndm][nchan] int32 integrations, to host `out`. */
rf_status rf_plan_delays(const struct rf_plan* plan, int32_t* out);

/* Copy the nearest cells, [nbl][nchan] each, to host arrays (any may be NULL):
 * iu, iv the unfolded cell indices and ongrid 1 if |iu| < N/2 and |iv| < N/2. */
rf_status rf_plan_cells(const struct rf_plan* plan, int32_t* iu, int32_t* iv, uint8_t* ongrid);

/* Number of images the search makes for a segment of nint integrations. */
rf_status rf_count_images(const struct rf_plan* plan, int32_t nint, int64_t* n_images);

/*
 * Per-kernel timing.  With profiling enabled a plan brackets every kernel
 * launch (and host-to-device copy) it issues with a pair of CUDA events on
 * the caller's stream and, when the call has synchronised, adds the elapsed
 * time to a per-kernel total.  The totals cover every call since profiling
 * was last enabled.  rf_plan_get_profile fills up to `cap` records and sets
 * *n to the number of kernel kinds.
 */
typedef struct rf_kernel_profile {
  char name[32];
  int64_t launches;
  double total_ms;
} rf_kernel_profile;

rf_status rf_plan_set_profiling(struct rf_plan* plan, int32_t enable);
rf_status rf_plan_get_profile(const struct rf_plan* plan, rf_kernel_profile* out, int32_t cap, int32_t* n);

/*
 * rf_image_stats_noalloc -- an entry point that allocates nothing.  The
 * paper has no counterpart to it: it exists for callers of this library that
 * cannot allocate device memory at the point where they image, such as code
 * recording a CUDA graph (cudaMalloc cannot be captured), a real-time loop
 * that cannot take the allocator's latency or failures, or a host framework
 * that owns the device memory pool.
 *
 * It images one uv half plane and measures the image as the search does:
 *   I[y][x] = (1 / 2W) sum over the Hermitian full plane of
 *             H[v][u] exp(+2 pi i (u (x - N/2) + v (y - N/2)) / N),
 * then peak (lowest y N + x on ties), mean, population sigma and peak/sigma.
 * half_plane  device [npix][npix/2 + 1] complex64 (interleaved float re, im),
 *             row v mod N, column u = 0 .. N/2.  Column 0 must hold the
 *             whole Hermitian column (both v and -v entries); column N/2 is
 *             ignored (treated as empty).
 * npix        a power of two in [16, RF_NOALLOC_MAX_NPIX].  Larger images
 *             are rejected with RF_ERR_INVALID_ARG: the scratch is a static
 *             device array sized for RF_NOALLOC_MAX_NPIX.
 * weight      W > 0, the normalisation of the image (samples gridded).
 * stream      cudaStream_t (NULL = default stream); the call is asynchronous.
 * stat        device pointer to one rf_image_stat (8-byte aligned); dm_idx,
 *             dt_idx and t_idx are written as 0.
 * Both pointers must be device memory of the current device: host memory
 * (pageable or pinned) and memory of another GPU are rejected with
 * RF_ERR_INVALID_ARG before anything is launched (checked with
 * cudaPointerGetAttributes, which allocates nothing).
 * It runs on the current CUDA device and calls no cudaMalloc or cudaFree.
 * Its scratch (the column-FFT intermediate and row partials, about 4 MiB
 * for RF_NOALLOC_MAX_NPIX = 1024) is one static device array per GPU, held
 * until the process exits and shared by every call: calls whose work
 * overlaps on the GPU (other streams, other threads) race on it, so issue
 * them one after another on one stream.  The first call on a device does a
 * one-time set-up (looks up the array's device address and uploads twiddle
 * tables with a synchronous copy); make that first call before any stream
 * capture.  Errors: RF_ERR_INVALID_ARG, RF_ERR_NO_DEVICE, RF_ERR_CUDA.
 */
#define RF_NOALLOC_MAX_NPIX 1024
rf_status rf_image_stats_noalloc(const void* half_plane, int32_t npix, double weight, void* stream,
                                 rf_image_stat* stat);

/* ---- serving --------------------------------------------------------
 * A server keeps plans resident on one device and searches segments as they
 * arrive (Sec. 3.2: segments are independent and are processed as they are
 * read; the state of each is fixed by its metadata and preferences).  Each
 * of `slots` workers runs one segment at a time on its own CUDA stream, so
 * segments admitted together overlap on the device.  Admission is in
 * arrival order: the oldest waiting segment starts when a worker is free and
 * its plan is resident and idle, or a new plan for it fits in the HBM budget
 * (idle resident plans are evicted least-recently-used first).
 */
typedef struct rf_server_desc {
  int32_t device;            /* CUDA device ordinal                          */
  int32_t slots;             /* segments in flight at once, 1 .. 16          */
  uint64_t hbm_budget_bytes; /* device memory the server's plans may hold     */
  int64_t wave_images;       /* RF_TUNE_WAVE_IMAGES for its plans (0 = default) */
} rf_server_desc;

/* Outcome and timing of one request; times in seconds since the server
 * was created (steady clock). */
typedef struct rf_request_info {
  int32_t status;     /* rf_status of the search (valid once done)          */
  int32_t done;       /* 1 when the search has finished                     */
  double submit_s;    /* when rf_server_submit accepted it                  */
  double start_s;     /* when a worker started it                           */
  double done_s;      /* when its candidates were on the host               */
  int64_t n_images;   /* images searched                                    */
  uint64_t n_candidates;
  int32_t plan_reused; /* 1 if a resident plan was used                     */
} rf_request_info;

rf_status rf_server_create(const rf_server_desc* desc, struct rf_server** out);

/* Queue one segment.  `desc` is copied (max_nint is taken as the plan's);
 * `vis` (host or device, layout as for rf_search_segment) must stay valid
 * and unchanged until the request is done.  *ticket identifies it.
 * Errors: RF_ERR_INVALID_ARG, RF_ERR_SHAPE (nint > desc->max_nint),
 * RF_ERR_NO_MEMORY (the plan cannot fit in the budget at all). */
rf_status rf_server_submit(struct rf_server* server, const rf_plan_desc* desc, const void* vis, int32_t nint,
                           int64_t* ticket);

/* Wait up to timeout_ms (negative: no limit) for the request to finish and
 * fill `info`.  Returns RF_ERR_TIMEOUT if it is still running (info then
 * has done = 0), RF_ERR_INVALID_ARG for an unknown ticket. */
rf_status rf_server_wait(struct rf_server* server, int64_t ticket, int32_t timeout_ms, rf_request_info* info);

/* Copy the candidates of a finished request (sorted as rf_search_segment)
 * and forget the request.  If n_out > cap the first cap are written and
 * RF_ERR_CAPACITY is returned (the request is kept). */
rf_status rf_server_results(struct rf_server* server, int64_t ticket, rf_candidate* out, size_t cap,
                            size_t* n_out);

/* Finish all queued work, then free the server and its plans. */
rf_status rf_server_destroy(struct rf_server* server);

/* ---- candidate products ----------------------------------------------
 * Statistics measured from each candidate's image and spectrum (Sec. 3.3:
 * kept for every candidate above a low threshold, about 6 sigma), and the
 * image and spectrum themselves (Sec. 3.3: candidate plots, above about
 * 7 sigma).  Which candidates get which product is the caller's choice.
 *
 * Spectrum of candidate (dm_idx, dt_idx, t_idx) at pixel (x, y): per channel
 * c (in the plan's channel order), the dedispersed, resampled visibilities
 * phased to (x, y) with the image's own cell phases
 * exp(+2 pi i (iu (x - N/2) + iv (y - N/2)) / N), summed over the on-grid
 * baselines and divided by w_c = (on-grid baselines at c) * (samples
 * present); 0 where w_c = 0.  Its w-weighted mean real part equals the image
 * value at (x, y).  Moments are population moments in FP64: image moments
 * over all N^2 pixels, spectrum moments over Re(spectrum) at the channels
 * with w_c > 0; kurtosis is the excess kurtosis m4 / m2^2 - 3.
 */
typedef struct rf_candidate_features {
  int32_t dm_idx;
  int32_t dt_idx;
  int32_t t_idx;
  int32_t x;
  int32_t y;
  int32_t nchan_used;        /* channels with w_c > 0                        */
  double image_mean;
  double image_sigma;
  double image_skew;
  double image_kurtosis;
  double spec_mean;
  double spec_std;
  double spec_skew;
  double spec_kurtosis;
  double peak_from_spectrum; /* sum_c w_c Re(spec_c) / sum_c w_c           */
} rf_candidate_features;

/* Products of n candidates of a segment (the same vis and nint they were
 * found in; only dm_idx, dt_idx, t_idx, x and y of each are read).
 * features [n] is required; spectra [n][nchan][2] (re, im) FP32 and
 * images [n][N][N] FP32 are written when not NULL.  The segment is ingested
 * again; device scratch is allocated for the call.  Errors:
 * RF_ERR_INVALID_ARG (a trial the plan does not search at nint, a pixel
 * outside the image), RF_ERR_SHAPE, RF_ERR_NO_MEMORY, RF_ERR_BUSY. */
rf_status rf_candidate_products(struct rf_plan* plan, const void* vis, int32_t nint, void* stream,
                                const rf_candidate* cands, int32_t n, rf_candidate_features* features,
                                float* spectra, float* images);

/* ---- periodicity search ---------------------------------------------
 * Sec. 3.1 (footnote): a time segment is Fourier transformed over time and
 * each fluctuation frequency is imaged to search for periodic signals (Fig. 2:
 * a change of the innermost loop).  For every DM trial whose window fits
 * (max delay + L <= nint) and every (baseline, channel), the dedispersed
 * window x[t] = S[t + delay[d][c]], t < L, gives at fluctuation frequency k
 *   U_k = (1/L) sum_t x[t] cos(2 pi k t / L),  Q_k = (1/L) sum_t x[t] sin(2 pi k t / L).
 * I_U and I_Q are their dirty images (the search's gridding and FFT, weight W =
 * on-grid pairs); imaging the time transform over each baseline and its mirror
 * gives 2 (I_U - i I_Q), so the power image is P = I_U^2 + I_Q^2.  A flux
 * A1 cos(2 pi k t / L + psi) at a pixel gives amplitude sqrt(P) = A1 / 2 there.
 * Per (DM, k): amplitude = sqrt(max P) (lowest pixel index on ties),
 * sigma = sqrt((var(I_U) + var(I_Q)) / 2) (population variances over the N^2
 * pixels), snr = amplitude / sigma; a candidate iff snr >= threshold.
 */
typedef struct rf_periodic_candidate {
  int32_t dm_idx;
  int32_t k;          /* fluctuation frequency index, kmin .. kmax           */
  int32_t x;
  int32_t y;
  float snr;
  float amplitude;
  float sigma;
  float pad;
  double dm;
  double freq_hz;     /* k / (L inttime_s)                                   */
  double l_rad;
  double m_rad;
} rf_periodic_candidate;

/* Periodicity search of one segment (vis and nint as for rf_search_segment).
 * L: window length, a power of two in [16, 8192], L <= nint;
 * 1 <= kmin <= kmax <= L/2; threshold > 0.  Candidates sorted by
 * (dm_idx, k) go to out (RF_ERR_CAPACITY and *n_out = total if cap is too
 * small).  stats (may be NULL) receives every (DM, k) searched, in the same
 * order, with snr etc. set whether or not it is a candidate; *n_stats =
 * (DM trials that fit) * (kmax - kmin + 1).  Device scratch is allocated for
 * the call.  Errors: RF_ERR_INVALID_ARG, RF_ERR_SHAPE, RF_ERR_NO_MEMORY,
 * RF_ERR_BUSY, RF_ERR_CAPACITY, RF_ERR_TIMEOUT (a bounded device-side wait
 * for a row-pass tile copy gave up; the plan stays usable). */
rf_status rf_periodicity_search(struct rf_plan* plan, const void* vis, int32_t nint, int32_t L, int32_t kmin,
                                int32_t kmax, double threshold, void* stream, rf_periodic_candidate* out,
                                size_t cap, size_t* n_out, rf_periodic_candidate* stats, size_t stats_cap,
                                size_t* n_stats);

/* ---- continuous search over overlapping segments ----------------------
 * A stream cuts an unbounded run of integrations into segments that overlap
 * by the plan's longest dispersion sweep (Sec. 3.2: consecutive segments
 * overlap by the maximum sweep so that every pulse lies whole inside one of
 * them).  Segment k holds integrations [k stride, k stride + stride + overlap)
 * with overlap = max over DM trials and channels of the delay; every
 * (DM, dt) searches t' < stride / dt in it, so each start time
 * k stride + t' dt is searched by exactly one segment and its whole sweep is
 * inside that segment.  rf_stream_flush searches what is left (from the next
 * segment start to the last integration pushed) under the plan's edge rule.
 * Without RF_MEAN_SUBTRACT the union of a stream's images is exactly the
 * image set of one rf_search_segment over the whole run; with it, each
 * segment subtracts its own mean.
 *
 * Outputs count t_idx from the start of the run: k stride / dt + t'.
 * The stream holds two device windows of stride + overlap raw integrations
 * ([nint][nbl][nchan][npol] complex64) on the plan's device and uses the
 * plan for its searches; the plan must outlive the stream and may not be
 * searched by another thread while a push or flush runs (RF_ERR_BUSY).  A
 * stream is used by one thread at a time.
 */
/* Keep every searched image's statistics for rf_stream_pop_stats. */
#define RF_STREAM_KEEP_STATS 0x1u

typedef struct rf_stream_info {
  int32_t stride;           /* integrations between segment starts            */
  int32_t overlap;          /* max dispersion delay, integrations             */
  int32_t segment_nint;     /* stride + overlap                               */
  int32_t fill;             /* integrations waiting in the current window     */
  int64_t pushed;           /* integrations pushed since creation or flush    */
  int64_t segments;         /* segments searched since creation or flush      */
  uint64_t pending_candidates;
  uint64_t pending_stats;
} rf_stream_info;

/* stride must be >= 1 and a multiple of every dt of the plan, and
 * stride + overlap <= the plan's max_nint.  Errors: RF_ERR_INVALID_ARG
 * (also for a RF_HOST_ONLY plan), RF_ERR_NO_MEMORY, RF_ERR_CUDA. */
rf_status rf_stream_create(struct rf_plan* plan, int32_t stride, uint32_t flags, struct rf_stream** out);

/* Append nint integrations (host or device memory, layout as for
 * rf_search_segment) and search every segment they complete, in order, on
 * `stream` (NULL: the default stream).  Returns when those searches are
 * done; their candidates (and stats) are queued.  *n_segments (may be NULL)
 * = segments searched by this call. */
rf_status rf_stream_push(struct rf_stream* s, const void* vis, int32_t nint, void* stream, int32_t* n_segments);

/* Search the integrations still in the window (if any) as the last segment
 * under the plan's edge rule, then start a new run (t_idx from 0 again). */
rf_status rf_stream_flush(struct rf_stream* s, void* stream, int32_t* n_segments);

/* Move up to cap queued candidates (oldest segment first, each segment's
 * sorted by (dm_idx, dt_idx, t_idx)) into out; *n_out = number moved. */
rf_status rf_stream_pop(struct rf_stream* s, rf_candidate* out, size_t cap, size_t* n_out);

/* Same for image statistics (only with RF_STREAM_KEEP_STATS). */
rf_status rf_stream_pop_stats(struct rf_stream* s, rf_image_stat* out, size_t cap, size_t* n_out);

rf_status rf_stream_get_info(const struct rf_stream* s, rf_stream_info* out);

/* Free the windows and queues (NULL-safe).  The plan is not destroyed. */
rf_status rf_stream_destroy(struct rf_stream* s);

/* Check of the bounded device-side waits (no counterpart in the paper): one
 * block waits, at most `polls` polls (1 .. 2^20) each, on an mbarrier that
 * nothing arrives at, as the row pass waits for its tile copies, and on a
 * global count that nothing raises, as the fused imaging pass waits for
 * work items of other blocks.  Both waits must give up and report it
 * instead of hanging: *gave_up = 1.  The device stays usable afterwards.
 * Errors: RF_ERR_INVALID_ARG, RF_ERR_NO_DEVICE, RF_ERR_CUDA. */
rf_status rf_selftest_bounded_wait(int32_t device, int32_t polls, int32_t* gave_up);

/* Library version string. */
const char* rf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* REALFAST_GB300_H */
